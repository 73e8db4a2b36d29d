// Counter-based Poisson noise (paper Sec. II.G-H: Poisson sampling of the
// counts reaching each pixel, flood scaled to H photons per pixel).
//
// The sampler is specified operation by operation in binary32 so that any
// implementation that follows it returns identical bits for identical rates:
//   * random words: Philox4x32-10 [Salmon et al., SC'11], key (seed low
//     word, seed high word), counter (iu, iv, projection k, block j);
//   * uniform from a word w: (2 (w >> 9) + 1) 2^-24, exactly representable;
//   * rate <= 0 or NaN -> 0; rate > 1e7 -> floor(rate + 1/2);
//   * rate < 10: inversion by sequential search (one uniform);
//   * rate >= 10: transformed rejection with squeeze, PTRS [Hormann 1993],
//     two uniforms per attempt, at most 64 attempts;
//   * log and exp are this file's own series (atanh series of the mantissa,
//     Taylor polynomial after Cody-Waite reduction), evaluated with the
//     correctly rounded intrinsics below so the compiler cannot fuse or
//     reorder them.
#pragma once

#include <stdint.h>

namespace fc {
namespace noise {

#define FADD __fadd_rn
#define FSUB __fsub_rn
#define FMUL __fmul_rn
#define FDIV __fdiv_rn

// The ten round keys of Philox4x32-10 for one seed (the key bumped by the
// Weyl constants after every round), built on the host and passed as a kernel
// parameter so that each round's xor takes its key from the constant bank.
struct PhiloxKeys {
    uint32_t x[10], y[10];
};

inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys k;
    uint32_t kx = (uint32_t)seed, ky = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.x[r] = kx;
        k.y[r] = ky;
        kx += 0x9E3779B9u;
        ky += 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x[r], lo1, hi0 ^ c.w ^ k.y[r], lo0);
    }
    return c;
}

// (2 (w >> 9) + 1) 2^-24 without an integer-to-float conversion: the bits of
// 1 + m 2^-23 (m = w >> 9), minus 1 (exact), plus 2^-24 (exact: the sum has at
// most 24 significant bits), so the value is the one the formula defines.
__device__ __forceinline__ float unif(uint32_t w)
{
    const float f = __uint_as_float(0x3f800000u | (w >> 9));
    return FADD(FSUB(f, 1.0f), 5.9604644775390625e-08f);
}

// natural log of a positive normal binary32 value
__device__ __forceinline__ float log_f32(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421354f) { m = FMUL(m, 0.5f); e = e + 1; }
    const float f = FSUB(m, 1.0f);
    const float s = FDIV(f, FADD(2.0f, f));
    const float z = FMUL(s, s);
    float acc = 0.0769230798f;
    acc = FADD(0.0909090936f, FMUL(z, acc));
    acc = FADD(0.111111112f, FMUL(z, acc));
    acc = FADD(0.142857149f, FMUL(z, acc));
    acc = FADD(0.200000003f, FMUL(z, acc));
    acc = FADD(0.333333343f, FMUL(z, acc));
    const float R = FMUL(z, acc);
    float t = FMUL(s, R);
    t = FADD(s, t);
    const float logm = FMUL(2.0f, t);
    const float ef = __int2float_rn(e);
    float lo = FMUL(ef, 1.42860677e-06f);
    lo = FADD(lo, logm);
    const float hi = FMUL(ef, 0.693145752f);
    return FADD(hi, lo);
}

// exp(x) for |x| < 80
__device__ __forceinline__ float exp_f32(float x)
{
    const float n = floorf(FADD(FMUL(x, 1.44269502f), 0.5f));
    float r = FSUB(x, FMUL(n, 0.693145752f));
    r = FSUB(r, FMUL(n, 1.42860677e-06f));
    float acc = 2.75573188e-06f;
    acc = FADD(2.48015876e-05f, FMUL(r, acc));
    acc = FADD(1.98412701e-04f, FMUL(r, acc));
    acc = FADD(1.38888892e-03f, FMUL(r, acc));
    acc = FADD(8.33333377e-03f, FMUL(r, acc));
    acc = FADD(4.16666679e-02f, FMUL(r, acc));
    acc = FADD(0.166666672f, FMUL(r, acc));
    acc = FADD(0.5f, FMUL(r, acc));
    acc = FADD(1.0f, FMUL(r, acc));
    const float p = FADD(1.0f, FMUL(r, acc));
    const int ni = (int)n;
    return FMUL(p, __uint_as_float((uint32_t)(ni + 127) << 23));
}

// D(k, lam) = k log(k / lam) + lam - k
__device__ __forceinline__ float deviance(float kf, float lam)
{
    const float diff = FSUB(kf, lam);
    const float sum = FADD(kf, lam);
    const float v = FDIV(diff, sum);
    if (fabsf(v) < 0.5f) {
        const float v2 = FMUL(v, v);
        float acc = 0.0399999991f;
        acc = FADD(0.0434782617f, FMUL(v2, acc));
        acc = FADD(0.0476190485f, FMUL(v2, acc));
        acc = FADD(0.0526315793f, FMUL(v2, acc));
        acc = FADD(0.0588235296f, FMUL(v2, acc));
        acc = FADD(0.0666666701f, FMUL(v2, acc));
        acc = FADD(0.0769230798f, FMUL(v2, acc));
        acc = FADD(0.0909090936f, FMUL(v2, acc));
        acc = FADD(0.111111112f, FMUL(v2, acc));
        acc = FADD(0.142857149f, FMUL(v2, acc));
        acc = FADD(0.200000003f, FMUL(v2, acc));
        acc = FADD(0.333333343f, FMUL(v2, acc));
        const float S = FMUL(v2, acc);
        float t = FMUL(kf, v);
        t = FMUL(t, S);
        t = FMUL(2.0f, t);
        const float d = FMUL(diff, v);
        return FADD(d, t);
    }
    float t = FDIV(kf, lam);
    t = log_f32(t);
    t = FMUL(kf, t);
    t = FADD(t, lam);
    return FSUB(t, kf);
}

__device__ __forceinline__ float log_pmf(float kf, float lam, float loglam)
{
    if (kf < 10.0f) {
        float lf = 0.0f;
        for (float i = 2.0f; i <= kf; i = FADD(i, 1.0f)) lf = FADD(lf, log_f32(i));
        float t = FMUL(kf, loglam);
        t = FSUB(t, lam);
        return FSUB(t, lf);
    }
    const float D = deviance(kf, lam);
    const float ik = FDIV(1.0f, kf);
    const float ik2 = FMUL(ik, ik);
    float dl = FMUL(ik2, 7.93650805e-04f);
    dl = FSUB(2.77777785e-03f, dl);
    dl = FMUL(ik2, dl);
    dl = FSUB(0.0833333358f, dl);
    dl = FMUL(ik, dl);
    float h = log_f32(kf);
    h = FMUL(0.5f, h);
    h = FADD(0.918938518f, h);
    const float r = FSUB(-D, h);
    return FSUB(r, dl);
}

// State of one transformed-rejection draw between attempts.
struct Ptrs {
    float lam, b, a, vr, loglam, invalpha;
    uint4 w;            // Philox block j
    uint32_t iu, iv, k, j;
    const PhiloxKeys *key;   // round keys of the seed (kernel parameter)
    int h;              // 0: attempt uses words (x, y) of block j, 1: words (z, w)
    bool have_slow;     // loglam and invalpha evaluated
};

// First stage of a draw.  Returns true with the count in r when it is decided
// without rejection sampling (rate <= 0 or NaN, rate > 1e7, rate < 10);
// otherwise prepares s for ptrs_attempt.
__device__ __forceinline__ bool poisson_begin(float lam, uint32_t iu, uint32_t iv, uint32_t k,
                                              const PhiloxKeys &key, Ptrs &s, float &r)
{
    if (!(lam > 0.0f)) { r = 0.0f; return true; }
    if (lam > 1.0e7f) { r = floorf(FADD(lam, 0.5f)); return true; }
    if (lam < 10.0f) {
        const uint4 w = philox4x32_10(make_uint4(iu, iv, k, 0u), key);
        const float u = unif(w.x);
        float p = exp_f32(-lam);
        float F = p, kf = 0.0f;
        while (u > F) {
            kf = FADD(kf, 1.0f);
            p = FMUL(p, lam);
            p = FDIV(p, kf);
            const float Fn = FADD(F, p);
            if (Fn == F) break;
            F = Fn;
        }
        r = kf;
        return true;
    }
    // log(lam) and 1/alpha only enter the final acceptance test; they are
    // evaluated when first needed (same values, fewer operations).
    const float slam = __fsqrt_rn(lam);
    float b = FMUL(2.53f, slam);
    b = FADD(0.931f, b);
    float a = FMUL(0.02483f, b);
    a = FADD(-0.059f, a);
    float vr = FSUB(b, 2.0f);
    vr = FDIV(3.6224f, vr);
    vr = FSUB(0.9277f, vr);
    s.lam = lam; s.b = b; s.a = a; s.vr = vr;
    s.loglam = 0.0f; s.invalpha = 0.0f; s.have_slow = false;
    s.iu = iu; s.iv = iv; s.k = k; s.j = 0; s.h = 0; s.key = &key;
    return false;
}

// Moves to the next attempt after a rejection; returns true with
// r = floor(lam + 1/2) when the 64-attempt limit is reached.
__device__ __forceinline__ bool ptrs_advance(Ptrs &s, float &r)
{
    if (s.h) {
        s.h = 0;
        if (++s.j == 32u) { r = floorf(FADD(s.lam, 0.5f)); return true; }
    } else {
        s.h = 1;
    }
    return false;
}

enum { kDone = 0, kReject = 1, kPending = 2 };

// First part of one PTRS attempt: the squeeze and the quick rejections.
// kDone: decided (r holds the count); kReject: rejected and the state moved
// to the next attempt; kPending: the final acceptance test must be made with
// ptrs_final(kf, us, V) before anything else happens to this draw.
__device__ __forceinline__ int ptrs_quick(Ptrs &s, float &r, float &kf_out, float &us_out,
                                          float &V_out)
{
    if (s.h == 0) s.w = philox4x32_10(make_uint4(s.iu, s.iv, s.k, s.j), *s.key);
    const float U = FSUB(unif(s.h ? s.w.z : s.w.x), 0.5f);
    const float V = unif(s.h ? s.w.w : s.w.y);
    const float us = FSUB(0.5f, fabsf(U));
    float t = FMUL(2.0f, s.a);
    t = FDIV(t, us);
    t = FADD(t, s.b);
    t = FMUL(t, U);
    t = FADD(t, s.lam);
    t = FADD(t, 0.43f);
    const float kf = floorf(t);
    if (us >= 0.07f && V <= s.vr) { r = kf; return kDone; }
    if (kf < 0.0f || (us < 0.013f && V > us)) return ptrs_advance(s, r) ? kDone : kReject;
    kf_out = kf;
    us_out = us;
    V_out = V;
    return kPending;
}

// Final acceptance test of a pending attempt: log(V / (alpha (a / us^2 + b)))
// against log P(k; lam).  Returns true when the draw is decided.
__device__ __forceinline__ bool ptrs_final(Ptrs &s, float kf, float us, float V, float &r)
{
    if (!s.have_slow) {
        s.loglam = log_f32(s.lam);
        float ia = FSUB(s.b, 3.4f);
        ia = FDIV(1.1328f, ia);
        s.invalpha = FADD(1.1239f, ia);
        s.have_slow = true;
    }
    float den = FMUL(us, us);
    den = FDIV(s.a, den);
    den = FADD(den, s.b);
    float q = FMUL(V, s.invalpha);
    q = FDIV(q, den);
    const float lhs = log_f32(q);
    if (lhs <= log_pmf(kf, s.lam, s.loglam)) { r = kf; return true; }
    return ptrs_advance(s, r);
}

// One complete PTRS attempt; returns true when the draw is decided.
__device__ __forceinline__ bool ptrs_attempt(Ptrs &s, float &r)
{
    float kf, us, V;
    const int q = ptrs_quick(s, r, kf, us, V);
    if (q == kDone) return true;
    if (q == kReject) return false;
    return ptrs_final(s, kf, us, V, r);
}

// Complete draw for pixel (iu, iv) of projection k.
__device__ __forceinline__ float poisson(float lam, uint32_t iu, uint32_t iv, uint32_t k,
                                         const PhiloxKeys &seed)
{
    Ptrs s;
    float r;
    if (poisson_begin(lam, iu, iv, k, seed, s, r)) return r;
    while (!ptrs_attempt(s, r)) {
    }
    return r;
}

#undef FADD
#undef FSUB
#undef FMUL
#undef FDIV

}  // namespace noise
}  // namespace fc

/*
 * Poisson detector noise -- CPU reference -- TEST INFRASTRUCTURE ONLY.
 *
 * Sec. II.G / II.H of the paper: noise is added by Poisson sampling of the
 * particle counts reaching each detector pixel, the flood scaled to a height
 * H photons per pixel.  The draw decides an integer, so this reference takes
 * it in the same precision as the GPU kernel (IEEE binary32), with only the
 * correctly rounded operations + - * / sqrt, floor and comparisons, in a
 * fixed order; compile with -ffp-contract=off so no multiply-add is fused.
 * Two implementations written to this specification return identical bits
 * for identical rate arrays.
 *
 * Specification (all arithmetic binary32 unless stated):
 *   Random words: Philox4x32-10 [Salmon, Moraes, Dror, Shaw, SC'11] with
 *   key (seed mod 2^32, seed div 2^32) and counter (iu, iv, k, j), block
 *   j = 0, 1, ... for pixel (iu, iv) of projection k.
 *   Uniform from a 32-bit word w:  u = (2 * (w >> 9) + 1) * 2^-24, in (0, 1).
 *   Rate lam <= 0 or NaN: 0.  lam > 1e7: floor(lam + 0.5).
 *   lam < 10: inversion by sequential search with u = block 0, word 0:
 *       p = exp(-lam), F = p, k = 0; while u > F: k += 1, p = (p * lam) / k,
 *       stop if F + p == F, else F = F + p.
 *   lam >= 10: transformed rejection with squeeze, PTRS [Hormann 1993],
 *       attempts 2j and 2j+1 use words (0, 1) and (2, 3) of block j, for at
 *       most 64 attempts, then floor(lam + 0.5).  The final acceptance test
 *       compares log(V * alpha^-1 / (a / us^2 + b)) with log P(k; lam), the
 *       latter written -D(k, lam) - log(2 pi k) / 2 - delta(k) for k >= 10
 *       (D = k log(k / lam) + lam - k, delta = Stirling remainder) and
 *       k log lam - lam - sum_{i=2..k} log i for k < 10.
 *   log, exp: own routines (atanh series / Taylor series with Cody-Waite
 *   argument reduction), see below.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ---------------- Philox4x32-10 (Salmon et al. 2011) ---------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static float unif(uint32_t w)
{
    return (float)(((w >> 9) << 1) | 1u) * 5.9604644775390625e-08f; /* 2^-24 */
}

static float bits_f(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t f_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* Natural log of a positive normal float: x = m 2^e with m in [sqrt(1/2),
 * sqrt(2)); log m = 2 atanh(s), s = (m - 1) / (m + 1), series to s^13;
 * e ln2 with ln2 split in a 16-bit head and a tail. */
float orc_log_f32(float x)
{
    uint32_t b = f_bits(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float m = bits_f((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421354f) { m = m * 0.5f; e = e + 1; }
    float f = m - 1.0f;
    float s = f / (2.0f + f);
    float z = s * s;
    float acc = 0.0769230798f;            /* 1/13 */
    acc = 0.0909090936f + z * acc;        /* 1/11 */
    acc = 0.111111112f + z * acc;         /* 1/9  */
    acc = 0.142857149f + z * acc;         /* 1/7  */
    acc = 0.200000003f + z * acc;         /* 1/5  */
    acc = 0.333333343f + z * acc;         /* 1/3  */
    float R = z * acc;
    float t = s * R;
    t = s + t;
    float logm = 2.0f * t;
    float ef = (float)e;
    float lo = ef * 1.42860677e-06f;      /* ln2 - ln2_hi */
    lo = lo + logm;
    float hi = ef * 0.693145752f;         /* ln2_hi = 45426 / 65536 */
    return hi + lo;
}

/* exp(x) for |x| < 80: n = round(x / ln2), r = x - n ln2 (two-part
 * reduction), Taylor polynomial of degree 9 at r, times 2^n. */
float orc_exp_f32(float x)
{
    float n = floorf(x * 1.44269502f + 0.5f);
    float r = x - n * 0.693145752f;
    r = r - n * 1.42860677e-06f;
    float acc = 2.75573188e-06f;          /* 1/9! */
    acc = 2.48015876e-05f + r * acc;      /* 1/8! */
    acc = 1.98412701e-04f + r * acc;      /* 1/7! */
    acc = 1.38888892e-03f + r * acc;      /* 1/6! */
    acc = 8.33333377e-03f + r * acc;      /* 1/5! */
    acc = 4.16666679e-02f + r * acc;      /* 1/4! */
    acc = 0.166666672f + r * acc;         /* 1/3! */
    acc = 0.5f + r * acc;                 /* 1/2! */
    acc = 1.0f + r * acc;                 /* 1/1! */
    float p = 1.0f + r * acc;
    int ni = (int)n;
    return p * bits_f((uint32_t)(ni + 127) << 23);
}

/* D(k, lam) = k log(k / lam) + lam - k >= 0 (saddle-point deviance). */
static float deviance(float kf, float lam)
{
    float diff = kf - lam;
    float sum = kf + lam;
    float v = diff / sum;
    if (fabsf(v) < 0.5f) {
        /* k log(k/lam) = 2k atanh(v) = 2k (v + v^3/3 + ...); the linear
         * term combines with lam - k into diff * v. */
        float v2 = v * v;
        float acc = 0.0399999991f;        /* 1/25 */
        acc = 0.0434782617f + v2 * acc;   /* 1/23 */
        acc = 0.0476190485f + v2 * acc;   /* 1/21 */
        acc = 0.0526315793f + v2 * acc;   /* 1/19 */
        acc = 0.0588235296f + v2 * acc;   /* 1/17 */
        acc = 0.0666666701f + v2 * acc;   /* 1/15 */
        acc = 0.0769230798f + v2 * acc;   /* 1/13 */
        acc = 0.0909090936f + v2 * acc;   /* 1/11 */
        acc = 0.111111112f + v2 * acc;    /* 1/9  */
        acc = 0.142857149f + v2 * acc;    /* 1/7  */
        acc = 0.200000003f + v2 * acc;    /* 1/5  */
        acc = 0.333333343f + v2 * acc;    /* 1/3  */
        float S = v2 * acc;
        float t = kf * v;
        t = t * S;
        t = 2.0f * t;
        float d = diff * v;
        return d + t;
    }
    float t = kf / lam;
    t = orc_log_f32(t);
    t = kf * t;
    t = t + lam;
    return t - kf;
}

static float log_pmf(float kf, float lam, float loglam)
{
    if (kf < 10.0f) {
        float lf = 0.0f;
        for (float i = 2.0f; i <= kf; i = i + 1.0f) lf = lf + orc_log_f32(i);
        float t = kf * loglam;
        t = t - lam;
        return t - lf;
    }
    float D = deviance(kf, lam);
    float ik = 1.0f / kf;
    float ik2 = ik * ik;
    float dl = ik2 * 7.93650805e-04f;     /* 1/1260 */
    dl = 2.77777785e-03f - dl;            /* 1/360  */
    dl = ik2 * dl;
    dl = 0.0833333358f - dl;              /* 1/12   */
    dl = ik * dl;
    float h = orc_log_f32(kf);
    h = 0.5f * h;
    h = 0.918938518f + h;                 /* log(2 pi) / 2 */
    float r = -D - h;
    return r - dl;
}

float orc_poisson_one(float lam, uint32_t iu, uint32_t iv, uint32_t k, uint64_t seed)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {iu, iv, k, 0u}, w[4];
    if (!(lam > 0.0f)) return 0.0f;
    if (lam > 1.0e7f) return floorf(lam + 0.5f);
    if (lam < 10.0f) {
        orc_philox4x32_10(ctr, key, w);
        float u = unif(w[0]);
        float p = orc_exp_f32(-lam);
        float F = p, kf = 0.0f;
        while (u > F) {
            kf = kf + 1.0f;
            p = p * lam;
            p = p / kf;
            float Fn = F + p;
            if (Fn == F) break;
            F = Fn;
        }
        return kf;
    }
    float slam = sqrtf(lam);
    float loglam = orc_log_f32(lam);
    float b = 2.53f * slam;
    b = 0.931f + b;
    float a = 0.02483f * b;
    a = -0.059f + a;
    float invalpha = b - 3.4f;
    invalpha = 1.1328f / invalpha;
    invalpha = 1.1239f + invalpha;
    float vr = b - 2.0f;
    vr = 3.6224f / vr;
    vr = 0.9277f - vr;
    for (uint32_t j = 0; j < 32u; ++j) {
        ctr[3] = j;
        orc_philox4x32_10(ctr, key, w);
        for (int h = 0; h < 2; ++h) {
            float U = unif(w[2 * h]) - 0.5f;
            float V = unif(w[2 * h + 1]);
            float us = 0.5f - fabsf(U);
            float t = 2.0f * a;
            t = t / us;
            t = t + b;
            t = t * U;
            t = t + lam;
            t = t + 0.43f;
            float kf = floorf(t);
            if (us >= 0.07f && V <= vr) return kf;
            if (kf < 0.0f || (us < 0.013f && V > us)) continue;
            float den = us * us;
            den = a / den;
            den = den + b;
            float q = V * invalpha;
            q = q / den;
            float lhs = orc_log_f32(q);
            if (lhs <= log_pmf(kf, lam, loglam)) return kf;
        }
    }
    return floorf(lam + 0.5f);
}

/* Counts K[k][iv][iu] ~ Poisson(lam[k][iv][iu]) for projections
 * k = k0 .. k0 + na - 1. */
void orc_poisson(const float *lam, int na, int nv, int nu, int k0, uint64_t seed,
                 float *out)
{
#pragma omp parallel for
    for (int k = 0; k < na; ++k)
        for (int iv = 0; iv < nv; ++iv)
            for (int iu = 0; iu < nu; ++iu) {
                size_t i = ((size_t)k * nv + iv) * nu + iu;
                out[i] = orc_poisson_one(lam[i], (uint32_t)iu, (uint32_t)iv,
                                         (uint32_t)(k0 + k), seed);
            }
}

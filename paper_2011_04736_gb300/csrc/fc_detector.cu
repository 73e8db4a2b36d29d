// Detector response: optical spread + scatter (paper Sec. II.E and II.G --
// intensity profiles convolved with the optical spread function, scatter
// added) and Poisson noise (Sec. II.H).
//
//   I = N0 (G_psf (x) T + SPR G_scatter (x) T),   K = Poisson(I)
//
// Both kernels are sampled Gaussians, separable and clamp-to-edge, so the
// paper's per-energy convolution followed by the energy sum equals one
// convolution of the energy-summed signal (linearity).  Two passes:
//   rows:    one CTA per detector row; the row (plus clamped halo) is staged
//            in shared memory and each thread produces 8 adjacent outputs of
//            both kernels from a sliding register window (8 FMAs per shared
//            load; the shared row is skewed by one word per 32 so the
//            stride-8 lane pattern is free of bank conflicts);
//   columns: one CTA per (projection, tile of TW columns); both row-pass
//            results are staged with replicated halos, each thread produces
//            8 adjacent outputs of one column, and the epilogue forms I.
// Poisson counts are drawn by k_poisson (a round phase of first attempts and
// a per-warp queue of the undecided draws).
#include <math.h>

#include "fc_internal.cuh"
#include "fc_noise.cuh"

namespace fc {

namespace {

constexpr int kOut = 8;       // outputs per thread (sliding window length)
constexpr int kRowThreads = 256;
constexpr int kColThreads = 256;

__device__ __forceinline__ int skew(int i) { return i + (i >> 5); }

// acc[o] += sum_j taps[j] * x[base + o + j], x read through the skewed row.
__device__ __forceinline__ void row_conv(const float *__restrict__ srow, int base,
                                         const float *taps, int ntaps, float (&acc)[kOut])
{
    float win[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) win[o] = srow[skew(base + o)];
    int j = 0;
    for (; j + kOut <= ntaps; j += kOut) {
#pragma unroll
        for (int q = 0; q < kOut; ++q) {
            const float gj = taps[j + q];
#pragma unroll
            for (int o = 0; o < kOut; ++o) acc[o] = fmaf(gj, win[(o + q) % kOut], acc[o]);
            win[q] = srow[skew(base + j + q + kOut)];
        }
    }
    // remaining taps: window is rotated by (j % kOut) == 0 here
    for (int q = 0; j + q < ntaps; ++q) {
        const float gj = taps[j + q];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            acc[o] = fmaf(gj, srow[skew(base + j + q + o)], acc[o]);
        }
    }
}

// Transposed clamp-to-edge pass, edge terms.  The forward pass read input 0
// for every tap j of output s with s + j < 0, so the transpose adds to output
// 0 the sum over s < r of x[s] times the mass of those taps,
//     sum_s x[s] sum_{i <= r - 1 - s} g[i] = sum_s g[r - 1 - s] P[s],
// P[s] = x[0] + ... + x[s]; the last output takes the mirror image.  x(s)
// returns the zero-padded staged input at s.
template <class X>
__device__ __forceinline__ float fold_lo(X x, const float *g, int r)
{
    float P = 0.0f, f = 0.0f;
    for (int s = 0; s < r; ++s) {
        P += x(s);
        f = fmaf(g[r - 1 - s], P, f);
    }
    return f;
}

template <class X>
__device__ __forceinline__ float fold_hi(X x, const float *g, int r, int n)
{
    float Q = 0.0f, f = 0.0f;
    for (int d = 0; d < r; ++d) {
        Q += x(n - 1 - d);
        f = fmaf(g[r + 1 + d], Q, f);
    }
    return f;
}

}  // namespace

// ADJ: the transposed pass (zero padding instead of clamped indices, plus the
// clamped taps' mass folded onto the first and last output).
template <bool ADJ>
__global__ void __launch_bounds__(kRowThreads)
k_blur_rows(const __grid_constant__ BlurParams p, const float *__restrict__ T,
            float *__restrict__ tp, float *__restrict__ ts)
{
    extern __shared__ float srow[];
    const int R = p.rs > p.rp ? p.rs : p.rp;
    const int n = p.n_u;
    const size_t row = blockIdx.x;
    const float *src = T + row * n;
    const int span = n + 2 * R + 2 * kOut;
    for (int i = threadIdx.x; i < span; i += blockDim.x) {
        int uu = i - R;
        if (ADJ) {
            srow[skew(i)] = uu >= 0 && uu < n ? src[uu] : 0.0f;
        } else {
            uu = uu < 0 ? 0 : (uu > n - 1 ? n - 1 : uu);
            srow[skew(i)] = src[uu];
        }
    }
    __syncthreads();
    for (int u0 = threadIdx.x * kOut; u0 < n; u0 += blockDim.x * kOut) {
        float ap[kOut], as[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) { ap[o] = 0.0f; as[o] = 0.0f; }
        row_conv(srow, u0 + R - p.rp, p.gp, 2 * p.rp + 1, ap);
        row_conv(srow, u0 + R - p.rs, p.gs, 2 * p.rs + 1, as);
        if (ADJ) {
            auto x = [&](int q) { return srow[skew(R + q)]; };
            if (u0 == 0) {
                ap[0] += fold_lo(x, p.gp, p.rp);
                as[0] += fold_lo(x, p.gs, p.rs);
            }
            if (n - 1 >= u0 && n - 1 < u0 + kOut) {
                const float fp = fold_hi(x, p.gp, p.rp, n), fs = fold_hi(x, p.gs, p.rs, n);
#pragma unroll
                for (int o = 0; o < kOut; ++o)
                    if (u0 + o == n - 1) { ap[o] += fp; as[o] += fs; }
            }
        }
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            if (u0 + o < n) {
                tp[row * n + u0 + o] = ap[o];
                ts[row * n + u0 + o] = as[o];
            }
        }
    }
}

// Column pass.  Tile: TW columns x (n_v + 2 R) rows of each row-pass result,
// row stride ST floats.  The 32 / TW column groups of a warp work on rows
// 8 apart; ST is chosen so those rows start 32 / (32 / TW) banks apart
// (ST = 32, 18, 9 for TW = 32, 16, 8), which keeps shared reads conflict-free.
template <int TW, int ST, bool ADJ>
__global__ void __launch_bounds__(kColThreads)
k_blur_cols(const __grid_constant__ BlurParams p, const float *__restrict__ tp,
            const float *__restrict__ ts, float *__restrict__ out)
{
    extern __shared__ float smem[];
    const int nv = p.n_v, nu = p.n_u;
    const int hp = nv + 2 * p.rp + kOut, hs = nv + 2 * p.rs + kOut;
    float *sp = smem;              // [hp][ST]
    float *ss = smem + hp * ST;    // [hs][ST]
    const int img = blockIdx.y;
    const int u_base = blockIdx.x * TW;
    const size_t plane = (size_t)nv * nu;
    const float *gp_src = tp + img * plane;
    const float *gs_src = ts + img * plane;
    const int col = threadIdx.x % TW;
    const int grp = threadIdx.x / TW;
    const int ngrp = kColThreads / TW;
    const int u = u_base + col;
    const int uc = u < nu ? u : nu - 1;
    for (int r = grp; r < hp; r += ngrp) {
        int vv = r - p.rp;
        if (ADJ) {
            sp[r * ST + col] = vv >= 0 && vv < nv ? gp_src[(size_t)vv * nu + uc] : 0.0f;
        } else {
            vv = vv < 0 ? 0 : (vv > nv - 1 ? nv - 1 : vv);
            sp[r * ST + col] = gp_src[(size_t)vv * nu + uc];
        }
    }
    for (int r = grp; r < hs; r += ngrp) {
        int vv = r - p.rs;
        if (ADJ) {
            ss[r * ST + col] = vv >= 0 && vv < nv ? gs_src[(size_t)vv * nu + uc] : 0.0f;
        } else {
            vv = vv < 0 ? 0 : (vv > nv - 1 ? nv - 1 : vv);
            ss[r * ST + col] = gs_src[(size_t)vv * nu + uc];
        }
    }
    __syncthreads();
    for (int v0 = grp * kOut; v0 < nv; v0 += ngrp * kOut) {
        float ap[kOut], as[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) { ap[o] = 0.0f; as[o] = 0.0f; }
        // psf taps over rows v0 + o + j (tile row = v + j)
        {
            float win[kOut];
#pragma unroll
            for (int o = 0; o < kOut; ++o) win[o] = sp[(v0 + o) * ST + col];
            const int nt = 2 * p.rp + 1;
            int j = 0;
            for (; j + kOut <= nt; j += kOut) {
#pragma unroll
                for (int q = 0; q < kOut; ++q) {
                    const float gj = p.gp[j + q];
#pragma unroll
                    for (int o = 0; o < kOut; ++o) ap[o] = fmaf(gj, win[(o + q) % kOut], ap[o]);
                    win[q] = sp[(v0 + j + q + kOut) * ST + col];
                }
            }
            for (int q = 0; j + q < nt; ++q) {
                const float gj = p.gp[j + q];
#pragma unroll
                for (int o = 0; o < kOut; ++o) ap[o] = fmaf(gj, sp[(v0 + j + q + o) * ST + col], ap[o]);
            }
        }
        {
            float win[kOut];
#pragma unroll
            for (int o = 0; o < kOut; ++o) win[o] = ss[(v0 + o) * ST + col];
            const int nt = 2 * p.rs + 1;
            int j = 0;
            for (; j + kOut <= nt; j += kOut) {
#pragma unroll
                for (int q = 0; q < kOut; ++q) {
                    const float gj = p.gs[j + q];
#pragma unroll
                    for (int o = 0; o < kOut; ++o) as[o] = fmaf(gj, win[(o + q) % kOut], as[o]);
                    win[q] = ss[(v0 + j + q + kOut) * ST + col];
                }
            }
            for (int q = 0; j + q < nt; ++q) {
                const float gj = p.gs[j + q];
#pragma unroll
                for (int o = 0; o < kOut; ++o) as[o] = fmaf(gj, ss[(v0 + j + q + o) * ST + col], as[o]);
            }
        }
        if (ADJ) {
            auto xp = [&](int q) { return sp[(q + p.rp) * ST + col]; };
            auto xs = [&](int q) { return ss[(q + p.rs) * ST + col]; };
            if (v0 == 0) {
                ap[0] += fold_lo(xp, p.gp, p.rp);
                as[0] += fold_lo(xs, p.gs, p.rs);
            }
            if (nv - 1 >= v0 && nv - 1 < v0 + kOut) {
                const float fp = fold_hi(xp, p.gp, p.rp, nv), fs = fold_hi(xs, p.gs, p.rs, nv);
#pragma unroll
                for (int o = 0; o < kOut; ++o)
                    if (v0 + o == nv - 1) { ap[o] += fp; as[o] += fs; }
            }
        }
        if (u < nu) {
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
                const int v = v0 + o;
                if (v < nv) {
                    out[img * plane + (size_t)v * nu + u] = p.n0 * (ap[o] + p.spr * as[o]);
                }
            }
        }
    }
}

static size_t col_smem_bytes(const BlurParams &p, int st)
{
    return (size_t)(2 * p.n_v + 2 * p.rp + 2 * p.rs + 2 * kOut) * st * sizeof(float);
}

template <int TW, int ST, bool ADJ>
static cudaError_t launch_cols_tw(const BlurParams &p, const float *tp, const float *ts, float *out,
                                  int n_img, cudaStream_t s)
{
    const size_t b = col_smem_bytes(p, ST);
    cudaError_t e = cudaFuncSetAttribute(k_blur_cols<TW, ST, ADJ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    if (e != cudaSuccess) return e;
    dim3 grid((p.n_u + TW - 1) / TW, n_img);
    k_blur_cols<TW, ST, ADJ><<<grid, kColThreads, b, s>>>(p, tp, ts, out);
    return cudaGetLastError();
}

static size_t row_smem_bytes(const BlurParams &p)
{
    const int R = p.rs > p.rp ? p.rs : p.rp;
    const int span = p.n_u + 2 * R + 2 * kOut;
    return (size_t)(span + span / 32 + 2) * sizeof(float);
}

namespace {
constexpr size_t kDirectSmemLimit = 220 * 1024;   // dynamic shared memory the direct passes ask for
}

bool blur_rows_fit(const BlurParams &p) { return row_smem_bytes(p) <= kDirectSmemLimit; }

bool blur_cols_fit(const BlurParams &p) { return col_smem_bytes(p, 9) <= kDirectSmemLimit; }

template <bool ADJ>
static cudaError_t rows_pass(const BlurParams &p, const float *T, float *tp, float *ts, int n_img,
                             cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    if (!blur_rows_fit(p)) return cudaErrorInvalidValue;
    const size_t row_smem = row_smem_bytes(p);
    cudaError_t e;
    if (row_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_blur_rows<ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)row_smem);
        if (e != cudaSuccess) return e;
    }
    int threads = ((p.n_u + kOut - 1) / kOut + 31) / 32 * 32;
    threads = threads < 32 ? 32 : (threads > kRowThreads ? kRowThreads : threads);
    k_blur_rows<ADJ><<<(unsigned)((size_t)n_img * p.n_v), threads, row_smem, s>>>(p, T, tp, ts);
    return cudaGetLastError();
}

template <bool ADJ>
static cudaError_t cols_pass(const BlurParams &p, const float *tp, const float *ts, float *out,
                             int n_img, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    // Prefer 16-column tiles (about 3 CTAs per SM for a 384-row detector);
    // fall back to narrower tiles for tall detectors.
    const size_t limit = kDirectSmemLimit;
    if (col_smem_bytes(p, 18) <= limit / 2) return launch_cols_tw<16, 18, ADJ>(p, tp, ts, out, n_img, s);
    if (col_smem_bytes(p, 9) <= limit) return launch_cols_tw<8, 9, ADJ>(p, tp, ts, out, n_img, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_blur_rows(const BlurParams &p, const float *T, float *tp, float *ts, int n_img,
                             cudaStream_t s)
{
    return rows_pass<false>(p, T, tp, ts, n_img, s);
}

cudaError_t launch_blur_cols(const BlurParams &p, const float *tp, const float *ts, float *out,
                             int n_img, cudaStream_t s)
{
    return cols_pass<false>(p, tp, ts, out, n_img, s);
}

// Transpose of out = n0 (C_p R_p + spr C_s R_s) in (clamp-to-edge passes):
// the row and column passes act on different axes and commute, so the
// transpose is n0 (C_p^T R_p^T + spr C_s^T R_s^T) gin: the transposed row pass
// (one input, both kernels) into tp and ts, then the transposed column pass
// combining them.
cudaError_t launch_blur_transpose(const BlurParams &p, const float *gin, float *tp, float *ts,
                                  float *gout, int n_img, cudaStream_t s)
{
    cudaError_t e = rows_pass<true>(p, gin, tp, ts, n_img, s);
    if (e != cudaSuccess) return e;
    return cols_pass<true>(p, tp, ts, gout, n_img, s);
}

// Each warp draws 32 * kPer pixels of one detector row (lane l: pixels
// base + l + 32 s).  Most draws are decided by their first PTRS attempt's
// squeeze; the final acceptance test (log P(k; lam)) is long and needed by
// ~14% of attempts, so a warp that ran it whenever any lane needed it would
// run it almost every pass with most lanes idle.  Instead:
//   round phase  every lane takes its next pixel: the early exits (rate <= 0,
//                > 1e7, < 10) or the first attempt's squeeze; undecided draws
//                (final test pending, or rejected) go to a per-warp queue in
//                shared memory with their state;
//   drain phase  the warp takes the queue 32 items at a time, one per lane,
//                and completes each draw (final test, further attempts).
// Each draw performs exactly the operations of noise::poisson in the same
// order, so the counts are those of the serial sampler.  A full queue (rare)
// makes the lane complete its draw on the spot.  lam and out may alias.
namespace {
constexpr int kPer = 8;
constexpr int kQueue = 96;          // queued draws per warp
constexpr int kWarps = 8;

// One queued draw in three 16-byte words (one shared store or load each):
// p = (lam, b, a, vr); t = bits of (kf, us, V) and jh = attempt block j << 1
// | word pair h, bit 31 set while the final test is pending; w = (iu, words
// z and w of block j, unused).
struct DrawQueue {
    float4 p[kQueue];
    uint4 t[kQueue];
    uint4 w[kQueue];
};
}  // namespace

__global__ void __launch_bounds__(32 * kWarps, 5)
k_poisson(const float *lam, float *out, int n_v, int n_u, int angle0,
          const __grid_constant__ noise::PhiloxKeys seed, int c_lo, int c_hi, float cst)
{
    __shared__ DrawQueue q_all[kWarps];
    DrawQueue &q = q_all[threadIdx.y];
    const int lane = threadIdx.x;
    const int iv = blockIdx.y * blockDim.y + threadIdx.y;
    if (iv >= n_v) return;                      // whole warps leave together
    const int k = blockIdx.z;
    const size_t row = ((size_t)k * n_v + iv) * n_u;
    const int u_base = blockIdx.x * (32 * kPer) + lane;
    const uint32_t kabs = (uint32_t)(angle0 + k);
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;                              // warp-uniform
    for (int sidx = 0; sidx < kPer; ++sidx) {
        const int iu = u_base + 32 * sidx;
        bool enq = false;
        noise::Ptrs st;
        float kf = 0.0f, us = 0.0f, V = 0.0f;
        bool pending = false;
        if (iu < n_u) {
            float r;
            // rows outside [c_lo, c_hi) have the rate cst (not read)
            const float lv = (iv >= c_lo && iv < c_hi) ? lam[row + iu] : cst;
            if (noise::poisson_begin(lv, (uint32_t)iu, (uint32_t)iv, kabs, seed, st, r)) {
                out[row + iu] = r;
            } else {
                const int o = noise::ptrs_quick(st, r, kf, us, V);
                if (o == noise::kDone) {
                    out[row + iu] = r;
                } else {
                    enq = true;
                    pending = o == noise::kPending;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, enq);
        if (enq) {
            const int pos = count + __popc(m & lt);
            if (pos < kQueue) {
                q.p[pos] = make_float4(st.lam, st.b, st.a, st.vr);
                q.t[pos] = make_uint4(__float_as_uint(kf), __float_as_uint(us), __float_as_uint(V),
                                      (st.j << 1) | (uint32_t)st.h | (pending ? 0x80000000u : 0u));
                q.w[pos] = make_uint4((uint32_t)iu, st.w.z, st.w.w, 0u);
            } else {
                // queue full: finish this draw here
                float r;
                bool done = pending ? noise::ptrs_final(st, kf, us, V, r) : false;
                while (!done) done = noise::ptrs_attempt(st, r);
                out[row + iu] = r;
            }
        }
        count = min(count + __popc(m), kQueue);
    }
    __syncwarp();
    for (int i = lane; i < count; i += 32) {
        const float4 qp = q.p[i];
        const uint4 qt = q.t[i], qw = q.w[i];
        noise::Ptrs st;
        st.lam = qp.x;
        st.b = qp.y;
        st.a = qp.z;
        st.vr = qp.w;
        st.loglam = 0.0f;
        st.invalpha = 0.0f;
        st.have_slow = false;
        st.iu = qw.x;
        st.iv = (uint32_t)iv;
        st.k = kabs;
        const uint32_t jh = qt.w;
        st.j = (jh & 0x7fffffffu) >> 1;
        st.h = (int)(jh & 1u);
        st.key = &seed;
        st.w = make_uint4(0u, 0u, qw.y, qw.z);
        float r;
        bool done = (jh & 0x80000000u)
                        ? noise::ptrs_final(st, __uint_as_float(qt.x), __uint_as_float(qt.y),
                                            __uint_as_float(qt.z), r)
                        : false;
        while (!done) done = noise::ptrs_attempt(st, r);
        out[row + qw.x] = r;
    }
}

cudaError_t launch_poisson(const float *lam, float *out, int n_img, int n_v, int n_u, int angle0,
                           uint64_t seed, cudaStream_t s, int c_lo, int c_hi, float cst)
{
    if (c_hi < 0) {
        c_lo = 0;
        c_hi = n_v;
    }
    if ((size_t)n_img * n_v * n_u == 0) return cudaSuccess;
    if ((n_v + kWarps - 1) / kWarps > 65535 || n_img > 65535) return cudaErrorInvalidValue;
    dim3 block(32, kWarps);
    dim3 grid((n_u + 32 * kPer - 1) / (32 * kPer), (n_v + kWarps - 1) / kWarps, n_img);
    k_poisson<<<grid, block, 0, s>>>(lam, out, n_v, n_u, angle0, noise::philox_keys(seed), c_lo, c_hi, cst);
    return cudaGetLastError();
}

}  // namespace fc

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
//            8 adjacent outputs of one column, and the epilogue forms I and
//            optionally draws the Poisson count in the same pass.
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

}  // namespace

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
        uu = uu < 0 ? 0 : (uu > n - 1 ? n - 1 : uu);
        srow[skew(i)] = src[uu];
    }
    __syncthreads();
    for (int u0 = threadIdx.x * kOut; u0 < n; u0 += blockDim.x * kOut) {
        float ap[kOut], as[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) { ap[o] = 0.0f; as[o] = 0.0f; }
        row_conv(srow, u0 + R - p.rp, p.gp, 2 * p.rp + 1, ap);
        row_conv(srow, u0 + R - p.rs, p.gs, 2 * p.rs + 1, as);
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            if (u0 + o < n) {
                tp[row * n + u0 + o] = ap[o];
                ts[row * n + u0 + o] = as[o];
            }
        }
    }
}

// Column pass.  Tile: TW columns x (n_v + 2 R) rows of each row-pass result.
template <int TW>
__global__ void __launch_bounds__(kColThreads)
k_blur_cols(const __grid_constant__ BlurParams p, const float *__restrict__ tp,
            const float *__restrict__ ts, float *__restrict__ out)
{
    extern __shared__ float smem[];
    const int nv = p.n_v, nu = p.n_u;
    const int hp = nv + 2 * p.rp + kOut, hs = nv + 2 * p.rs + kOut;
    float *sp = smem;              // [hp][TW]
    float *ss = smem + hp * TW;    // [hs][TW]
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
        vv = vv < 0 ? 0 : (vv > nv - 1 ? nv - 1 : vv);
        sp[r * TW + col] = gp_src[(size_t)vv * nu + uc];
    }
    for (int r = grp; r < hs; r += ngrp) {
        int vv = r - p.rs;
        vv = vv < 0 ? 0 : (vv > nv - 1 ? nv - 1 : vv);
        ss[r * TW + col] = gs_src[(size_t)vv * nu + uc];
    }
    __syncthreads();
    const int k_abs = p.angle0 + img;
    for (int v0 = grp * kOut; v0 < nv; v0 += ngrp * kOut) {
        float ap[kOut], as[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) { ap[o] = 0.0f; as[o] = 0.0f; }
        // psf taps over rows v0 + o + j (tile row = v + j)
        {
            float win[kOut];
#pragma unroll
            for (int o = 0; o < kOut; ++o) win[o] = sp[(v0 + o) * TW + col];
            const int nt = 2 * p.rp + 1;
            int j = 0;
            for (; j + kOut <= nt; j += kOut) {
#pragma unroll
                for (int q = 0; q < kOut; ++q) {
                    const float gj = p.gp[j + q];
#pragma unroll
                    for (int o = 0; o < kOut; ++o) ap[o] = fmaf(gj, win[(o + q) % kOut], ap[o]);
                    win[q] = sp[(v0 + j + q + kOut) * TW + col];
                }
            }
            for (int q = 0; j + q < nt; ++q) {
                const float gj = p.gp[j + q];
#pragma unroll
                for (int o = 0; o < kOut; ++o) ap[o] = fmaf(gj, sp[(v0 + j + q + o) * TW + col], ap[o]);
            }
        }
        {
            float win[kOut];
#pragma unroll
            for (int o = 0; o < kOut; ++o) win[o] = ss[(v0 + o) * TW + col];
            const int nt = 2 * p.rs + 1;
            int j = 0;
            for (; j + kOut <= nt; j += kOut) {
#pragma unroll
                for (int q = 0; q < kOut; ++q) {
                    const float gj = p.gs[j + q];
#pragma unroll
                    for (int o = 0; o < kOut; ++o) as[o] = fmaf(gj, win[(o + q) % kOut], as[o]);
                    win[q] = ss[(v0 + j + q + kOut) * TW + col];
                }
            }
            for (int q = 0; j + q < nt; ++q) {
                const float gj = p.gs[j + q];
#pragma unroll
                for (int o = 0; o < kOut; ++o) as[o] = fmaf(gj, ss[(v0 + j + q + o) * TW + col], as[o]);
            }
        }
        if (u < nu) {
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
                const int v = v0 + o;
                if (v < nv) {
                    float I = p.n0 * (ap[o] + p.spr * as[o]);
                    if (p.noise)
                        I = noise::poisson(I, (uint32_t)u, (uint32_t)v, (uint32_t)k_abs, p.seed);
                    out[img * plane + (size_t)v * nu + u] = I;
                }
            }
        }
    }
}

static size_t col_smem_bytes(const BlurParams &p, int tw)
{
    return (size_t)(2 * p.n_v + 2 * p.rp + 2 * p.rs + 2 * kOut) * tw * sizeof(float);
}

cudaError_t launch_blur_rows(const BlurParams &p, const float *T, float *tp, float *ts, int n_img,
                             cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const int R = p.rs > p.rp ? p.rs : p.rp;
    const int span = p.n_u + 2 * R + 2 * kOut;
    const size_t row_smem = (size_t)(span + span / 32 + 2) * sizeof(float);
    cudaError_t e;
    if (row_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_blur_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)row_smem);
        if (e != cudaSuccess) return e;
    }
    int threads = ((p.n_u + kOut - 1) / kOut + 31) / 32 * 32;
    threads = threads < 32 ? 32 : (threads > kRowThreads ? kRowThreads : threads);
    k_blur_rows<<<(unsigned)((size_t)n_img * p.n_v), threads, row_smem, s>>>(p, T, tp, ts);
    return cudaGetLastError();
}

cudaError_t launch_blur_cols(const BlurParams &p, const float *tp, const float *ts, float *out,
                             int n_img, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    cudaError_t e;
    const size_t limit = 220 * 1024;
    dim3 grid;
    grid.y = n_img;
    if (col_smem_bytes(p, 32) <= limit) {
        const size_t b = col_smem_bytes(p, 32);
        e = cudaFuncSetAttribute(k_blur_cols<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        if (e != cudaSuccess) return e;
        grid.x = (p.n_u + 31) / 32;
        k_blur_cols<32><<<grid, kColThreads, b, s>>>(p, tp, ts, out);
    } else if (col_smem_bytes(p, 16) <= limit) {
        const size_t b = col_smem_bytes(p, 16);
        e = cudaFuncSetAttribute(k_blur_cols<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        if (e != cudaSuccess) return e;
        grid.x = (p.n_u + 15) / 16;
        k_blur_cols<16><<<grid, kColThreads, b, s>>>(p, tp, ts, out);
    } else {
        const size_t b = col_smem_bytes(p, 8);
        if (b > limit) return cudaErrorInvalidValue;
        e = cudaFuncSetAttribute(k_blur_cols<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        if (e != cudaSuccess) return e;
        grid.x = (p.n_u + 7) / 8;
        k_blur_cols<8><<<grid, kColThreads, b, s>>>(p, tp, ts, out);
    }
    return cudaGetLastError();
}

__global__ void k_poisson(const float *lam, float *out, int n_img, int n_v, int n_u, int angle0,
                          uint64_t seed)
{
    const size_t n = (size_t)n_img * n_v * n_u;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int iu = (int)(i % n_u);
        const int iv = (int)((i / n_u) % n_v);
        const int k = (int)(i / ((size_t)n_u * n_v));
        out[i] = noise::poisson(lam[i], (uint32_t)iu, (uint32_t)iv, (uint32_t)(angle0 + k), seed);
    }
}

cudaError_t launch_poisson(const float *lam, float *out, int n_img, int n_v, int n_u, int angle0,
                           uint64_t seed, cudaStream_t s)
{
    const size_t n = (size_t)n_img * n_v * n_u;
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_poisson<<<(unsigned)blocks, 256, 0, s>>>(lam, out, n_img, n_v, n_u, angle0, seed);
    return cudaGetLastError();
}

}  // namespace fc

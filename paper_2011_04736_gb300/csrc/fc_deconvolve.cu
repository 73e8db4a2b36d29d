// Richardson-Lucy deconvolution of projections (discussion, Sec. IV: the
// detector PSF estimated by the simulation deconvolved from the projection
// images before reconstruction), as the EM update for Poisson data
//
//   u_{k+1} = u_k * H^T (d / max(H u_k, floor)) / H^T 1,    u_0 = d,
//
// with H the detector's clamp-to-edge separable sampled-Gaussian blur and
// H^T its exact adjoint.  Along one axis of length n,
//   (H^T r)(q) = sum_j g_j r(q - j)       (r = 0 outside [0, n))
//              + [q = 0]     sum_p r(p) sum_{j < -p} g_j
//              + [q = n - 1] sum_p r(p) sum_{j > n - 1 - p} g_j,
// the last two terms being the mass the clamp moves onto the edge samples.
// H^T 1 is the outer product of the per-axis column sums (k_rl_norm).
//
// One launch per iteration (k_rl_step): a CTA owns a 64 x 32 output tile,
// stages u with a clamped halo of 2R, forms H u on the tile plus an R halo,
// the ratio r = d / H u (zero outside the image), then H^T r along v and u
// (with the edge folds) and the update.  Every intermediate stays in shared
// memory: per iteration HBM sees u and d once and the new u once.
#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr int kTu = 64, kTv = 32;
constexpr int kThreads = 256;

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

size_t rl_smem_floats(int R)
{
    const size_t su = (size_t)(kTv + 4 * R) * (kTu + 4 * R);
    const size_t b = (size_t)(kTv + 4 * R) * (kTu + 2 * R);   // H_u u, then H_v^T r
    const size_t c = (size_t)(kTv + 2 * R) * (kTu + 2 * R);   // H u, then r
    return su + b + c;
}

}  // namespace

// norm[0 .. n_v) = column sums of B_v, norm[n_v .. n_v + n_u) = of B_u.
__global__ void k_rl_norm(const __grid_constant__ RlParams p, float *norm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_v + p.n_u) return;
    const int n = i < p.n_v ? p.n_v : p.n_u;
    const int q = i < p.n_v ? i : i - p.n_v;
    float s = 0.0f;
    for (int j = -p.R; j <= p.R; ++j)
        if (q - j >= 0 && q - j < n) s += p.taps[j + p.R];
    if (q == 0)
        for (int k = 0; k < p.R && k < n; ++k) s += p.cl[k];
    if (q == n - 1)
        for (int k = 0; k < p.R && k < n; ++k) s += p.cl[k];
    norm[i] = s;
}

template <int R>
__global__ void __launch_bounds__(kThreads)
k_rl_step(const __grid_constant__ RlParams p, const float *__restrict__ d,
          const float *__restrict__ uin, float *__restrict__ uout, const float *__restrict__ norm)
{
    extern __shared__ float sm[];
    constexpr int nt = 2 * R + 1;
    const int WA = kTu + 4 * R, HA = kTv + 4 * R;   // su
    const int WB = kTu + 2 * R;                      // eu (HA rows), later t (kTv rows)
    const int HC = kTv + 2 * R, WC = kTu + 2 * R;    // e, then r
    float *su = sm;
    float *sb = su + HA * WA;
    float *sc = sb + HA * WB;
    const int tid = threadIdx.x;
    const int u0 = blockIdx.x * kTu, v0 = blockIdx.y * kTv;
    const size_t img = (size_t)blockIdx.z * p.n_u * p.n_v;
    const float *g = p.taps;

    // u on rows v0 - 2R .., columns u0 - 2R .., clamped
    for (int i = tid; i < HA * WA; i += kThreads) {
        const int r = i / WA, c = i % WA;
        su[i] = __ldg(uin + img + (size_t)clampi(v0 - 2 * R + r, p.n_v) * p.n_u +
                      clampi(u0 - 2 * R + c, p.n_u));
    }
    __syncthreads();
    // H_u u: rows as su, columns u0 - R ..
    for (int i = tid; i < HA * WB; i += kThreads) {
        const int r = i / WB, c = i % WB;
        const float *x = su + r * WA + c;
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < nt; ++j) s = fmaf(g[j], x[j], s);
        sb[i] = s;
    }
    __syncthreads();
    // H u on rows v0 - R .., columns u0 - R ..; then r = d / max(H u, floor),
    // zero outside the image
    for (int i = tid; i < HC * WC; i += kThreads) {
        const int r = i / WC, c = i % WC;
        const float *x = sb + r * WB + c;
        float e = 0.0f;
#pragma unroll
        for (int j = 0; j < nt; ++j) e = fmaf(g[j], x[j * WB], e);
        const int v = v0 - R + r, u = u0 - R + c;
        float ratio = 0.0f;
        if (v >= 0 && v < p.n_v && u >= 0 && u < p.n_u)
            ratio = __ldg(d + img + (size_t)v * p.n_u + u) / fmaxf(e, p.floor_);
        sc[i] = ratio;
    }
    __syncthreads();
    // H_v^T r: tile rows, columns u0 - R ..
    for (int i = tid; i < kTv * WC; i += kThreads) {
        const int q = i / WC, c = i % WC;
        const int vq = v0 + q;
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < nt; ++j) s = fmaf(g[j], sc[(q + 2 * R - j) * WC + c], s);
        if (vq == 0)
            for (int k = 0; k < R; ++k) s = fmaf(p.cl[k], sc[(k + R) * WC + c], s);
        if (vq == p.n_v - 1)
            for (int k = 0; k < R; ++k) s = fmaf(p.cl[k], sc[(p.n_v - 1 - k - v0 + R) * WC + c], s);
        sb[i] = s;
    }
    __syncthreads();
    // H_u^T, the update
    for (int i = tid; i < kTv * kTu; i += kThreads) {
        const int q = i / kTu, c = i % kTu;
        const int vq = v0 + q, uq = u0 + c;
        if (vq >= p.n_v || uq >= p.n_u) continue;
        const float *t = sb + q * WC;
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < nt; ++j) s = fmaf(g[j], t[c + 2 * R - j], s);
        if (uq == 0)
            for (int k = 0; k < R; ++k) s = fmaf(p.cl[k], t[k + R], s);
        if (uq == p.n_u - 1)
            for (int k = 0; k < R; ++k) s = fmaf(p.cl[k], t[p.n_u - 1 - k - u0 + R], s);
        const float uc = su[(q + 2 * R) * WA + c + 2 * R];
        uout[img + (size_t)vq * p.n_u + uq] = uc * s / (norm[vq] * norm[p.n_v + uq]);
    }
}

cudaError_t launch_rl(const RlParams &p, const float *d, float *ua, float *ub, float *norm,
                      int n_img, int n_iter, float **result, cudaStream_t s)
{
    *result = nullptr;
    if (n_img <= 0 || n_iter <= 0) return cudaSuccess;
    k_rl_norm<<<(p.n_u + p.n_v + 127) / 128, 128, 0, s>>>(p, norm);
    const size_t bytes = rl_smem_floats(p.R) * sizeof(float);
    void (*kern)(RlParams, const float *, const float *, float *, const float *) = nullptr;
    switch (p.R) {
#define FC_RL_CASE(r) case r: kern = k_rl_step<r>; break;
        FC_RL_CASE(0) FC_RL_CASE(1) FC_RL_CASE(2) FC_RL_CASE(3) FC_RL_CASE(4) FC_RL_CASE(5)
        FC_RL_CASE(6) FC_RL_CASE(7) FC_RL_CASE(8) FC_RL_CASE(9) FC_RL_CASE(10) FC_RL_CASE(11)
        FC_RL_CASE(12) FC_RL_CASE(13) FC_RL_CASE(14) FC_RL_CASE(15) FC_RL_CASE(16)
#undef FC_RL_CASE
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    const size_t plane = (size_t)p.n_u * p.n_v;
    const float *src = d;
    float *dst = ua;
    for (int it = 0; it < n_iter; ++it) {
        for (int i0 = 0; i0 < n_img; i0 += 65535) {   // grid z limit
            const int n = n_img - i0 < 65535 ? n_img - i0 : 65535;
            dim3 grid((p.n_u + kTu - 1) / kTu, (p.n_v + kTv - 1) / kTv, n);
            kern<<<grid, kThreads, bytes, s>>>(p, d + i0 * plane, src + i0 * plane,
                                               dst + i0 * plane, norm);
        }
        src = dst;
        dst = dst == ua ? ub : ua;
    }
    *result = const_cast<float *>(src);
    return cudaGetLastError();
}

}  // namespace fc

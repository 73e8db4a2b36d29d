// Energy-group detector model: the scatter profile of Sec. II.E added to each
// group's primary and the optical spread of Sec. II.G applied per group
// ("convolved with the OSF at each energy and summed"):
//
//   I = N0 sum_g G_g (x) (P_g + A_g y_g(x)),   y_g(x) = (a_g / sqrt(x^2 + a_g^2))^b_g
//
// The scatter term depends on the detector column only, and a clamp-to-edge
// blur leaves a row-constant image constant along v, so it reduces to one
// profile prof[u] = N0 sum_g A_g (g_g (x)_u y_g)(u) (k_group_profile).  The
// primaries go through k_group_blur: one CTA per 64 x 32 output tile, each
// group's tile (with a clamped halo of its radius) staged in shared memory,
// the next group's copy in flight while the current one is filtered,
// separable row then column passes, the groups accumulated in registers.
#include <math.h>
#include <string.h>

#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr int kTu = 64, kTv = 32;                 // output tile (columns x rows)
constexpr int kThreads = 256;                     // 64 columns x 4 row groups of 8

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// shared bytes of k_group_blur<RM>: two input tiles and the row-pass tile
constexpr size_t group_blur_smem(int rm)
{
    return sizeof(float) * (2 * (size_t)(kTv + 2 * rm) * (kTu + 2 * rm + 1) + (size_t)(kTv + 2 * rm) * (kTu + 1));
}

}  // namespace

__global__ void k_group_profile(const __grid_constant__ GroupParams p, float *__restrict__ prof)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= p.n_u) return;
    float acc = 0.0f;
    for (int gi = 0; gi < p.n_groups; ++gi) {
        if (!(p.amp[gi] > 0.0f)) continue;
        const int R = p.r[gi];
        const float a = p.a_cm[gi];
        float s = 0.0f;
        for (int j = -R; j <= R; ++j) {
            const float x = ((float)clampi(u + j, p.n_u) - p.cu) * p.du;
            s = fmaf(p.taps[gi][j + R], powf(a / sqrtf(fmaf(x, x, a * a)), p.b[gi]), s);
        }
        acc = fmaf(p.amp[gi], s, acc);
    }
    prof[u] = p.n0 * acc;
}

// RM: the largest radius of the groups; every group's taps are read zero
// padded to RM (p.tpad[g][j + RM]), so the tap loops unroll at compile time.
// The next group's tile is copied (cp.async) into the second input buffer
// while the current one is filtered.
template <int RM>
__global__ void __launch_bounds__(kThreads)
k_group_blur(const __grid_constant__ GroupParams p, const float *__restrict__ P,
             const float *__restrict__ prof, float *__restrict__ out)
{
    constexpr int H = kTv + 2 * RM, Wd = kTu + 2 * RM, nt = 2 * RM + 1;
    extern __shared__ float smem[];
    float (*sin_)[H][Wd + 1] = reinterpret_cast<float (*)[H][Wd + 1]>(smem);
    float (*smid)[kTu + 1] = reinterpret_cast<float (*)[kTu + 1]>(smem + 2 * H * (Wd + 1));
    const int tid = threadIdx.x, tx = tid % kTu, ty = tid / kTu;
    const int u0 = blockIdx.x * kTu, v0 = blockIdx.y * kTv;
    const size_t img = (size_t)blockIdx.z * p.n_u * p.n_v;
    const int lane = tid % 32, warp = tid / 32;
    auto stage = [&](int gi, int b) {
        const float *src = P + (size_t)gi * p.grp_stride + img;
        for (int r = warp; r < H; r += kThreads / 32) {
            const float *row = src + (size_t)clampi(v0 - RM + r, p.n_v) * p.n_u;
            for (int c = lane; c < Wd; c += 32) cp_async4(&sin_[b][r][c], row + clampi(u0 - RM + c, p.n_u));
        }
        cp_async_commit();
    };
    float acc[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[o] = 0.0f;
    if (p.n_groups > 0) stage(0, 0);
    for (int gi = 0; gi < p.n_groups; ++gi) {
        const int b = gi & 1;
        const float *tap = p.tpad[gi];
        if (gi + 1 < p.n_groups) {
            stage(gi + 1, b ^ 1);     // its buffer was last read before the previous barrier
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // row pass: 8 adjacent outputs per item from a register window of
        // 8 + 2 RM inputs; the lanes of a warp take different rows (row
        // pitches Wd + 1 and kTu + 1 keep them on different banks)
        for (int it = tid; it < H * (kTu / 8); it += kThreads) {
            const int r = it % H, c0 = (it / H) * 8;
            float w[8 + 2 * RM], o8[8];
#pragma unroll
            for (int k = 0; k < 8 + 2 * RM; ++k) w[k] = sin_[b][r][c0 + k];
#pragma unroll
            for (int o = 0; o < 8; ++o) o8[o] = 0.0f;
#pragma unroll
            for (int j = 0; j < nt; ++j) {
                const float t = tap[j];
#pragma unroll
                for (int o = 0; o < 8; ++o) o8[o] = fmaf(t, w[o + j], o8[o]);
            }
#pragma unroll
            for (int o = 0; o < 8; ++o) smid[r][c0 + o] = o8[o];
        }
        __syncthreads();
        // column pass: 8 outputs of column tx from a window of 8 + 2 RM rows
        {
            float w[8 + 2 * RM];
#pragma unroll
            for (int k = 0; k < 8 + 2 * RM; ++k) w[k] = smid[ty * 8 + k][tx];
#pragma unroll
            for (int j = 0; j < nt; ++j) {
                const float t = tap[j];
#pragma unroll
                for (int o = 0; o < 8; ++o) acc[o] = fmaf(t, w[o + j], acc[o]);
            }
        }
    }
    const int u = u0 + tx;
    if (u >= p.n_u) return;
    const float pu = prof[u];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int v = v0 + ty * 8 + o;
        if (v < p.n_v) out[img + (size_t)v * p.n_u + u] = fmaf(p.n0, acc[o], pu);
    }
}

cudaError_t launch_group_blur(const GroupParams &g, const float *P, float *prof, float *out,
                              int angle0, int n_img, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    k_group_profile<<<(g.n_u + 127) / 128, 128, 0, s>>>(g, prof);
    int rm = 0;
    for (int i = 0; i < g.n_groups; ++i) rm = g.r[i] > rm ? g.r[i] : rm;
    GroupParams q = g;
    memset(q.tpad, 0, sizeof(q.tpad));
    for (int i = 0; i < g.n_groups; ++i)
        for (int j = -g.r[i]; j <= g.r[i]; ++j) q.tpad[i][j + rm] = g.taps[i][j + g.r[i]];
    void (*kern)(GroupParams, const float *, const float *, float *) = nullptr;
    switch (rm) {
#define FC_GB_CASE(r) case r: kern = k_group_blur<r>; break;
        FC_GB_CASE(0) FC_GB_CASE(1) FC_GB_CASE(2) FC_GB_CASE(3) FC_GB_CASE(4) FC_GB_CASE(5)
        FC_GB_CASE(6) FC_GB_CASE(7) FC_GB_CASE(8) FC_GB_CASE(9) FC_GB_CASE(10) FC_GB_CASE(11)
        FC_GB_CASE(12) FC_GB_CASE(13) FC_GB_CASE(14) FC_GB_CASE(15) FC_GB_CASE(16)
#undef FC_GB_CASE
    default: return cudaErrorInvalidValue;
    }
    const size_t smem = group_blur_smem(rm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t plane = (size_t)g.n_u * g.n_v;
    for (int i0 = 0; i0 < n_img; i0 += 65535) {   // grid z limit
        const int n = n_img - i0 < 65535 ? n_img - i0 : 65535;
        const size_t off = (size_t)(angle0 + i0) * plane;
        dim3 grid((g.n_u + kTu - 1) / kTu, (g.n_v + kTv - 1) / kTv, n);
        kern<<<grid, kThreads, smem, s>>>(q, P + off, prof, out + off);
    }
    return cudaGetLastError();
}

}  // namespace fc

// Detector blur of a primary that differs from 1 on a band of rows only
// (paper Sec. II.G optical spread and Sec. II.E scatter, the same operator as
// the two-pass blur):
//
//   I = n0 (G_psf (x) T + spr G_sc (x) T),  T = 1 + D,  D = 0 outside rows [b0, b0 + hb)
//
// The projector's primary has this form: rays of rows that cannot meet the
// voxel slab give T = 1 exactly.  Both kernels are separable and
// clamp-to-edge, so the row pass of an all-ones row is S = sum of the taps
// and its column pass S^2; by linearity
//
//   I = C + n0 (G_psf,v (x) A_psf + spr G_sc,v (x) A_sc),  C = n0 (S_psf^2 + spr S_sc^2),
//   A_b = G_b,u (x) D   (the row pass of the band rows only),
//
// and where the band touches neither detector edge, the column pass of A
// (zero outside the band) at output row c is the plain sum over band rows j
// of g_b[j - c] A_b[j]: a clamped tap index lands on row 0 or n_v - 1, which
// holds zero.  Output rows farther than the larger radius from the band are
// C.  One CTA per (projection, 128-column tile) stages the band rows of D
// (T - 1, exact for T in [1/2, 1] and within 2^-25 below) with the clamped
// halo, forms both row passes in shared memory, and writes every output row
// of its tile: the column sums for rows near the band (each thread keeps its
// column's band values in registers), C elsewhere.  Binary32 throughout;
// the whole image is written once and only the band rows of T are read, so
// the kernel is bound by the output stores.
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {
constexpr int kTW = 128;          // output columns per CTA
constexpr int kThreads = 256;     // two threads per column in the column phase
}  // namespace

template <int HB>
__global__ void __launch_bounds__(kThreads)
k_blur_band(const __grid_constant__ BlurParams bp, const float *__restrict__ T, float *__restrict__ out,
            int b0, int hb, float cst)
{
    extern __shared__ float sm[];
    const int R = bp.rp > bp.rs ? bp.rp : bp.rs;
    const int W = kTW + 2 * R;                     // staged columns per band row
    const int off = R + HB;                        // padded-tap offset
    const int ntp = 2 * off + 1;
    float *D = sm;                                 // [hb][W]
    float *Ap = D + hb * W;                        // [hb][kTW]
    float *As = Ap + hb * kTW;                     // [hb][kTW]
    float *Gp = As + hb * kTW;                     // [ntp]: g_psf[q - off], zero beyond rp
    float *Gs = Gp + ntp;                          // [ntp]
    const int n_u = bp.n_u, n_v = bp.n_v;
    const int x0 = blockIdx.x * kTW;
    const size_t img = (size_t)blockIdx.y * n_v * n_u;
    const int tid = threadIdx.x;

    for (int q = tid; q < ntp; q += kThreads) {
        const int k = q - off;
        Gp[q] = (k >= -bp.rp && k <= bp.rp) ? bp.gp[k + bp.rp] : 0.0f;
        Gs[q] = (k >= -bp.rs && k <= bp.rs) ? bp.gs[k + bp.rs] : 0.0f;
    }
    for (int e = tid; e < hb * W; e += kThreads) {
        const int j = e / W, c = e - j * W;
        const int col = min(max(x0 - R + c, 0), n_u - 1);
        D[e] = T[img + (size_t)(b0 + j) * n_u + col] - 1.0f;
    }
    __syncthreads();
    // row passes of the band rows: A_b[j][x] = sum_k g_b[k] D[j][x + R + k]
    for (int e = tid; e < hb * kTW; e += kThreads) {
        const int j = e / kTW, x = e - j * kTW;
        const float *d = D + j * W + x + R;
        float ap = 0.0f, as = 0.0f;
        for (int k = -bp.rp; k <= bp.rp; ++k) ap = fmaf(bp.gp[k + bp.rp], d[k], ap);
        for (int k = -bp.rs; k <= bp.rs; ++k) as = fmaf(bp.gs[k + bp.rs], d[k], as);
        Ap[e] = ap;
        As[e] = as;
    }
    __syncthreads();
    const int x = tid % kTW, half = tid / kTW;
    if (x0 + x >= n_u) return;                     // no barrier follows
    float ap[HB], as[HB];
#pragma unroll
    for (int j = 0; j < HB; ++j) {
        ap[j] = j < hb ? Ap[j * kTW + x] : 0.0f;
        as[j] = j < hb ? As[j * kTW + x] : 0.0f;
    }
    const int c_lo = max(b0 - R, 0), c_hi = min(b0 + hb + R, n_v);
    float *o = out + img + x0 + x;
    for (int c = half; c < n_v; c += 2) {
        float v = cst;
        if (c >= c_lo && c < c_hi) {
            // band row j meets output row c through tap b0 + j - c
            const float *gp = Gp + off + b0 - c, *gs = Gs + off + b0 - c;
            float sp = 0.0f, ss = 0.0f;
#pragma unroll
            for (int j = 0; j < HB; ++j) {
                sp = fmaf(gp[j], ap[j], sp);
                ss = fmaf(gs[j], as[j], ss);
            }
            v = fmaf(bp.n0, fmaf(bp.spr, ss, sp), cst);
        }
        o[(size_t)c * n_u] = v;
    }
}

namespace {
size_t band_smem(const BlurParams &bp, int hb, int HB)
{
    const int R = bp.rp > bp.rs ? bp.rp : bp.rs;
    return ((size_t)hb * (kTW + 2 * R) + 2 * (size_t)hb * kTW + 2 * (size_t)(2 * (R + HB) + 1)) *
           sizeof(float);
}
constexpr size_t kBandSmemLimit = 200 * 1024;
}  // namespace

// The band kernel applies to bands of at most 32 rows that touch neither
// detector edge and whose staging fits shared memory.
bool blur_band_supported(const BlurParams &bp, int b_lo, int b_hi)
{
    const int hb = b_hi - b_lo;
    if (hb < 1 || hb > 32 || b_lo < 1 || b_hi > bp.n_v - 1) return false;
    return band_smem(bp, hb, hb <= 16 ? 16 : 32) <= kBandSmemLimit;
}

cudaError_t launch_blur_band(const BlurParams &bp, const float *T, float *out, int n_img, int b_lo,
                             int b_hi, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    if (!blur_band_supported(bp, b_lo, b_hi) || n_img > 65535) return cudaErrorInvalidValue;
    const int hb = b_hi - b_lo;
    double sp = 0.0, ss = 0.0;
    for (int j = 0; j <= 2 * bp.rp; ++j) sp += bp.gp[j];
    for (int j = 0; j <= 2 * bp.rs; ++j) ss += bp.gs[j];
    const float cst = (float)((double)bp.n0 * (sp * sp + (double)bp.spr * ss * ss));
    const dim3 grid((bp.n_u + kTW - 1) / kTW, n_img);
    cudaError_t e;
    if (hb <= 16) {
        const size_t smem = band_smem(bp, hb, 16);
        e = cudaFuncSetAttribute(k_blur_band<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_blur_band<16><<<grid, kThreads, smem, s>>>(bp, T, out, b_lo, hb, cst);
    } else {
        const size_t smem = band_smem(bp, hb, 32);
        e = cudaFuncSetAttribute(k_blur_band<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_blur_band<32><<<grid, kThreads, smem, s>>>(bp, T, out, b_lo, hb, cst);
    }
    return cudaGetLastError();
}

}  // namespace fc

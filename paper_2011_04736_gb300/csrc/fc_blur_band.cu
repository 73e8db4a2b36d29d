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
// of its tile: the column sums for rows near the band, C elsewhere.  Binary32 throughout;
// the whole image is written once and only the band rows of T are read, so
// the kernel is bound by the output stores.
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {
constexpr int kTW = 128;          // output columns per CTA
constexpr int kThreads = 256;
constexpr int kRun = 8;           // outputs per thread and task (register tile)
}  // namespace

// Column sums of one task (kRun adjacent output rows from c0, columns x and
// x + 1 of the tile): the optical-spread (PSF) and scatter sums over the band
// rows of A, then I = n0 (psf + spr sc) + cst.  PSF false: the optical
// spread's taps are all zero for these rows and its sums are left out.
template <int HB, bool PSF>
__device__ __forceinline__ void band_column_sums(const BlurParams &bp, const float *Ap, const float *As,
                                                 const float *Gp, const float *Gs, int off, int b0, int c0,
                                                 int c_hi, int x, int x0, int n_u, float cst, float *img)
{
    // band row j meets output row c0 + o through tap b0 + j - c0 - o,
    // padded index off + b0 + j - c0 - o = gp[j + kRun - 1 - o] below
    const float *gp = Gp + off + b0 - c0 - (kRun - 1), *gs = Gs + off + b0 - c0 - (kRun - 1);
    float2 accp[kRun], accs[kRun];
#pragma unroll
    for (int o = 0; o < kRun; ++o) accp[o] = accs[o] = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int jb = 0; jb < HB; jb += kRun) {     // rows hb.. of A are zero
        // taps of this block of kRun band rows: gp[jb + i], i < 2 kRun - 1
        float tp[2 * kRun - 1], ts[2 * kRun - 1];
#pragma unroll
        for (int i = 0; i < 2 * kRun - 1; ++i) {
            if (PSF) tp[i] = gp[jb + i];
            ts[i] = gs[jb + i];
        }
#pragma unroll
        for (int q = 0; q < kRun; ++q) {
            const float2 as = *reinterpret_cast<const float2 *>(As + (jb + q) * kTW + x);
            float2 ap = make_float2(0.0f, 0.0f);
            if (PSF) ap = *reinterpret_cast<const float2 *>(Ap + (jb + q) * kTW + x);
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                const float b = ts[q + kRun - 1 - o];
                if (PSF) {
                    const float a = tp[q + kRun - 1 - o];
                    accp[o].x = fmaf(a, ap.x, accp[o].x);
                    accp[o].y = fmaf(a, ap.y, accp[o].y);
                }
                accs[o].x = fmaf(b, as.x, accs[o].x);
                accs[o].y = fmaf(b, as.y, accs[o].y);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
        const int c = c0 + o;
        if (c >= c_hi) break;
        const float vx = fmaf(bp.n0, fmaf(bp.spr, accs[o].x, accp[o].x), cst);
        const float vy = fmaf(bp.n0, fmaf(bp.spr, accs[o].y, accp[o].y), cst);
        float *dst = img + (size_t)c * n_u + x0 + x;
        if (x0 + x + 1 < n_u && (n_u & 1) == 0) {
            *reinterpret_cast<float2 *>(dst) = make_float2(vx, vy);
        } else {
            if (x0 + x < n_u) dst[0] = vx;
            if (x0 + x + 1 < n_u) dst[1] = vy;
        }
    }
}

// Work split: row passes as tasks of kRun adjacent outputs of one band row
// (a sliding window of D in registers: one shared load per tap for kRun
// FMAs); column sums as tasks of kRun adjacent output rows x 2 columns (per
// band row one pair of A values and one new tap per kernel, 4 kRun FMAs);
// the constant rows as float4 stores.
// 4 CTAs per SM (64 registers, a 20-byte spill) against 3 at the 79
// registers the compiler takes unbounded: paper-scale 0.458 -> 0.427 ms.
template <int HB>
__global__ void __launch_bounds__(kThreads, 4)
k_blur_band(const __grid_constant__ BlurParams bp, const float *__restrict__ T, float *__restrict__ out,
            int b0, int hb, float cst, int write_const)
{
    extern __shared__ float sm[];
    const int R = bp.rp > bp.rs ? bp.rp : bp.rs;
    const int W = kTW + 2 * R + kRun;              // staged columns per band row
    const int off = R + HB + kRun;                 // padded-tap offset
    const int ntp = 2 * off + 1;
    float *D = sm;                                 // [hb][W]
    float *Ap = D + hb * W;                        // [HB][kTW], rows hb.. zero
    float *As = Ap + HB * kTW;                     // [HB][kTW], rows hb.. zero
    float *Gp = As + HB * kTW;                     // [ntp]: g_psf[q - off], zero beyond rp
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
    for (int e = hb * kTW + tid; e < HB * kTW; e += kThreads) {
        Ap[e] = 0.0f;
        As[e] = 0.0f;
    }
    __syncthreads();
    // row passes: A_b[j][x + o] = sum_k g_b[k] D[j][x + o + R + k], o < kRun
    for (int task = tid; task < hb * (kTW / kRun); task += kThreads) {
        const int j = task / (kTW / kRun), x = (task - j * (kTW / kRun)) * kRun;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int r = b ? bp.rs : bp.rp;
            const float *g = b ? bp.gs : bp.gp;
            const float *d = D + j * W + x + R - r;    // window start for tap k = -r
            float acc[kRun], win[kRun];
#pragma unroll
            for (int o = 0; o < kRun; ++o) {
                acc[o] = 0.0f;
                win[o] = d[o];
            }
            int k = 0;
            for (; k + kRun <= 2 * r + 1; k += kRun) {
#pragma unroll
                for (int q = 0; q < kRun; ++q) {
                    const float gk = g[k + q];
#pragma unroll
                    for (int o = 0; o < kRun; ++o) acc[o] = fmaf(gk, win[(o + q) % kRun], acc[o]);
                    win[q] = d[k + q + kRun];
                }
            }
            for (int q = 0; k + q < 2 * r + 1; ++q) {
                const float gk = g[k + q];
#pragma unroll
                for (int o = 0; o < kRun; ++o) acc[o] = fmaf(gk, d[k + q + o], acc[o]);
            }
            float *A = (b ? As : Ap) + j * kTW + x;
#pragma unroll
            for (int o = 0; o < kRun; ++o) A[o] = acc[o];
        }
    }
    __syncthreads();
    // output rows near the band: c in [c_lo, c_hi); the rest hold cst
    const int c_lo = max(b0 - R, 0), c_hi = min(b0 + hb + R, n_v);
    const int n_runs = (c_hi - c_lo + kRun - 1) / kRun;
    for (int task = tid; task < n_runs * (kTW / 2); task += kThreads) {
        const int run = task / (kTW / 2), x = 2 * (task - run * (kTW / 2));
        const int c0 = c_lo + run * kRun;
        // the optical spread reaches output rows [b0 - rp, b0 + hb + rp) only;
        // elsewhere its sums are exact zeros and are skipped (the same value:
        // fma(spr, s, +0) rounds as spr s).  Uniform over a warp: the 64 tasks
        // of a run are consecutive.
        const bool psf = c0 + kRun > b0 - bp.rp && c0 < b0 + hb + bp.rp;
        if (psf)
            band_column_sums<HB, true>(bp, Ap, As, Gp, Gs, off, b0, c0, c_hi, x, x0, n_u, cst, out + img);
        else
            band_column_sums<HB, false>(bp, Ap, As, Gp, Gs, off, b0, c0, c_hi, x, x0, n_u, cst, out + img);
    }
    // constant rows: the image's rows [0, c_lo) and [c_hi, n_v) are two
    // contiguous address ranges; the projection's CTAs split them into
    // contiguous chunks written in address order (whole DRAM pages rather
    // than 512-byte row segments at the row pitch), unless the consumer
    // takes them as cst itself
    if (write_const) {
        const size_t n0 = (size_t)c_lo * n_u, n1 = (size_t)(n_v - c_hi) * n_u, ntot = n0 + n1;
        const size_t hi0 = (size_t)c_hi * n_u;
        const bool vec = (n_u & 3) == 0;     // both ranges and the image start on 16 bytes
        if (vec) {
            const size_t nq = ntot / 4;       // float4 items (n0 is a multiple of 4)
            const size_t per = (nq + gridDim.x - 1) / gridDim.x;
            const size_t q0 = (size_t)blockIdx.x * per, q1 = q0 + per < nq ? q0 + per : nq;
            const float4 c4 = make_float4(cst, cst, cst, cst);
            for (size_t q = q0 + tid; q < q1; q += kThreads) {
                const size_t e = 4 * q;
                const size_t pos = e < n0 ? e : hi0 + (e - n0);
                *reinterpret_cast<float4 *>(out + img + pos) = c4;
            }
        } else {
            const size_t per = (ntot + gridDim.x - 1) / gridDim.x;
            const size_t e0 = (size_t)blockIdx.x * per, e1 = e0 + per < ntot ? e0 + per : ntot;
            for (size_t e = e0 + tid; e < e1; e += kThreads) out[img + (e < n0 ? e : hi0 + (e - n0))] = cst;
        }
    }
}

namespace {
size_t band_smem(const BlurParams &bp, int hb, int HB)
{
    const int R = bp.rp > bp.rs ? bp.rp : bp.rs;
    return ((size_t)hb * (kTW + 2 * R + kRun) + 2 * (size_t)HB * kTW +
            2 * (size_t)(2 * (R + HB + kRun) + 1)) * sizeof(float);
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

void blur_band_rows(const BlurParams &bp, int b_lo, int b_hi, int *c_lo, int *c_hi, float *cst)
{
    const int R = bp.rp > bp.rs ? bp.rp : bp.rs;
    *c_lo = b_lo - R > 0 ? b_lo - R : 0;
    *c_hi = b_hi + R < bp.n_v ? b_hi + R : bp.n_v;
    double sp = 0.0, ss = 0.0;
    for (int j = 0; j <= 2 * bp.rp; ++j) sp += bp.gp[j];
    for (int j = 0; j <= 2 * bp.rs; ++j) ss += bp.gs[j];
    *cst = (float)((double)bp.n0 * (sp * sp + (double)bp.spr * ss * ss));
}

cudaError_t launch_blur_band(const BlurParams &bp, const float *T, float *out, int n_img, int b_lo,
                             int b_hi, cudaStream_t s, bool write_const)
{
    if (n_img <= 0) return cudaSuccess;
    if (!blur_band_supported(bp, b_lo, b_hi) || n_img > 65535) return cudaErrorInvalidValue;
    const int hb = b_hi - b_lo;
    int c_lo, c_hi;
    float cst;
    blur_band_rows(bp, b_lo, b_hi, &c_lo, &c_hi, &cst);
    const int wc = write_const ? 1 : 0;
    const dim3 grid((bp.n_u + kTW - 1) / kTW, n_img);
    cudaError_t e;
    if (hb <= 16) {
        const size_t smem = band_smem(bp, hb, 16);
        e = cudaFuncSetAttribute(k_blur_band<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_blur_band<16><<<grid, kThreads, smem, s>>>(bp, T, out, b_lo, hb, cst, wc);
    } else {
        const size_t smem = band_smem(bp, hb, 32);
        e = cudaFuncSetAttribute(k_blur_band<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_blur_band<32><<<grid, kThreads, smem, s>>>(bp, T, out, b_lo, hb, cst, wc);
    }
    return cudaGetLastError();
}

}  // namespace fc

// Detector blur on the tensor cores: the optical spread (Sec. II.B/G, the
// OSF convolution) and the scatter kernel (Sec. II.E) as banded Toeplitz
// products issued with tcgen05.mma.
//
//   rows pass:    tp = G_psf (x)_u T,   ts = G_sc (x)_u T
//   columns pass: I  = n0 (G_psf (x)_v tp + spr G_sc (x)_v ts)
//
// Each pass convolves along one detector axis ("conv", length Lc) with up to
// two clamp-to-edge sampled-Gaussian kernels ("bands").  A CTA owns 128
// outputs along the conv axis (one MMA M tile) for kN = 32 lines across it.
// For band b with radius R_b and pad P_b = 8 ceil(R_b / 8) the input window
// of 128 + 2 P_b samples per line, read at clamped indices (so the clamp
// lives in the operand and the matrix is a pure Toeplitz band), is the MMA B
// operand (kN x K, K-major).  The A operand is the 128 x (128 + 2 P_b) band
// matrix with its rows in reverse output order, m' = 127 - i.  Then element
// (r, k) of core matrix (g, c) equals g_b[8 (g + c) + r + k - P_b - 127]: it
// depends on g + c only, so every core matrix (g, c) is core g + c of a short
// "Hankel" array and one descriptor whose k-group and row-group byte offsets
// are both 128 walks the whole band.  That array (15 + (128 + 2 P_b) / 8
// cores of 128 bytes) is built once per call and copied into each CTA with a
// bulk asynchronous copy.
//
// Precision: samples and taps are split into bf16 hi + lo and every K step
// issues hi*hi + hi*lo + lo*hi (the dropped lo*lo term is ~2^-18 relative),
// accumulating in f32 in TMEM: ~1e-5 relative to the f32 direct sum.
//
// Waits are bounded: a CTA whose copies or MMAs do not complete sets the
// error word, waits once more (bounded) for its own operations, frees its
// TMEM and skips its stores.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fc_internal.cuh"
#include "fc_tc.cuh"

namespace fc {

namespace {

constexpr int kN = 32;                 // lines across the conv axis per tile
constexpr int kProdWarps = 8;          // warps 0-7 fill the B stages
constexpr int kEpiWarps = 4;           // warps 8-11 drain TMEM
constexpr int kMmaWarp = kProdWarps + kEpiWarps;   // warp 12 issues the MMAs
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr int kBatch = 8;              // window items a producer thread loads at once
constexpr uint32_t kLbo = kN / 8 * 128;   // k-group stride of a B operand
constexpr uint32_t kTmemCols = 128;    // two accumulator buffers x two bands x kN
constexpr uint32_t kPolls = 1u << 24;  // bounded mbarrier polls
constexpr uint32_t kHdr = 128;         // mbarriers, TMEM slot, abort flag

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t bf16_bits(float x)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// hi = bf16(v), lo = bf16(v - hi), eight values packed into 16 bytes each.
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 a = __float2bfloat16_rn(v[2 * q]);
        const __nv_bfloat16 b = __float2bfloat16_rn(v[2 * q + 1]);
        h[q] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
        l[q] = bf16_bits(v[2 * q] - __bfloat162float(a)) |
               (bf16_bits(v[2 * q + 1] - __bfloat162float(b)) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(bar)) : "memory");
}

// Bounded wait for phase `parity` that also gives up once `abort_flag` is set.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    for (uint32_t i = 0; i < kPolls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 63u && *abort_flag) return false;
    }
    return false;
}

}  // namespace

// Hankel arrays of both bands: [band 0 hi][band 0 lo][band 1 hi][band 1 lo],
// each ncore_b * 64 bf16; core d, element (r, k) = g_b[8 d + r + k - P_b - 127].
__global__ void k_blur_hankel(const __grid_constant__ BlurParams bp, TcBlurParams tp, uint16_t *H)
{
    for (int b = 0; b < tp.n_band; ++b) {
        const TcBand &bd = tp.band[b];
        const float *g = b == 0 ? bp.gp : bp.gs;
        const int R = b == 0 ? bp.rp : bp.rs;
        const int n = bd.ncore * 64;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
            const int d = e >> 6, r = (e >> 3) & 7, k = e & 7;
            const int j = 8 * d + r + k - bd.pad - 127;
            const float t = (j >= -R && j <= R) ? g[j + R] : 0.0f;
            const __nv_bfloat16 hi = __float2bfloat16_rn(t);
            H[bd.h_off + e] = __bfloat16_as_ushort(hi);
            H[bd.h_off + n + e] = (uint16_t)bf16_bits(t - __bfloat162float(hi));
        }
    }
}

// Persistent, warp-specialised pass.  One CTA per SM walks tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... (128 conv positions x kN
// lines of one image each):
//   warps 0-7   producers: fill B stage (j mod n_stage) with the tile's
//               windows (bf16 hi/lo, both bands), arrive on full[stage];
//   warp 12     MMA issuer (lane 0): waits full[stage] and acc_empty[buf],
//               issues 3 MMAs per K step and band into accumulator buffer
//               j mod 2, commits to empty[stage] and acc_full[buf];
//   warps 8-11  epilogue: wait acc_full[buf], read TMEM lanes 32 q .. 32 q + 31
//               (q = warp - 8), store, arrive on acc_empty[buf].
// Every wait is bounded and gives up early once another role has aborted.
template <bool ROWS>
__global__ void __launch_bounds__(kThreads, 1)
k_blur_tc(const __grid_constant__ TcBlurParams p, int n_stage)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);         // [2]
    uint64_t *empty = full + 2;                                   // [2]
    uint64_t *accf = full + 4;                                    // [2]
    uint64_t *acce = full + 6;                                    // [2]
    uint64_t *bar_h = full + 8;
    uint64_t *bar_fin = full + 9;
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 80);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 84);

    uint32_t hoff[2] = {0, 0}, boff[2] = {0, 0};
    uint32_t stage_bytes = 0;
    {
        uint32_t o = kHdr;
        for (int b = 0; b < p.n_band; ++b) {
            hoff[b] = o;
            o += 2u * p.band[b].ncore * 128u;
        }
        for (int b = 0; b < p.n_band; ++b) {
            boff[b] = o + stage_bytes;
            stage_bytes += 4u * kN * p.band[b].kw;
        }
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int conv_len = ROWS ? p.n_u : p.n_v;
    const int cross_len = ROWS ? p.n_v : p.n_u;
    const int n_m = (conv_len + 127) / 128, n_x = (cross_len + kN - 1) / kN;
    const long long total = (long long)n_m * n_x * p.n_img;
    const size_t plane = (size_t)p.n_u * p.n_v;

    if (warp == kMmaWarp) tc::tmem_alloc(slot, kTmemCols);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], kProdWarps * 32);
            tc::mbar_init(&empty[i], 1);
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], kEpiWarps * 32);
        }
        tc::mbar_init(bar_h, 1);
        tc::mbar_init(bar_fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;

    if (warp < kProdWarps) {
        // ---------------- producers
        const int ptid = tid;
        const int ni0 = kN * (p.band[0].kw >> 3);
        const int ntot = ni0 + (p.n_band > 1 ? kN * (p.band[1].kw >> 3) : 0);
        for (long long j = 0;; ++j) {
            const long long t = blockIdx.x + j * gridDim.x;
            if (t >= total) break;
            const int st = (int)(j % n_stage);
            const uint32_t ph = (uint32_t)((j / n_stage) & 1);
            if (!wait_bar(&empty[st], ph ^ 1u, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            const int m0 = (int)(t % n_m) * 128;
            const int x0 = (int)((t / n_m) % n_x) * kN;
            const size_t img = (size_t)(t / ((long long)n_m * n_x)) * plane;
            for (int base = ptid; base < ntot; base += kProdWarps * 32 * kBatch) {
                float v[kBatch][8];
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = base + q * kProdWarps * 32;
                    if (i < ntot) {
                        const int b = i < ni0 ? 0 : 1;
                        const int ii = b ? i - ni0 : i;
                        const int n = ii % kN, cg = ii / kN;
                        const TcBand &bd = p.band[b];
                        const float *src = bd.src + img;
                        const int x = clampi(x0 + n, cross_len);
                        const int c0 = m0 - bd.pad + 8 * cg;
                        if (ROWS) {
                            const float *row = src + (size_t)x * p.n_u;
                            if (c0 >= 0 && c0 + 8 <= conv_len && (p.n_u & 3) == 0) {
                                const float4 a = __ldg(reinterpret_cast<const float4 *>(row + c0));
                                const float4 c = __ldg(reinterpret_cast<const float4 *>(row + c0 + 4));
                                v[q][0] = a.x; v[q][1] = a.y; v[q][2] = a.z; v[q][3] = a.w;
                                v[q][4] = c.x; v[q][5] = c.y; v[q][6] = c.z; v[q][7] = c.w;
                            } else {
#pragma unroll
                                for (int tt = 0; tt < 8; ++tt)
                                    v[q][tt] = __ldg(row + clampi(c0 + tt, conv_len));
                            }
                        } else {
#pragma unroll
                            for (int tt = 0; tt < 8; ++tt)
                                v[q][tt] = __ldg(src + (size_t)clampi(c0 + tt, conv_len) * p.n_u + x);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = base + q * kProdWarps * 32;
                    if (i < ntot) {
                        const int b = i < ni0 ? 0 : 1;
                        const int ii = b ? i - ni0 : i;
                        const int n = ii % kN, cg = ii / kN;
                        uint8_t *bhi = smem + boff[b] + (uint32_t)st * stage_bytes;
                        uint8_t *blo = bhi + 2 * kN * p.band[b].kw;
                        uint4 hi, lo;
                        split8(v[q], hi, lo);
                        const uint32_t o = (uint32_t)cg * kLbo + (uint32_t)(n >> 3) * 128u +
                                           (uint32_t)(n & 7) * 16u;
                        *reinterpret_cast<uint4 *>(bhi + o) = hi;
                        *reinterpret_cast<uint4 *>(blo + o) = lo;
                    }
                }
            }
            tc::fence_async_smem();
            mbar_arrive(&full[st]);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            uint32_t bytes = 0;
            for (int b = 0; b < p.n_band; ++b) bytes += 2u * p.band[b].ncore * 128u;
            mbar_expect_tx(bar_h, bytes);
            for (int b = 0; b < p.n_band; ++b)
                bulk_g2s(smem + hoff[b], p.H + p.band[b].h_off, 2u * p.band[b].ncore * 128u, bar_h);
            bool ok = wait_bar(bar_h, 0, abort_flag);
            constexpr uint32_t idesc = tc::idesc_bf16(128, kN);
            for (long long j = 0; ok; ++j) {
                const long long t = blockIdx.x + j * gridDim.x;
                if (t >= total) break;
                const int st = (int)(j % n_stage);
                const uint32_t ph = (uint32_t)((j / n_stage) & 1);
                const int buf = (int)(j & 1);
                const uint32_t bph = (uint32_t)((j >> 1) & 1);
                if (!wait_bar(&full[st], ph, abort_flag) || !wait_bar(&acce[buf], bph ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int b = 0; b < p.n_band; ++b) {
                    const TcBand &bd = p.band[b];
                    const uint32_t ah = tc::smem_u32(smem + hoff[b]);
                    const uint32_t al = ah + (uint32_t)bd.ncore * 128u;
                    const uint32_t bh = tc::smem_u32(smem + boff[b] + (uint32_t)st * stage_bytes);
                    const uint32_t bl = bh + 2u * kN * bd.kw;
                    const uint32_t d = tbase + (uint32_t)(buf * 2 * kN + b * kN);
                    for (int s = 0; s < (bd.kw >> 4); ++s) {
                        const uint64_t dah = tc::sdesc(ah + 256u * s, 128, 128);
                        const uint64_t dal = tc::sdesc(al + 256u * s, 128, 128);
                        const uint64_t dbh = tc::sdesc(bh + 2u * kLbo * s, kLbo, 128);
                        const uint64_t dbl = tc::sdesc(bl + 2u * kLbo * s, kLbo, 128);
                        tc::mma_bf16(d, dah, dbh, idesc, s > 0 ? 1u : 0u);
                        tc::mma_bf16(d, dah, dbl, idesc, 1u);
                        tc::mma_bf16(d, dal, dbh, idesc, 1u);
                    }
                }
                tc::mma_commit(&empty[st]);
                tc::mma_commit(&accf[buf]);
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued so far has completed before TMEM is freed, and
            // the table copy has landed before the CTA exits
            tc::mma_commit(bar_fin);
            tc::mbar_wait(bar_fin, 0, kPolls);
            tc::mbar_wait(bar_h, 0, kPolls);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 8-11: TMEM lane quarter q)
        const int q = warp - kProdWarps;
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16);
        const int mr = 32 * q + lane;
        for (long long j = 0;; ++j) {
            const long long t = blockIdx.x + j * gridDim.x;
            if (t >= total) break;
            const int buf = (int)(j & 1);
            const uint32_t bph = (uint32_t)((j >> 1) & 1);
            int ok = lane == 0 ? (int)wait_bar(&accf[buf], bph, abort_flag) : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const int m0 = (int)(t % n_m) * 128;
            const int x0 = (int)((t / n_m) % n_x) * kN;
            const size_t img = (size_t)(t / ((long long)n_m * n_x)) * plane;
            const int c = m0 + 127 - mr;
            const uint32_t acc = lane_base + (uint32_t)(buf * 2 * kN);
            if (ROWS) {
                for (int b = 0; b < p.n_band; ++b) {
                    float *out = b == 0 ? p.out0 : p.out1;
#pragma unroll
                    for (int j0 = 0; j0 < kN; j0 += 16) {
                        float v[16];
                        tc::tmem_ld16(acc + (uint32_t)(b * kN + j0), v);
                        if (c < conv_len) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int x = x0 + j0 + i;
                                if (x < cross_len) out[img + (size_t)x * p.n_u + c] = v[i];
                            }
                        }
                    }
                }
            } else {
#pragma unroll
                for (int j0 = 0; j0 < kN; j0 += 16) {
                    float vp[16], vs[16];
                    tc::tmem_ld16(acc + (uint32_t)j0, vp);
                    if (p.n_band > 1) {
                        tc::tmem_ld16(acc + (uint32_t)(kN + j0), vs);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) vs[i] = 0.0f;
                    }
                    if (c < conv_len) {
                        float r[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) r[i] = p.n0 * (vp[i] + p.spr * vs[i]);
                        const int xs = x0 + j0;
                        float *dst = p.out0 + img + (size_t)c * p.n_u + xs;
                        if (xs + 16 <= cross_len && (p.n_u & 3) == 0) {
#pragma unroll
                            for (int i = 0; i < 16; i += 4)
                                *reinterpret_cast<float4 *>(dst + i) =
                                    make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (xs + i < cross_len) dst[i] = r[i];
                        }
                    }
                }
            }
            tc::fence_before_sync();
            mbar_arrive(&acce[buf]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicOr(p.err, 1u);
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

// Band geometry for radius R: pad, window, Hankel cores.
static TcBand make_band(const float *src, int R, uint32_t h_off)
{
    TcBand b;
    b.src = src;
    b.pad = (R + 7) / 8 * 8;
    b.kw = 128 + 2 * b.pad;
    b.ncore = 15 + b.kw / 8;
    b.h_off = h_off;
    return b;
}

static size_t tc_smem(const TcBlurParams &p, int n_stage)
{
    size_t o = kHdr;
    for (int b = 0; b < p.n_band; ++b)
        o += 2u * p.band[b].ncore * 128u + (size_t)n_stage * 4u * kN * p.band[b].kw;
    return o;
}

template <bool ROWS>
static cudaError_t launch_tc(TcBlurParams p, int n_img, cudaStream_t s)
{
    const size_t limit = 227 * 1024;
    const int n_stage = tc_smem(p, 2) <= limit ? 2 : 1;
    const size_t bytes = tc_smem(p, n_stage);
    if (bytes > limit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_blur_tc<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int conv = ROWS ? p.n_u : p.n_v, cross = ROWS ? p.n_v : p.n_u;
    const long long tiles = (long long)((conv + 127) / 128) * ((cross + kN - 1) / kN) * n_img;
    p.n_img = n_img;
    const int grid = (int)(tiles < sms ? tiles : sms);
    k_blur_tc<ROWS><<<grid, kThreads, bytes, s>>>(p, n_stage);
    return cudaGetLastError();
}

static TcBlurParams tc_params(const BlurParams &bp, const uint16_t *hankel, unsigned int *err)
{
    TcBlurParams p;
    p.n_band = 2;
    p.H = hankel;
    p.n_u = bp.n_u;
    p.n_v = bp.n_v;
    p.n0 = bp.n0;
    p.spr = bp.spr;
    p.err = err;
    p.band[0] = make_band(nullptr, bp.rp, 0);
    p.band[1] = make_band(nullptr, bp.rs, (uint32_t)(2 * 64 * p.band[0].ncore));
    p.out0 = p.out1 = nullptr;
    p.n_img = 0;
    return p;
}

cudaError_t launch_blur_tc_rows(const BlurParams &bp, const float *in, float *tp, float *ts,
                                uint16_t *hankel, unsigned int *err, int n_img, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    TcBlurParams p = tc_params(bp, hankel, err);
    k_blur_hankel<<<16, 256, 0, s>>>(bp, p, hankel);
    p.band[0].src = in;
    p.band[1].src = in;
    p.out0 = tp;
    p.out1 = ts;
    return launch_tc<true>(p, n_img, s);
}

cudaError_t launch_blur_tc_cols(const BlurParams &bp, const float *tp, const float *ts, float *out,
                                const uint16_t *hankel, unsigned int *err, int n_img, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    TcBlurParams p = tc_params(bp, hankel, err);
    p.band[0].src = tp;
    p.band[1].src = ts;
    p.out0 = out;
    return launch_tc<false>(p, n_img, s);
}

}  // namespace fc

// Detector blur on the tensor cores: the optical spread (Sec. II.B/G, the
// OSF convolution) and the scatter kernel (Sec. II.E) as banded Toeplitz
// products issued with tcgen05.mma.
//
//   rows pass:    tp = G_psf (x)_u T,   ts = G_sc (x)_u T
//   columns pass: I  = n0 (G_psf (x)_v tp + spr G_sc (x)_v ts)
//
// A pass convolves along one detector axis ("conv") with clamp-to-edge
// sampled Gaussians ("bands").  A tile is 128 outputs along the conv axis
// (the MMA M) for kN = 64 detector lines across it (the MMA N).  For band b
// with radius R_b and pad P_b = 8 ceil(R_b / 8), output i of line n is
//   sum_k A_b[i][k] W[n][k],   W[n][k] = src(line n, m0 - P_b + k) (clamped)
// with k over the 128 + 2 P_b window: the clamp lives in the window, so A_b is
// a pure Toeplitz band.  W is the MMA B operand (kN x K, K-major core
// matrices).  With the rows of A_b in reverse output order, m' = 127 - i,
// element (r, k) of core matrix (g, c) is g_b[8 (g + c) + r + k - P_b - 127]:
// it depends on g + c only, so the whole band matrix is a "Hankel" array of
// 15 + (128 + 2 P_b) / 8 cores of 128 bytes walked by one descriptor whose
// k-group and row-group byte offsets are both 128.
//
//   rows pass:    both bands on the tensor cores; they share one window (the
//                 wider band's; the narrower one starts (P_w - P_b) / 8
//                 k-groups in), A from the Hankel arrays in shared memory.
//   columns pass: the scatter band on the tensor cores with its full band
//                 matrix resident in TMEM (written once per CTA), so only W
//                 streams from shared memory; the optical spread (a few taps)
//                 on the CUDA cores in the epilogue, from a staged tile of tp.
//
// Each pass is a persistent, warp-specialised kernel (one CTA per SM):
//   warps 0-7   producers: load the tile's inputs (f32), split them into
//               bf16 hi + lo, store the W stage, arrive on full[stage];
//   warp 12     MMA issuer (lane 0): 3 MMAs per K step (hi*hi, hi*lo,
//               lo*hi; the dropped lo*lo term is ~2^-18 relative) into
//               accumulator buffer j mod 2, commits to empty[stage] and
//               acc_full[buf];
//   warps 8-11  epilogue: TMEM lane quarter q = warp - 8, stores, arrive on
//               acc_empty[buf] (and, in the columns pass, on empty[stage]).
// Accumulation is f32 in TMEM: ~1e-5 relative to the f32 direct sum.  Every
// wait is bounded and gives up early once another role has aborted; an
// aborting CTA sets the error word, waits (bounded) for its own MMAs and
// copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "fc_internal.cuh"
#include "fc_tc.cuh"

namespace fc {

namespace {

constexpr int kN = 64;                 // detector lines per tile (MMA N)
constexpr int kProdWarps = 8;          // warps 0-7 fill the stages
constexpr int kEpiWarps = 4;           // warps 8-11 drain TMEM
constexpr int kMmaWarp = kProdWarps + kEpiWarps;   // warp 12 issues the MMAs
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr int kProd = kProdWarps * 32;
constexpr int kBatch = 8;              // window items a producer thread loads at once
constexpr uint32_t kLbo = kN / 8 * 128;   // k-group stride of a W operand
constexpr uint32_t kPolls = 1u << 24;  // bounded mbarrier polls
constexpr uint32_t kHdr = 128;         // mbarriers, TMEM slot, abort flag
constexpr int kTpPitch = kN + 4;       // staged tp tile row: 16-byte rows, 17 16-byte groups apart
constexpr size_t kSmemLimit = 227 * 1024;

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
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
        h[q] = *reinterpret_cast<const uint32_t *>(&hb);
        l[q] = *reinterpret_cast<const uint32_t *>(&lb);
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
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                         uint32_t polls = kPolls)
{
    for (uint32_t i = 0; i < polls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 63u && *abort_flag) return false;
    }
    return false;
}

// 16-byte global -> shared copy that bypasses the registers (both addresses
// 16-byte aligned), and waiting for this thread's copies.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(tc::smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Lane 0 waits, the warp follows (keeps .sync.aligned TMEM accesses converged).
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          uint32_t polls = kPolls)
{
    int ok = (threadIdx.x & 31) == 0 ? (int)wait_bar(bar, parity, abort_flag, polls) : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Tile t -> (conv start m0, line start x0, image offset).
struct Tile {
    int m0, x0;
    size_t img;
};

__device__ __forceinline__ Tile tile_of(long long t, int n_m, int n_x, size_t plane, int x_off = 0,
                                        int m_off = 0)
{
    Tile r;
    r.m0 = (int)(t % n_m) * 128 + m_off;
    r.x0 = ((int)((t / n_m) % n_x) + x_off) * kN;
    r.img = (size_t)(t / ((long long)n_m * n_x)) * plane;
    return r;
}

// Split window item (line n, k-group cg) of a W stage into its hi and lo blocks.
__device__ __forceinline__ void store_item(uint8_t *whi, uint32_t lo_off, int n, int cg,
                                           const float (&v)[8])
{
    uint4 hi, lo;
    split8(v, hi, lo);
    const uint32_t o = (uint32_t)cg * kLbo + (uint32_t)(n >> 3) * 128u + (uint32_t)(n & 7) * 16u;
    *reinterpret_cast<uint4 *>(whi + o) = hi;
    *reinterpret_cast<uint4 *>(whi + lo_off + o) = lo;
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

// Rows pass (conv = u, lines = detector rows v).  W is the wider band's
// window of T; band b's MMAs start (P_w - P_b) / 8 k-groups into it.  A comes
// from the Hankel arrays in shared memory; TMEM holds two accumulator buffers
// x two bands x kN columns.
__global__ void __launch_bounds__(kThreads, 1)
k_blur_rows_tc(const __grid_constant__ TcBlurParams p, int n_stage)
{
    constexpr uint32_t kCols = 4 * kN;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);   // [2]
    uint64_t *empty = full + 2;                             // [2]
    uint64_t *accf = full + 4;                              // [2]
    uint64_t *acce = full + 6;                              // [2]
    uint64_t *bar_h = full + 8;
    uint64_t *bar_fin = full + 9;
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 80);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 84);

    const int wb = p.n_band > 1 && p.band[1].kw > p.band[0].kw ? 1 : 0;
    const int kw = p.band[wb].kw, pad = p.band[wb].pad;
    const uint32_t h_bytes =
        2u * 128u * (uint32_t)(p.band[0].ncore + (p.n_band > 1 ? p.band[1].ncore : 0));
    const uint32_t w0 = kHdr + h_bytes;                   // stage 0 of W
    const uint32_t wlo = 2u * kN * (uint32_t)kw;          // hi -> lo block
    const uint32_t stage_bytes = 2u * wlo;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_m = (p.n_u + 127) / 128, n_x = p.x_cnt;   // line tiles [x_off, x_off + x_cnt)
    const long long total = (long long)n_m * n_x * p.n_img;
    const size_t plane = (size_t)p.n_u * p.n_v;

    if (warp == kMmaWarp) tc::tmem_alloc(slot, kCols);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], kProd);
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
        // items (line n, k-group cg): each run of 32 is 8 lines x 4 k-groups,
        // so a warp's loads cover 8 row segments of 128 bytes and its shared
        // stores 4 contiguous 128-byte core rows
        const int ngrp = kw >> 3, ng4 = (ngrp + 3) & ~3;
        const int nitems = kN * ng4;
        const float *src = p.band[0].src;
        for (long long j = 0;; ++j) {
            const long long t = blockIdx.x + j * gridDim.x;
            if (t >= total) break;
            const int st = (int)(j % n_stage);
            const uint32_t ph = (uint32_t)((j / n_stage) & 1);
            if (!wait_bar(&empty[st], ph ^ 1u, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            const Tile tl = tile_of(t, n_m, n_x, plane, p.x_off);
            uint8_t *whi = smem + w0 + (uint32_t)st * stage_bytes;
            for (int base = tid; base < nitems; base += kProd * kBatch) {
                float v[kBatch][8];
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = base + q * kProd;
                    const int blk = i >> 5;
                    const int n = (i & 7) + 8 * (blk % (kN / 8));
                    const int cg = ((i >> 3) & 3) + 4 * (blk / (kN / 8));
                    if (i >= nitems || cg >= ngrp) continue;
                    const float *row = src + tl.img + (size_t)clampi(tl.x0 + n, p.n_v) * p.n_u;
                    const int c0 = tl.m0 - pad + 8 * cg;
                    if (c0 >= 0 && c0 + 8 <= p.n_u && (p.n_u & 3) == 0) {
                        const float4 a = __ldg(reinterpret_cast<const float4 *>(row + c0));
                        const float4 c = __ldg(reinterpret_cast<const float4 *>(row + c0 + 4));
                        v[q][0] = a.x; v[q][1] = a.y; v[q][2] = a.z; v[q][3] = a.w;
                        v[q][4] = c.x; v[q][5] = c.y; v[q][6] = c.z; v[q][7] = c.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[q][e] = __ldg(row + clampi(c0 + e, p.n_u));
                    }
                }
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = base + q * kProd;
                    const int blk = i >> 5;
                    const int n = (i & 7) + 8 * (blk % (kN / 8));
                    const int cg = ((i >> 3) & 3) + 4 * (blk / (kN / 8));
                    if (i >= nitems || cg >= ngrp) continue;
                    store_item(whi, wlo, n, cg, v[q]);
                }
            }
            tc::fence_async_smem();
            mbar_arrive(&full[st]);
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            mbar_expect_tx(bar_h, h_bytes);
            bulk_g2s(smem + kHdr, p.H, h_bytes, bar_h);
            uint64_t da[2] = {0, 0}, dal[2] = {0, 0}, dw[2] = {0, 0};
            uint32_t ha = kHdr;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (b >= p.n_band) break;
                da[b] = tc::sdesc(tc::smem_u32(smem + ha), 128, 128);
                dal[b] = (uint64_t)((p.band[b].ncore * 128u) >> 4);
                ha += 2u * p.band[b].ncore * 128u;
                const uint32_t koff = (uint32_t)((pad - p.band[b].pad) >> 3) * kLbo;
                dw[b] = tc::sdesc(tc::smem_u32(smem + w0 + koff), kLbo, 128);
            }
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
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    if (b >= p.n_band) break;
                    // descriptors advance by whole K steps: the start-address
                    // field (bits 0-13, bytes / 16) grows by 256 / 16 for A and
                    // 2 kLbo / 16 for W; shared memory < 256 KB keeps it in range
                    uint64_t ah = da[b], al = da[b] + dal[b];
                    uint64_t wh = dw[b] + (uint64_t)(((uint32_t)st * stage_bytes) >> 4);
                    uint64_t wl = wh + (uint64_t)(wlo >> 4);
                    const uint32_t d = tbase + (uint32_t)(buf * 2 * kN + b * kN);
                    const int ns = p.band[b].kw >> 4;
                    for (int s = 0; s < ns; ++s) {
                        tc::mma_bf16(d, ah, wh, idesc, s > 0 ? 1u : 0u);
                        tc::mma_bf16(d, ah, wl, idesc, 1u);
                        tc::mma_bf16(d, al, wh, idesc, 1u);
                        ah += 16u;
                        al += 16u;
                        wh += 2u * kLbo / 16u;
                        wl += 2u * kLbo / 16u;
                    }
                }
                tc::mma_commit(&empty[st]);
                tc::mma_commit(&accf[buf]);
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued so far completes before TMEM is freed, and the
            // table copy lands before the CTA exits
            tc::mma_commit(bar_fin);
            tc::mbar_wait(bar_fin, 0, kPolls);
            tc::mbar_wait(bar_h, 0, kPolls);
        }
        __syncwarp();
    } else {
        const int q = warp - kProdWarps;
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16);
        const int mr = 32 * q + lane;
        for (long long j = 0;; ++j) {
            const long long t = blockIdx.x + j * gridDim.x;
            if (t >= total) break;
            const int buf = (int)(j & 1);
            const uint32_t bph = (uint32_t)((j >> 1) & 1);
            if (!warp_wait(&accf[buf], bph, abort_flag, p.epi_polls)) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const Tile tl = tile_of(t, n_m, n_x, plane, p.x_off);
            const int c = tl.m0 + 127 - mr;
            const uint32_t acc = lane_base + (uint32_t)(buf * 2 * kN);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (b >= p.n_band) break;
                float *out = b == 0 ? p.out0 : p.out1;
#pragma unroll
                for (int j0 = 0; j0 < kN; j0 += 16) {
                    float v[16];
                    tc::tmem_ld16(acc + (uint32_t)(b * kN + j0), v);
                    if (c < p.n_u) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int x = tl.x0 + j0 + i;
                            if (x < p.n_v) out[tl.img + (size_t)x * p.n_u + c] = v[i];
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
        tc::tmem_dealloc(tbase, kCols);
    }
}

// Columns pass (conv = v, lines = detector columns u).  W is the scatter
// band's window of ts; its full 128 x kw band matrix (hi, then lo; two bf16
// per column) sits in TMEM columns [2 kN, 2 kN + kw) beside two accumulator
// buffers of kN columns, so only W streams from shared memory.  The producers
// also stage tp rows m0 - R_p .. m0 + 127 + R_p of the tile's columns (f32,
// padded rows); the epilogue forms the optical spread from them on the CUDA
// cores.  A stage is released once both its MMAs and its epilogue are done:
// empty[stage] counts one commit and the 128 epilogue threads.
__global__ void __launch_bounds__(kThreads, 1)
k_blur_cols_tc(const __grid_constant__ TcBlurParams p, int n_stage)
{
    constexpr uint32_t kCols = 512;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);   // [2]
    uint64_t *empty = full + 2;                             // [2]
    uint64_t *accf = full + 4;                              // [2]
    uint64_t *acce = full + 6;                              // [2]
    uint64_t *bar_fin = full + 9;
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 80);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 84);

    const TcBand &bs = p.band[1];
    const int kw = bs.kw, pad = bs.pad;
    const int rp = p.rp, trows = 128 + 2 * rp;
    const uint32_t wlo = 2u * kN * (uint32_t)kw;
    const uint32_t tp_bytes = ((uint32_t)(trows * kTpPitch) * 4u + 127u) & ~127u;
    const uint32_t stage_bytes = 2u * wlo + tp_bytes;
    const uint32_t acol = 2 * kN;                          // TMEM column of A (hi)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_m = p.m_cnt, n_x = (p.n_u + kN - 1) / kN;
    const long long total = (long long)n_m * n_x * p.n_img;
    const size_t plane = (size_t)p.n_u * p.n_v;

    if (warp == kMmaWarp) tc::tmem_alloc(slot, kCols);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], kProd);
            tc::mbar_init(&empty[i], 1 + kEpiWarps * 32);
            tc::mbar_init(&accf[i], 1);
            tc::mbar_init(&acce[i], kEpiWarps * 32);
        }
        tc::mbar_init(bar_fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *slot;
    if (warp >= kProdWarps && warp < kMmaWarp) {
        // row m' of the band matrix, A'[m'][k] = g_s[k + m' - P - 127], read
        // from the Hankel table (core d, in-core r + k = s - 8 d, r <= 7)
        const int q = warp - kProdWarps, mr = 32 * q + lane;
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16);
        const uint16_t *hh = p.H + bs.h_off, *hl = hh + bs.ncore * 64;
        const int nw = kw >> 1;
        for (int c0 = 0; c0 < nw; c0 += 8) {
            uint32_t wh[8], wl[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                uint32_t eh[2], el[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int sidx = 2 * (c0 + w) + e + mr;
                    const int d = min(sidx >> 3, bs.ncore - 1);
                    const int rem = sidx - 8 * d, r = min(rem, 7);
                    const int idx = d * 64 + r * 8 + (rem - r);
                    eh[e] = __ldg(hh + idx);
                    el[e] = __ldg(hl + idx);
                }
                wh[w] = eh[0] | (eh[1] << 16);
                wl[w] = el[0] | (el[1] << 16);
            }
            tc::tmem_st8(lane_base + acol + (uint32_t)c0, wh);
            tc::tmem_st8(lane_base + acol + (uint32_t)(nw + c0), wl);
        }
        tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    if (warp < kProdWarps) {
        const int ngrp = kw >> 3, nitems = kN * ngrp;
        const float *ts = bs.src;
        for (long long j = 0;; ++j) {
            const long long t = blockIdx.x + j * gridDim.x;
            if (t >= total) break;
            const int st = (int)(j % n_stage);
            const uint32_t ph = (uint32_t)((j / n_stage) & 1);
            if (!wait_bar(&empty[st], ph ^ 1u, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            const Tile tl = tile_of(t, n_m, n_x, plane, 0, p.m_off);
            uint8_t *whi = smem + kHdr + (uint32_t)st * stage_bytes;
            {
                // tp tile: rows m0 - R_p + r, columns x0 + n (both clamped),
                // copied asynchronously while the W items are processed; rows
                // outside [tp_lo, tp_hi) hold the constant the row pass
                // stands for there and are not loaded
                float *tpt = reinterpret_cast<float *>(whi + 2u * wlo);
                const bool vec = tl.x0 + kN <= p.n_u && (p.n_u & 3) == 0;
                const int nq = trows * (kN / 4);
                for (int e = tid; e < nq; e += kProd) {
                    const int r = e / (kN / 4), n = 4 * (e % (kN / 4));
                    const int src_row = clampi(tl.m0 - rp + r, p.n_v);
                    const float *row = p.tp + tl.img + (size_t)src_row * p.n_u;
                    float *d = tpt + r * kTpPitch + n;
                    if (src_row < p.tp_lo || src_row >= p.tp_hi) {
                        *reinterpret_cast<float4 *>(d) = make_float4(p.tp_const, p.tp_const, p.tp_const,
                                                                     p.tp_const);
                    } else if (vec) {
                        cp_async16(d, row + tl.x0 + n);
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) d[c] = __ldg(row + clampi(tl.x0 + n + c, p.n_u));
                    }
                }
                cp_async_commit();
            }
            // W items (line n = column u, k-group cg): a warp's loads are
            // eight rows of 32 consecutive columns
            for (int base = tid; base < nitems; base += kProd * kBatch) {
                float v[kBatch][8];
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = base + q * kProd;
                    if (i >= nitems) continue;
                    const int n = i % kN, cg = i / kN;
                    const float *col = ts + tl.img + clampi(tl.x0 + n, p.n_u);
                    const int c0 = tl.m0 - pad + 8 * cg;
                    // an item's 8 rows start on a multiple of 8 and the rows
                    // the row pass computed are whole 64-row tiles, so the
                    // item lies wholly inside them or holds the constant
                    const int rc = clampi(c0, p.n_v);
                    if (rc >= p.ts_lo && rc < p.ts_hi) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            v[q][e] = __ldg(col + (size_t)clampi(c0 + e, p.n_v) * p.n_u);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[q][e] = p.ts_const;
                    }
                }
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = base + q * kProd;
                    if (i >= nitems) continue;
                    store_item(whi, wlo, i % kN, i / kN, v[q]);
                }
            }
            cp_async_wait_all();
            tc::fence_async_smem();
            mbar_arrive(&full[st]);
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint64_t dw = tc::sdesc(tc::smem_u32(smem + kHdr), kLbo, 128);
            constexpr uint32_t idesc = tc::idesc_bf16(128, kN);
            const int ns = kw >> 4;
            const uint32_t tl_off = (uint32_t)(kw >> 1);
            bool ok = true;
            for (long long j = 0;; ++j) {
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
                uint64_t wh = dw + (uint64_t)(((uint32_t)st * stage_bytes) >> 4);
                uint64_t wl = wh + (uint64_t)(wlo >> 4);
                uint32_t ah = tbase + acol;
                const uint32_t d = tbase + (uint32_t)(buf * kN);
                for (int s = 0; s < ns; ++s) {
                    tc::mma_bf16_ta(d, ah, wh, idesc, s > 0 ? 1u : 0u);
                    tc::mma_bf16_ta(d, ah, wl, idesc, 1u);
                    tc::mma_bf16_ta(d, ah + tl_off, wh, idesc, 1u);
                    ah += 8u;
                    wh += 2u * kLbo / 16u;
                    wl += 2u * kLbo / 16u;
                }
                tc::mma_commit(&empty[st]);
                tc::mma_commit(&accf[buf]);
            }
            if (!ok) *abort_flag = 1;
            tc::mma_commit(bar_fin);
            tc::mbar_wait(bar_fin, 0, kPolls);
        }
        __syncwarp();
    } else {
        const int q = warp - kProdWarps;
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16);
        const int mr = 32 * q + lane;
        for (long long j = 0;; ++j) {
            const long long t = blockIdx.x + j * gridDim.x;
            if (t >= total) break;
            const int st = (int)(j % n_stage);
            const int buf = (int)(j & 1);
            const uint32_t bph = (uint32_t)((j >> 1) & 1);
            // acc_full follows full[st] through the MMA commit; waiting on
            // full[st] too makes the producers' tp tile visible here directly
            if (!warp_wait(&accf[buf], bph, abort_flag, p.epi_polls) ||
                !warp_wait(&full[st], (uint32_t)((j / n_stage) & 1), abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const Tile tl = tile_of(t, n_m, n_x, plane, 0, p.m_off);
            const int c = tl.m0 + 127 - mr;              // detector row of this lane
            // tile row of output row c's first optical-spread tap
            const float *tpt = reinterpret_cast<const float *>(smem + kHdr + (uint32_t)st * stage_bytes +
                                                               2u * wlo) + (127 - mr) * kTpPitch;
#pragma unroll
            for (int j0 = 0; j0 < kN; j0 += 16) {
                float v[16];
                tc::tmem_ld16(lane_base + (uint32_t)(buf * kN + j0), v);
                float r[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) r[i] = 0.0f;
                for (int jj = 0; jj <= 2 * rp; ++jj) {
                    const float g = p.gp[jj];
                    const float4 *row = reinterpret_cast<const float4 *>(tpt + jj * kTpPitch + j0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 x = row[i];
                        r[4 * i] = fmaf(g, x.x, r[4 * i]);
                        r[4 * i + 1] = fmaf(g, x.y, r[4 * i + 1]);
                        r[4 * i + 2] = fmaf(g, x.z, r[4 * i + 2]);
                        r[4 * i + 3] = fmaf(g, x.w, r[4 * i + 3]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) r[i] = p.n0 * (r[i] + p.spr * v[i]);
                if (c < p.n_v) {
                    const int xs = tl.x0 + j0;
                    float *dst = p.out0 + tl.img + (size_t)c * p.n_u + xs;
                    if (xs + 16 <= p.n_u && (p.n_u & 3) == 0) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            *reinterpret_cast<float4 *>(dst + i) =
                                make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (xs + i < p.n_u) dst[i] = r[i];
                    }
                }
            }
            tc::fence_before_sync();
            mbar_arrive(&acce[buf]);
            mbar_arrive(&empty[st]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicOr(p.err, 1u);
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kCols);
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

bool blur_tc_supported(const BlurParams &bp)
{
    return bp.rp >= 0 && bp.rp <= kTcMaxPsfR && bp.rs >= 0 && bp.rs <= kTcMaxScR;
}

static TcBlurParams tc_params(const BlurParams &bp, const uint16_t *hankel, unsigned int *err,
                              int n_img)
{
    TcBlurParams p;
    memset(&p, 0, sizeof(p));
    p.n_band = 2;
    p.H = hankel;
    p.n_u = bp.n_u;
    p.n_v = bp.n_v;
    p.n_img = n_img;
    p.n0 = bp.n0;
    p.spr = bp.spr;
    p.err = err;
    p.band[0] = make_band(nullptr, bp.rp, 0);
    p.band[1] = make_band(nullptr, bp.rs, (uint32_t)(2 * 64 * p.band[0].ncore));
    p.rp = bp.rp;
    for (int j = 0; j <= 2 * bp.rp && j < 2 * kTcMaxPsfR + 1; ++j) p.gp[j] = bp.gp[j];
    p.x_off = 0;
    p.x_cnt = (bp.n_v + kN - 1) / kN;
    p.ts_lo = 0;
    p.ts_hi = bp.n_v;
    p.ts_const = 0.0f;
    p.tp_lo = 0;
    p.tp_hi = bp.n_v;
    p.tp_const = 0.0f;
    p.m_off = 0;
    p.m_cnt = (bp.n_v + 127) / 128;
    // an injected timeout (testing) makes the epilogue give up its first
    // accumulator wait at once, which exercises the abort path
    p.epi_polls = bp.inject_timeout ? 0u : kPolls;
    return p;
}

static cudaError_t persistent_grid(long long tiles, int *grid)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *grid = (int)(tiles < sms ? tiles : sms);
    return cudaSuccess;
}

// Rows the tensor-core row pass computes when the rows of its input outside
// [one_lo, one_hi) are all ones (one_hi < 0: no such knowledge, every row):
// the 64-line tiles holding rows of [one_lo, one_hi), as tiles [x_off, x_off
// + x_cnt) and rows [r_lo, r_hi).
static void rows_computed(const BlurParams &bp, int one_lo, int one_hi, int &x_off, int &x_cnt, int &r_lo,
                          int &r_hi)
{
    x_off = 0;
    x_cnt = (bp.n_v + kN - 1) / kN;
    r_lo = 0;
    r_hi = bp.n_v;
    if (one_hi < 0) return;
    const int lo = one_lo > 0 ? one_lo : 0, hi = one_hi < bp.n_v ? one_hi : bp.n_v;
    if (lo >= hi) {
        x_cnt = 0;
        r_lo = r_hi = 0;
        return;
    }
    x_off = lo / kN;
    x_cnt = (hi - 1) / kN - x_off + 1;
    r_lo = x_off * kN;
    r_hi = (x_off + x_cnt) * kN < bp.n_v ? (x_off + x_cnt) * kN : bp.n_v;
}

// the row pass of an all-ones row: the sums of the taps
static void ones_row_pass(const BlurParams &bp, float &vp, float &vs)
{
    vp = 0.0f;
    vs = 0.0f;
    for (int j = 0; j <= 2 * bp.rp; ++j) vp += bp.gp[j];
    for (int j = 0; j <= 2 * bp.rs; ++j) vs += bp.gs[j];
}

// Rows [0, r_lo) and [r_hi, n_v) of image blockIdx.y of tp get the constant
// vp (the column pass's output rows that see only constant inputs).  VEC:
// four floats per store (n_u a multiple of 4 and tp 16-byte aligned, so no
// store straddles the gap between the two row ranges).
template <bool VEC>
__global__ void __launch_bounds__(256)
k_fill_const_rows(float *__restrict__ tp, float vp, int n_u, int n_v, int r_lo, int r_hi)
{
    constexpr int w = VEC ? 4 : 1;
    const size_t lo = (size_t)r_lo * n_u / w, hs = (size_t)r_hi * n_u / w, end = (size_t)n_v * n_u / w;
    const size_t n_fill = lo + (end - hs);
    const size_t base = (size_t)blockIdx.y * end;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_fill;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = base + (e < lo ? e : hs + (e - lo));
        if (VEC)
            reinterpret_cast<float4 *>(tp)[i] = make_float4(vp, vp, vp, vp);
        else
            tp[i] = vp;
    }
}

// one_lo, one_hi: when one_hi >= 0, every row of `in` outside [one_lo,
// one_hi) is known to be all ones (the primary of rays that cannot meet the
// voxels).  Only the 64-line tiles that hold rows of [one_lo, one_hi) are
// computed; the other rows of tp and ts are left unwritten, and the column
// pass (given the same one_lo, one_hi) takes for them the row pass of an
// all-ones row, the sum of each kernel's taps.
cudaError_t launch_blur_tc_rows(const BlurParams &bp, const float *in, float *tp, float *ts,
                                uint16_t *hankel, unsigned int *err, int n_img, cudaStream_t s,
                                int one_lo, int one_hi)
{
    if (n_img <= 0) return cudaSuccess;
    if (!blur_tc_supported(bp)) return cudaErrorInvalidValue;
    TcBlurParams p = tc_params(bp, hankel, err, n_img);
    k_blur_hankel<<<16, 256, 0, s>>>(bp, p, hankel);
    p.band[0].src = in;
    p.band[1].src = in;
    p.out0 = tp;
    p.out1 = ts;
    const int kw = p.band[0].kw > p.band[1].kw ? p.band[0].kw : p.band[1].kw;
    const size_t fixed = kHdr + 2u * 128u * (size_t)(p.band[0].ncore + p.band[1].ncore);
    const size_t stage = 4u * kN * (size_t)kw;
    const int n_stage = fixed + 2 * stage <= kSmemLimit ? 2 : 1;
    const size_t bytes = fixed + n_stage * stage;
    if (bytes > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_blur_rows_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    int r_lo, r_hi;                                // rows the tensor-core pass computes
    rows_computed(bp, one_lo, one_hi, p.x_off, p.x_cnt, r_lo, r_hi);
    if (p.x_cnt > 0) {
        const long long tiles = (long long)((bp.n_u + 127) / 128) * p.x_cnt * n_img;
        int grid = 0;
        if ((e = persistent_grid(tiles, &grid)) != cudaSuccess) return e;
        k_blur_rows_tc<<<grid, kThreads, bytes, s>>>(p, n_stage);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    (void)r_lo;
    (void)r_hi;
    return cudaGetLastError();
}

void blur_tc_rows_read(const BlurParams &bp, int one_lo, int one_hi, int *lo, int *hi)
{
    int x_off, x_cnt;
    rows_computed(bp, one_lo, one_hi, x_off, x_cnt, *lo, *hi);
}

// Kernels launch_blur_tc_rows starts: band matrices and the tensor-core pass
// (unless no tile is computed).  The rows it skips are not written: the
// column pass takes the constant they stand for.
int blur_tc_rows_launches(const BlurParams &bp, int one_lo, int one_hi)
{
    int x_off, x_cnt, r_lo, r_hi;
    rows_computed(bp, one_lo, one_hi, x_off, x_cnt, r_lo, r_hi);
    return 1 + (x_cnt > 0);
}

// Output rows the tensor-core column pass computes when the rows of the
// primary outside [one_lo, one_hi) are all ones: every row within R (the
// larger radius) of that band, as 128-row tiles from m_off (a multiple of 8,
// so a window item of 8 rows never straddles a computed-tile edge of the row
// pass); the other output rows see only constant inputs.  Without that
// knowledge (one_hi < 0): every row.
static void out_rows_computed(const BlurParams &bp, int one_lo, int one_hi, int &m_off, int &m_cnt)
{
    m_off = 0;
    m_cnt = (bp.n_v + 127) / 128;
    if (one_hi < 0) return;
    const int R = bp.rs > bp.rp ? bp.rs : bp.rp;
    const int lo_b = one_lo > 0 ? one_lo : 0, hi_b = one_hi < bp.n_v ? one_hi : bp.n_v;
    if (lo_b >= hi_b) {
        m_cnt = 0;
        return;
    }
    const int lo = lo_b - R > 0 ? lo_b - R : 0;
    const int hi = hi_b + R < bp.n_v ? hi_b + R : bp.n_v;
    m_off = lo & ~7;
    m_cnt = (hi - m_off + 127) / 128;
}

// Kernels launch_blur_tc_cols starts: the tensor-core pass (unless no tile is
// computed) and the constant fill of the other output rows.
int blur_tc_cols_launches(const BlurParams &bp, int one_lo, int one_hi)
{
    int m_off, m_cnt;
    out_rows_computed(bp, one_lo, one_hi, m_off, m_cnt);
    const int hi = m_off + 128 * m_cnt < bp.n_v ? m_off + 128 * m_cnt : bp.n_v;
    return (m_cnt > 0) + (hi - m_off < bp.n_v);
}

// one_lo, one_hi: as for launch_blur_tc_rows with the same values; the rows
// of tp and ts that pass did not compute are taken as the constants they
// stand for.  Only the output rows within the larger radius of [one_lo,
// one_hi) are computed on the tensor cores (whole 128-row tiles); every
// other output row sees constant inputs only and gets the column pass of
// those constants from a store-only kernel.
cudaError_t launch_blur_tc_cols(const BlurParams &bp, const float *tp, const float *ts, float *out,
                                const uint16_t *hankel, unsigned int *err, int n_img, cudaStream_t s,
                                int one_lo, int one_hi)
{
    if (n_img <= 0) return cudaSuccess;
    if (!blur_tc_supported(bp)) return cudaErrorInvalidValue;
    TcBlurParams p = tc_params(bp, hankel, err, n_img);
    {
        int x_off, x_cnt;
        rows_computed(bp, one_lo, one_hi, x_off, x_cnt, p.ts_lo, p.ts_hi);
        p.tp_lo = p.ts_lo;
        p.tp_hi = p.ts_hi;
        ones_row_pass(bp, p.tp_const, p.ts_const);
        out_rows_computed(bp, one_lo, one_hi, p.m_off, p.m_cnt);
    }
    p.band[1].src = ts;
    p.tp = tp;
    p.out0 = out;
    const size_t tp_bytes = ((size_t)(128 + 2 * bp.rp) * kTpPitch * 4u + 127u) & ~(size_t)127u;
    const size_t stage = 4u * kN * (size_t)p.band[1].kw + tp_bytes;
    const int n_stage = kHdr + 2 * stage <= kSmemLimit ? 2 : 1;
    size_t bytes = kHdr + n_stage * stage;
    if (bytes > kSmemLimit || 2 * kN + p.band[1].kw > 512) return cudaErrorInvalidValue;
    // the kernel takes all 512 TMEM columns: reserve enough shared memory that
    // a second CTA never shares the SM (its allocation would wait for ours)
    if (bytes < kSmemLimit / 2 + 1024) bytes = kSmemLimit / 2 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_blur_cols_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    if (p.m_cnt > 0) {
        const long long tiles = (long long)p.m_cnt * ((bp.n_u + kN - 1) / kN) * n_img;
        int grid = 0;
        if ((e = persistent_grid(tiles, &grid)) != cudaSuccess) return e;
        k_blur_cols_tc<<<grid, kThreads, bytes, s>>>(p, n_stage);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int r_lo = p.m_cnt > 0 ? p.m_off : 0;
    const int r_hi = p.m_cnt > 0 ? (p.m_off + 128 * p.m_cnt < bp.n_v ? p.m_off + 128 * p.m_cnt : bp.n_v) : 0;
    if (r_hi - r_lo < bp.n_v) {
        // output rows whose every tap reads constant inputs: the column pass
        // of the constant rows, n0 (vp sum g_psf + spr vs sum g_scatter)
        double sp = 0.0, ss = 0.0;
        for (int j = 0; j <= 2 * bp.rp; ++j) sp += bp.gp[j];
        for (int j = 0; j <= 2 * bp.rs; ++j) ss += bp.gs[j];
        const float c = (float)((double)bp.n0 * ((double)p.tp_const * sp + (double)bp.spr * (double)p.ts_const * ss));
        const bool vec = bp.n_u % 4 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0;
        const size_t per = (size_t)(bp.n_v - (r_hi - r_lo)) * bp.n_u / (vec ? 4 : 1);
        const size_t want = (per + 256 * 8 - 1) / (256 * 8);
        if (n_img > 65535) return cudaErrorInvalidValue;
        dim3 fgrid((unsigned)(want < 1024 ? want : 1024), n_img);
        if (vec)
            k_fill_const_rows<true><<<fgrid, 256, 0, s>>>(out, c, bp.n_u, bp.n_v, r_lo, r_hi);
        else
            k_fill_const_rows<false><<<fgrid, 256, 0, s>>>(out, c, bp.n_u, bp.n_v, r_lo, r_hi);
    }
    return cudaGetLastError();
}

}  // namespace fc

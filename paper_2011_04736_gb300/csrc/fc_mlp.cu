// Learned surrogate of the energy integral: ln T(L) from the per-material
// path lengths L of a ray (the quantity the projector's energy loop
// computes, paper Sec. II.F, I_f equation), replacing the N_E-bin sum.
//
//   ln T ~ ln sum_k a_k exp(-sum_m mu_km L_m) + MLP(L * scale)
//   MLP: 8 -> 128 -> 128 -> 128 -> 1, SiLU activations.
// The baseline is the energy integral with the spectrum lumped into four
// groups of equal weight (a_k = group weight, mu_km = group-mean
// attenuation); with one group it is the first-order term -mubar . L.  The
// network learns the residual of this baseline.
//
// The three 128-wide layers run on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, bf16 operands in shared memory, f32 accumulators
// in tensor memory); biases, SiLU and the 128 -> 1 output layer run in the
// epilogues.  Activations are carried as two bf16 parts, hi = bf16(h) and
// lo = bf16(h - hi), and each layer multiplies both (W hi + W lo), so the
// activations keep ~16 significant bits while every product is a bf16
// tensor-core product; the 8 inputs use the same split, with the lo part in
// the padded K columns 8..15 and W1 duplicated there.  One CTA handles tiles of 128 rays; thread r of the 128 owns
// ray r of the tile (TMEM lane r).
//
// Training: a fused forward + backward kernel per 128-sample tile keeps the
// three pre-activations in TMEM (384 of 512 columns) and the data-gradient
// accumulator in the rest; it writes the activations and back-propagated
// errors feature-major, [feature][batch], so that the weight gradients
// dW = dZ^T H are split-K tensor-core GEMMs over the batch (k_mlp_wgrad).
// k_mlp_adam sums the split-K partials and applies Adam.
//
// Every wait on the tensor core is a bounded mbarrier poll; on expiry the
// kernel records FC_ETIMEOUT in an error word, skips the dependent work,
// releases its TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "fc_internal.cuh"
#include "fc_tc.cuh"

namespace fc {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kH = kMlpHidden;       // 128
constexpr int kInP = 16;             // inputs padded to one MMA K-step
constexpr uint32_t kKgs128 = (kH / 8) * 128;   // k-group stride of a 128-row operand
constexpr uint32_t kPolls = 1u << 24;          // bounded mbarrier polls (~0.5 s)

__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sigma(z) = (1 + tanh(z / 2)) / 2, the logistic function
__device__ __forceinline__ float sigma_fast(float z) { return fmaf(0.5f, tanh_fast(0.5f * z), 0.5f); }

// SiLU(z) = z sigma(z)
__device__ __forceinline__ float silu(float z) { return z * sigma_fast(z); }

// SiLU of a pair with packed binary32 arithmetic (each element rounded as
// the scalar silu rounds it).
__device__ __forceinline__ float2 silu2(float2 z)
{
    const float2 half = make_float2(0.5f, 0.5f);
    const float2 hz = __fmul2_rn(z, half);
    const float2 t = make_float2(tanh_fast(hz.x), tanh_fast(hz.y));
    return __fmul2_rn(z, __ffma2_rn(half, t, half));
}

// d SiLU / dz = sigma + z sigma (1 - sigma)
__device__ __forceinline__ float dsilu(float z)
{
    const float s = sigma_fast(z);
    return fmaf(z * s, 1.0f - s, s);
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Copy a row-major bf16 matrix [rows][k] from global memory into the K-major
// no-swizzle operand layout (16-byte chunks = one core-matrix row each).
__device__ __forceinline__ void stage_kmajor(unsigned char *dst, const bf16 *src, int rows, int k,
                                             uint32_t kgs)
{
    const int chunks = rows * (k / 8);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        const int r = c / (k / 8), kc = (c % (k / 8)) * 8;
        *reinterpret_cast<uint4 *>(dst + tc::kmajor_off(r, kc, kgs)) =
            *reinterpret_cast<const uint4 *>(src + (size_t)r * k + kc);
    }
}

// Issue the K/16 MMAs of D[128 x N] (+)= A[128 x K] B[N x K]^T.
__device__ __forceinline__ void issue_gemm(uint32_t d, const unsigned char *a, uint32_t kgsa,
                                           const unsigned char *b, uint32_t kgsb, int K, int N,
                                           bool accumulate_first)
{
    const uint32_t id = tc::idesc_bf16(128, N);
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t ad = tc::sdesc(tc::smem_u32(a) + ks * 2 * kgsa, kgsa, 128);
        const uint64_t bd = tc::sdesc(tc::smem_u32(b) + ks * 2 * kgsb, kgsb, 128);
        tc::mma_bf16(d, ad, bd, id, (ks > 0 || accumulate_first) ? 1u : 0u);
    }
}

// Barrier of the nt threads that share a tile: bar 0 is the whole CTA
// (__syncthreads), bar > 0 the named barrier of one group of nt threads.
__device__ __forceinline__ void tile_sync(int bar, int nt = 128)
{
    if (bar == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" :: "r"(bar), "r"(nt) : "memory");
}

// tile_sync that also returns whether ok holds on every thread of the barrier.
__device__ __forceinline__ bool tile_sync_and(int bar, bool ok, int nt = 128)
{
    if (bar == 0) return __syncthreads_and(ok);
    uint32_t all;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.and.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(all) : "r"((uint32_t)ok), "r"(bar), "r"(nt) : "memory");
    return all != 0;
}

// Make shared-memory writes visible to the tensor core and order
// tensor-memory accesses around the barrier of the tile's threads.
__device__ __forceinline__ void sync_for_mma(int bar = 0, int nt = 128)
{
    tc::fence_async_smem();
    tc::fence_before_sync();
    tile_sync(bar, nt);
    tc::fence_after_sync();
}

// The first thread of the tile's group (nt threads, a power of two) issues a
// GEMM and commits; the group waits for it.  Returns false (and records the
// timeout) if the wait bound is exhausted.
__device__ __forceinline__ bool run_gemm(uint32_t d, const unsigned char *a, uint32_t kgsa,
                                         const unsigned char *b, uint32_t kgsb, int K, int N,
                                         uint64_t *mbar, uint32_t &phase, int *err, int bar = 0,
                                         int nt = 128)
{
    const bool issuer = (threadIdx.x & (nt - 1)) == 0;
    if (issuer) {
        issue_gemm(d, a, kgsa, b, kgsb, K, N, false);
        tc::mma_commit(mbar);
    }
    const bool ok = tc::mbar_wait(mbar, phase, kPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok && issuer) atomicExch(err, FC_ETIMEOUT);
    return tile_sync_and(bar, ok, nt);
}

// Per-lane TMEM address of this thread's row (row = thread index mod 128; a
// warp reaches the lanes of its index mod 4), column col.
__device__ __forceinline__ uint32_t trow(uint32_t tbase, int col)
{
    return tbase + ((uint32_t)(threadIdx.x & 96) << 16) + (uint32_t)col;
}

// Epilogue: h = SiLU(acc + bias) of this thread's row, columns [c_lo, c_hi)
// (CW columns per tensor-memory load, c_hi - c_lo a multiple of CW) -> row
// r of the K-major operands dst (bf16(h)) and dlo (bf16(h - bf16(h))), and,
// if ht != nullptr, the feature-major global copy ht[j * ldh + col] of
// bf16(h).
template <int CW = 16>
__device__ __forceinline__ void epi_silu(uint32_t tacc, const float *bias, unsigned char *dst,
                                         unsigned char *dlo, bf16 *ht, size_t ldh, size_t col,
                                         int c_lo = 0, int c_hi = kH)
{
    static_assert(CW == 16 || CW == 32, "16 or 32 columns per load");
    const int r = threadIdx.x & 127;
#pragma unroll 1
    for (int cl = c_lo; cl < c_hi; cl += CW) {
        float vw[CW];
        if constexpr (CW == 32)
            tc::tmem_ld32(tacc + cl, vw);
        else
            tc::tmem_ld16(tacc + cl, vw);
#pragma unroll
        for (int hh = 0; hh < CW / 16; ++hh) {
            const int c0 = cl + 16 * hh;
            const float *v = vw + 16 * hh;
            uint32_t p[8], q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 h = silu2(__fadd2_rn(make_float2(v[2 * i], v[2 * i + 1]),
                                                  *reinterpret_cast<const float2 *>(bias + c0 + 2 * i)));
                p[i] = pack2(h.x, h.y);
                const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&p[i]);
                // h - bf16(h), exact (the multiply by -1 is exact)
                const float2 lo = __ffma2_rn(__bfloat1622float2(hb), make_float2(-1.0f, -1.0f), h);
                q[i] = pack2(lo.x, lo.y);
                if (ht) {
                    ht[(size_t)(c0 + 2 * i) * ldh + col] = hb.x;
                    ht[(size_t)(c0 + 2 * i + 1) * ldh + col] = hb.y;
                }
            }
            *reinterpret_cast<uint4 *>(dst + tc::kmajor_off(r, c0, kKgs128)) =
                make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4 *>(dst + tc::kmajor_off(r, c0 + 8, kKgs128)) =
                make_uint4(p[4], p[5], p[6], p[7]);
            *reinterpret_cast<uint4 *>(dlo + tc::kmajor_off(r, c0, kKgs128)) =
                make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(dlo + tc::kmajor_off(r, c0 + 8, kKgs128)) =
                make_uint4(q[4], q[5], q[6], q[7]);
        }
    }
}

// Stage this thread's inputs x = L * scale as hi (K columns 0..7) and lo
// (columns 8..15) parts into row r of the 128 x 16 operand; optionally the
// feature-major copy xt[k * ldx + col].
__device__ __forceinline__ void stage_x(unsigned char *sX, const float (&Lr)[kMaxMat],
                                        const float *scale, bf16 *xt, size_t ldx, size_t col)
{
    uint32_t q[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float a = Lr[2 * k] * scale[2 * k], b = Lr[2 * k + 1] * scale[2 * k + 1];
        q[k] = pack2(a, b);
        const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&q[k]);
        q[k + 4] = pack2(a - __low2float(hb), b - __high2float(hb));
    }
    const int r = threadIdx.x & 127;
    *reinterpret_cast<uint4 *>(sX + tc::kmajor_off(r, 0, kKgs128)) = make_uint4(q[0], q[1], q[2], q[3]);
    *reinterpret_cast<uint4 *>(sX + tc::kmajor_off(r, 8, kKgs128)) = make_uint4(q[4], q[5], q[6], q[7]);
    if (xt) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&q[k]);
            xt[(size_t)(2 * k) * ldx + col] = hb.x;
            xt[(size_t)(2 * k + 1) * ldx + col] = hb.y;
        }
    }
}

// The group's first thread issues D = A_hi B^T + A_lo B^T (K = 128) and
// commits; the group waits.  Returns false (and records the timeout) if the
// wait bound expires.
__device__ __forceinline__ bool run_gemm_split(uint32_t d, const unsigned char *ahi,
                                               const unsigned char *alo, const unsigned char *b,
                                               uint64_t *mbar, uint32_t &phase, int *err, int bar = 0,
                                               int nt = 128)
{
    const bool issuer = (threadIdx.x & (nt - 1)) == 0;
    if (issuer) {
        issue_gemm(d, ahi, kKgs128, b, kKgs128, kH, kH, false);
        issue_gemm(d, alo, kKgs128, b, kKgs128, kH, kH, true);
        tc::mma_commit(mbar);
    }
    const bool ok = tc::mbar_wait(mbar, phase, kPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok && issuer) atomicExch(err, FC_ETIMEOUT);
    return tile_sync_and(bar, ok, nt);
}

// Exact ln T from path lengths: the projector's energy-integral epilogue.
__device__ __forceinline__ float exact_lnT(const float (&L)[kMaxMat], const float *wd,
                                           const float (*mu2)[kMaxMat], int n_e)
{
    float sum = 0.0f, comp = 0.0f;
    for (int e = 0; e < n_e; ++e) {
        float a = 0.0f;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) a = fmaf(mu2[e][m], L[m], a);
        const float term = wd[e] * exp2_hw(-a);
        const float y = term - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    return logf(sum);
}

// Spectral-group baseline ln sum_k a_k exp(-sum_m mu_km L_m); g holds a[4]
// then mu[4][8] (mu in 1/cm).
__device__ __forceinline__ float group_base(const float (&L)[kMaxMat], const float *g)
{
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kMlpGroups; ++k) {
        float a = 0.0f;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) a = fmaf(g[kMlpGroups + k * kMaxMat + m], L[m], a);
        s = fmaf(g[k], __expf(-a), s);
    }
    return __logf(s);
}

// shared-memory map of the inference kernel (bytes): the weights once, then
// per group of 128 threads its own X / H / Hlo operands
constexpr int kInfGroups = 2;
constexpr int kInfW1 = 0, kInfW2 = 4096, kInfW3 = 4096 + 32768, kInfG0 = 4096 + 2 * 32768;
constexpr int kInfX = 0, kInfH = 4096, kInfHlo = kInfH + 32768, kInfGroupBytes = kInfHlo + 32768;
constexpr int kInfGroupThreads = 256;     // two threads per row: columns 0-63 and 64-127
constexpr int kInfPart = kInfG0 + kInfGroups * kInfGroupBytes;   // [groups][128] partial sums
constexpr int kInfF = kInfPart + kInfGroups * 128 * 4;
constexpr int kInfSmem = kInfF + (4 * kH + 2 * kMaxMat + kMlpGroups * (kMaxMat + 1) + 8) * 4;

}  // namespace

// ---------------------------------------------------------------- inference
// Two groups of 256 threads (8 warps each) share the resident weights and
// the tensor core, each working through its own tiles of 128 rays with its
// own operands in shared memory, accumulator in tensor memory (columns
// 128 g .. 128 g + 127), mbarrier and named barrier: while one group runs
// its SiLU epilogue on the CUDA cores the other group's MMAs run.  Within a
// group, row r is served by two threads (warps 0-3 and 4-7 reach the same
// tensor-memory lanes), one for hidden units 0-63 and one for 64-127; the
// first owns the ray (inputs, baseline, result, fallback).
__global__ void __launch_bounds__(kInfGroupThreads * kInfGroups)
k_mlp_eval(const __grid_constant__ SurrogateParams p, const float *__restrict__ L, long long n,
           float *__restrict__ lnT, unsigned int *n_fallback, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[kInfGroups];
    __shared__ uint32_t tbase_s;
    constexpr int NT = kInfGroupThreads;
    const int g = threadIdx.x / NT;                 // group
    const int r = threadIdx.x & 127;                // row of the group's tile
    const bool owner = (threadIdx.x & (NT - 1)) < 128;
    const int c_lo = owner ? 0 : kH / 2, c_hi = c_lo + kH / 2;
    const int bar = 1 + g;                          // the group's named barrier
    unsigned char *sW1 = smem + kInfW1, *sW2 = smem + kInfW2, *sW3 = smem + kInfW3;
    unsigned char *grp_smem = smem + kInfG0 + g * kInfGroupBytes;
    unsigned char *sX = grp_smem + kInfX, *sH = grp_smem + kInfH, *sHlo = grp_smem + kInfHlo;
    float *part = reinterpret_cast<float *>(smem + kInfPart) + g * 128;
    float *fb = reinterpret_cast<float *>(smem + kInfF);
    float *b1 = fb, *b2 = fb + kH, *b3 = fb + 2 * kH, *w4 = fb + 3 * kH;
    float *scale = fb + 4 * kH, *box = scale + kMaxMat, *grp = box + kMaxMat;
    if (threadIdx.x < 32) tc::tmem_alloc(&tbase_s, 128 * kInfGroups);
    if (threadIdx.x < kInfGroups) tc::mbar_init(&mbar[threadIdx.x], 1);
    stage_kmajor(sW1, p.W1b, kH, kInP, kKgs128);
    stage_kmajor(sW2, p.W2b, kH, kH, kKgs128);
    stage_kmajor(sW3, p.W3b, kH, kH, kKgs128);
    const float *P = p.P;
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        b1[i] = P[kOffB1 + i];
        b2[i] = P[kOffB2 + i];
        b3[i] = P[kOffB3 + i];
        w4[i] = P[kOffW4 + i];
    }
    if (threadIdx.x < kMaxMat) {
        scale[threadIdx.x] = P[kOffScale + threadIdx.x];
        box[threadIdx.x] = P[kOffBox + threadIdx.x];
    }
    if (threadIdx.x < kMlpGroups * (kMaxMat + 1)) grp[threadIdx.x] = P[kOffGa + threadIdx.x];
    const float b4 = P[kOffB4];
    sync_for_mma();                                  // whole CTA
    const uint32_t tb = tbase_s + 128u * (uint32_t)g;
    uint64_t *mb = &mbar[g];
    uint32_t phase = 0;
    unsigned int my_fallback = 0;
    const long long ntiles = (n + 127) / 128;
    const long long stride = (long long)gridDim.x * kInfGroups;
    // inputs of the group's next tile, loaded one tile ahead by the owner
    float Ln[kMaxMat];
    {
        const long long i0 = ((long long)blockIdx.x * kInfGroups + g) * 128 + r;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m)
            Ln[m] = (owner && i0 < n && m < p.n_mat) ? L[i0 * p.n_mat + m] : 0.0f;
    }
    for (long long tile = (long long)blockIdx.x * kInfGroups + g; tile < ntiles; tile += stride) {
        const long long i = tile * 128 + r;
        const bool valid = i < n;
        float Lr[kMaxMat];
        bool outside = false;
        float ylin = 0.0f;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) Lr[m] = Ln[m];
        if (owner) {
#pragma unroll
            for (int m = 0; m < kMaxMat; ++m) outside = outside || Lr[m] > box[m];
            ylin = group_base(Lr, grp);
            stage_x(sX, Lr, scale, nullptr, 0, 0);
            const long long in = i + stride * 128;
#pragma unroll
            for (int m = 0; m < kMaxMat; ++m) Ln[m] = (in < n && m < p.n_mat) ? L[in * p.n_mat + m] : 0.0f;
        }
        sync_for_mma(bar, NT);
        if (!run_gemm(tb, sX, kKgs128, sW1, kKgs128, kInP, kH, mb, phase, err, bar, NT)) break;
        epi_silu<32>(trow(tb, 0), b1, sH, sHlo, nullptr, 0, 0, c_lo, c_hi);
        sync_for_mma(bar, NT);
        if (!run_gemm_split(tb, sH, sHlo, sW2, mb, phase, err, bar, NT)) break;
        epi_silu<32>(trow(tb, 0), b2, sH, sHlo, nullptr, 0, 0, c_lo, c_hi);
        sync_for_mma(bar, NT);
        if (!run_gemm_split(tb, sH, sHlo, sW3, mb, phase, err, bar, NT)) break;
        float res = owner ? b4 : 0.0f;
#pragma unroll 1
        for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
            float v[32];
            tc::tmem_ld32(trow(tb, c0), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) res = fmaf(w4[c0 + j], silu(v[j] + b3[c0 + j]), res);
        }
        if (!owner) part[r] = res;
        // the partial sums exchanged; every tensor-memory read of this tile
        // is complete before the group's next MMA
        tc::fence_before_sync();
        tile_sync(bar, NT);
        tc::fence_after_sync();
        if (owner && valid) {
            float y = ylin + (res + part[r]);
            // outside the training box, or attenuated as strongly as a ray
            // the guard saw miss the tolerance: the exact sum decides
            if (outside || -ylin >= p.guard) {
                y = exact_lnT(Lr, p.wd, p.mu2, p.n_e);
                ++my_fallback;
            }
            lnT[i] = y;
        }
    }
    if (my_fallback) atomicAdd(n_fallback, my_fallback);
    tc::fence_before_sync();
    __syncthreads();                                 // both groups done with tensor memory
    if (threadIdx.x < 32) tc::tmem_dealloc(tbase_s, 128 * kInfGroups);
}

// Order-preserving integer image of a float (smaller float, smaller int).
__device__ __forceinline__ int ordered_int(float v)
{
    const int b = __float_as_int(v);
    return b >= 0 ? b : b ^ 0x7fffffff;
}

__global__ void __launch_bounds__(256)
k_guard_scan(const __grid_constant__ SurrogateParams p, const float *__restrict__ L,
             const float *__restrict__ y, const float *__restrict__ ys, long long n, float tol,
             int *best)
{
    int mine = 0x7fffffff;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!(fabsf(ys[i] - y[i]) > tol)) continue;
        float Lr[kMaxMat];
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) Lr[m] = m < p.n_mat ? L[i * p.n_mat + m] : 0.0f;
        mine = min(mine, ordered_int(-group_base(Lr, p.P + kOffGa)));
    }
    for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(0xffffffffu, mine, o));
    if ((threadIdx.x & 31) == 0 && mine != 0x7fffffff) atomicMin(best, mine);
}

cudaError_t launch_guard_scan(const SurrogateParams &p, const float *L, const float *y,
                              const float *ys, long long n, float tol, int *best, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    k_guard_scan<<<(int)blocks, 256, 0, s>>>(p, L, y, ys, n, tol, best);
    return cudaGetLastError();
}

// sigma of every element, as the surrogate kernels evaluate it (the error
// of the activations is measured through this kernel).
__global__ void __launch_bounds__(256) k_sigma_probe(const float *__restrict__ z, float *__restrict__ s,
                                                     long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s[i] = sigma_fast(z[i]);
}

cudaError_t launch_sigma_probe(const float *z, float *s, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    k_sigma_probe<<<(int)blocks, 256, 0, st>>>(z, s, n);
    return cudaGetLastError();
}

// Exact ln T of each ray from its path lengths (the plain energy-sum path).
__global__ void __launch_bounds__(256)
k_energy_sum_lengths(const __grid_constant__ SurrogateParams p, const float *__restrict__ L,
                     long long n, float *__restrict__ lnT)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float Lr[kMaxMat];
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) Lr[m] = m < p.n_mat ? L[i * p.n_mat + m] : 0.0f;
        lnT[i] = exact_lnT(Lr, p.wd, p.mu2, p.n_e);
    }
}

// ---------------------------------------------------------------- training
namespace {
// shared-memory map of the training kernel (bytes)
constexpr int kTrW1 = 0, kTrW2 = 4096, kTrW3 = kTrW2 + 32768, kTrW2T = kTrW3 + 32768,
              kTrW3T = kTrW2T + 32768, kTrX = kTrW3T + 32768, kTrH = kTrX + 4096,
              kTrD = kTrH + 32768, kTrF = kTrD + 32768;
constexpr int kTrSmem = kTrF + (4 * kH + kMaxMat + kMlpGroups * (kMaxMat + 1) + 8) * 4;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
}  // namespace

// One training step's forward and backward for tiles of 128 samples.
// Writes (feature-major, [feature][batch]): xt [16][B], h1t, h2t, h3t,
// dz1t, dz2t, dz3t [128][B], and g [16][B] whose row 0 holds dLoss/dy_hat
// (rows 1..15 stay zero); adds the batch's summed squared error to *loss.
__global__ void __launch_bounds__(128, 1)
k_mlp_train(const __grid_constant__ SurrogateParams p, const float *__restrict__ L,
            const float *__restrict__ y, long long n, int B, int sample, unsigned long long seed,
            int step, MlpWork w, float *loss, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase_s;
    __shared__ float red[4];
    unsigned char *sW1 = smem + kTrW1, *sW2 = smem + kTrW2, *sW3 = smem + kTrW3;
    unsigned char *sW2T = smem + kTrW2T, *sW3T = smem + kTrW3T;
    unsigned char *sX = smem + kTrX, *sH = smem + kTrH, *sD = smem + kTrD;
    float *fb = reinterpret_cast<float *>(smem + kTrF);
    float *b1 = fb, *b2 = fb + kH, *b3 = fb + 2 * kH, *w4 = fb + 3 * kH;
    float *scale = fb + 4 * kH, *grp = scale + kMaxMat;
    const int r = threadIdx.x;
    if (r < 32) tc::tmem_alloc(&tbase_s, 512);
    if (r == 0) tc::mbar_init(&mbar, 1);
    stage_kmajor(sW1, p.W1b, kH, kInP, kKgs128);
    stage_kmajor(sW2, p.W2b, kH, kH, kKgs128);
    stage_kmajor(sW3, p.W3b, kH, kH, kKgs128);
    stage_kmajor(sW2T, p.W2Tb, kH, kH, kKgs128);
    stage_kmajor(sW3T, p.W3Tb, kH, kH, kKgs128);
    const float *P = p.P;
    for (int i = r; i < kH; i += blockDim.x) {
        b1[i] = P[kOffB1 + i];
        b2[i] = P[kOffB2 + i];
        b3[i] = P[kOffB3 + i];
        w4[i] = P[kOffW4 + i];
    }
    if (r < kMaxMat) scale[r] = P[kOffScale + r];
    if (r < kMlpGroups * (kMaxMat + 1)) grp[r] = P[kOffGa + r];
    const float b4 = P[kOffB4];
    sync_for_mma();
    const uint32_t tb = tbase_s;
    const uint32_t tZ1 = trow(tb, 0), tZ2 = trow(tb, 128), tZ3 = trow(tb, 256), tD = trow(tb, 384);
    uint32_t phase = 0;
    float sq = 0.0f;
    const int ntiles = (B + 127) / 128;
    const float inv_b = 1.0f / (float)B;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int col = tile * 128 + r;   // position in the batch
        const bool valid = col < B;
        long long idx = col;
        if (sample) idx = (long long)(mix64(seed ^ mix64(((unsigned long long)step << 32) | (unsigned)col)) % (unsigned long long)n);
        float Lr[kMaxMat];
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) Lr[m] = (valid && m < p.n_mat) ? L[idx * p.n_mat + m] : 0.0f;
        const float ylin = group_base(Lr, grp);
        const float yt = valid ? y[idx] : 0.0f;
        stage_x(sX, Lr, scale, valid ? w.xt : nullptr, B, col);
        sync_for_mma();
        // forward: Z1, Z2, Z3 stay in TMEM columns [0,128), [128,256), [256,384);
        // sD holds the lo parts of the activations until the backward pass
        if (!run_gemm(tb, sX, kKgs128, sW1, kKgs128, kInP, kH, &mbar, phase, err)) break;
        epi_silu(tZ1, b1, sH, sD, valid ? w.h1t : nullptr, B, col);
        sync_for_mma();
        if (!run_gemm_split(tb + 128, sH, sD, sW2, &mbar, phase, err)) break;
        epi_silu(tZ2, b2, sH, sD, valid ? w.h2t : nullptr, B, col);
        sync_for_mma();
        if (!run_gemm_split(tb + 256, sH, sD, sW3, &mbar, phase, err)) break;
        float res = b4;
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tZ3 + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float h = silu(v[j] + b3[c0 + j]);
                res = fmaf(w4[c0 + j], h, res);
                if (valid) w.h3t[(size_t)(c0 + j) * B + col] = __float2bfloat16_rn(h);
            }
        }
        const float e = valid ? (ylin + res - yt) : 0.0f;
        sq = fmaf(e, e, sq);
        const float gr = 2.0f * e * inv_b;   // dLoss / dy_hat for this sample
        if (valid) w.g[col] = __float2bfloat16_rn(gr);
        // dZ3 = g w4 SiLU'(Z3)
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tZ3 + c0, v);
            uint32_t q[8];
#pragma unroll
            for (int i2 = 0; i2 < 8; ++i2) {
                const float a = gr * w4[c0 + 2 * i2] * dsilu(v[2 * i2] + b3[c0 + 2 * i2]);
                const float b = gr * w4[c0 + 2 * i2 + 1] * dsilu(v[2 * i2 + 1] + b3[c0 + 2 * i2 + 1]);
                q[i2] = pack2(a, b);
                if (valid) {
                    const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&q[i2]);
                    w.dz3t[(size_t)(c0 + 2 * i2) * B + col] = hb.x;
                    w.dz3t[(size_t)(c0 + 2 * i2 + 1) * B + col] = hb.y;
                }
            }
            *reinterpret_cast<uint4 *>(sD + tc::kmajor_off(r, c0, kKgs128)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(sD + tc::kmajor_off(r, c0 + 8, kKgs128)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        sync_for_mma();
        // dH2 = dZ3 W3  (B operand W3^T: rows = layer input, K = layer output)
        if (!run_gemm(tb + 384, sD, kKgs128, sW3T, kKgs128, kH, kH, &mbar, phase, err)) break;
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float dv[16], zv[16];
            tc::tmem_ld16(tD + c0, dv);
            tc::tmem_ld16(tZ2 + c0, zv);
            uint32_t q[8];
#pragma unroll
            for (int i2 = 0; i2 < 8; ++i2) {
                const float a = dv[2 * i2] * dsilu(zv[2 * i2] + b2[c0 + 2 * i2]);
                const float b = dv[2 * i2 + 1] * dsilu(zv[2 * i2 + 1] + b2[c0 + 2 * i2 + 1]);
                q[i2] = pack2(a, b);
                if (valid) {
                    const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&q[i2]);
                    w.dz2t[(size_t)(c0 + 2 * i2) * B + col] = hb.x;
                    w.dz2t[(size_t)(c0 + 2 * i2 + 1) * B + col] = hb.y;
                }
            }
            *reinterpret_cast<uint4 *>(sD + tc::kmajor_off(r, c0, kKgs128)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(sD + tc::kmajor_off(r, c0 + 8, kKgs128)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        sync_for_mma();
        // dH1 = dZ2 W2
        if (!run_gemm(tb + 384, sD, kKgs128, sW2T, kKgs128, kH, kH, &mbar, phase, err)) break;
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 16) {
            float dv[16], zv[16];
            tc::tmem_ld16(tD + c0, dv);
            tc::tmem_ld16(tZ1 + c0, zv);
            if (valid) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    w.dz1t[(size_t)(c0 + j) * B + col] =
                        __float2bfloat16_rn(dv[j] * dsilu(zv[j] + b1[c0 + j]));
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    // squared-error sum of this CTA -> *loss
    float v = sq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((r & 31) == 0) red[r >> 5] = v;
    tc::fence_before_sync();
    __syncthreads();
    if (r == 0) atomicAdd(loss, red[0] + red[1] + red[2] + red[3]);
    if (r < 32) tc::tmem_dealloc(tb, 512);
}

// Split-K weight-gradient GEMMs over the batch.  Job j (blockIdx.y):
//   0: dW3 = dZ3^T H2 (+ db3 = row sums of dZ3^T)
//   1: dW2 = dZ2^T H1 (+ db2)
//   2: dW1 = dZ1^T X  (+ db1)
//   3: dw4 = H3^T g   (column 0) and db4 = sum g
// Chunk c (blockIdx.x) covers batch columns [c kChunk, (c + 1) kChunk);
// results go to part[job][c][128][16 or 128] and rsum[job][c][128].
__global__ void __launch_bounds__(128)
k_mlp_wgrad(MlpWork w, int B, int n_chunks, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase_s;
    const int job = blockIdx.y, c = blockIdx.x, r = threadIdx.x;
    const bf16 *A = job == 0 ? w.dz3t : job == 1 ? w.dz2t : job == 2 ? w.dz1t : w.h3t;
    const bf16 *Bm = job == 0 ? w.h2t : job == 1 ? w.h1t : job == 2 ? w.xt : w.g;
    const int N = job <= 1 ? kH : 16;
    const uint32_t kgsb = (uint32_t)(N / 8) * 128;
    unsigned char *sA = smem, *sB = smem + 32768;
    if (r < 32) tc::tmem_alloc(&tbase_s, 128);
    if (r == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tbase_s;
    uint32_t phase = 0;
    float rs = 0.0f;
    bool ok = true;
    const int k0 = c * kWgradChunk;
    for (int kk = 0; kk < kWgradChunk && ok; kk += 128) {
        const int kb = k0 + kk;
        // stage 128 x 128 of A (row r) and N x 128 of B; zero beyond the batch
        for (int q = 0; q < 16; ++q) {
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (kb + q * 8 + 8 <= B)
                val = *reinterpret_cast<const uint4 *>(A + (size_t)r * B + kb + q * 8);
            *reinterpret_cast<uint4 *>(sA + tc::kmajor_off(r, q * 8, kKgs128)) = val;
            const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&val);
#pragma unroll
            for (int t = 0; t < 4; ++t) rs += __low2float(h2[t]) + __high2float(h2[t]);
        }
        if (r < N) {
            for (int q = 0; q < 16; ++q) {
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (kb + q * 8 + 8 <= B)
                    val = *reinterpret_cast<const uint4 *>(Bm + (size_t)r * B + kb + q * 8);
                *reinterpret_cast<uint4 *>(sB + tc::kmajor_off(r, q * 8, kgsb)) = val;
            }
        }
        sync_for_mma();
        if (r == 0) {
            issue_gemm(tb, sA, kKgs128, sB, kgsb, 128, N, kk > 0);
            tc::mma_commit(&mbar);
        }
        ok = tc::mbar_wait(&mbar, phase, kPolls);
        phase ^= 1u;
        tc::fence_after_sync();
        if (!ok && r == 0) atomicExch(err, FC_ETIMEOUT);
        ok = __syncthreads_and(ok);
    }
    if (ok) {
        float *out = w.part + ((size_t)job * n_chunks + c) * (size_t)kH * kH;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(trow(tb, c0), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[(size_t)r * N + c0 + j] = v[j];
        }
        w.rsum[((size_t)job * n_chunks + c) * kH + r] = rs;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (r < 32) tc::tmem_dealloc(tb, 128);
}

// Sum the split-K partials; either write the gradient (grad != nullptr) or
// apply one Adam step to the fp32 parameters and refresh the bf16 copies.
__global__ void k_mlp_adam(MlpWork w, int n_chunks, float *P, float *m1, float *m2, float lr,
                           float bc1, float bc2, float *grad, bf16 *W1b, bf16 *W2b, bf16 *W3b,
                           bf16 *W2Tb, bf16 *W3Tb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float g = 0.0f;
    auto part = [&](int job, int row, int colN, int N) {
        float s = 0.0f;
        for (int c = 0; c < n_chunks; ++c)
            s += w.part[((size_t)job * n_chunks + c) * (size_t)kH * kH + (size_t)row * N + colN];
        return s;
    };
    auto rsum = [&](int job, int row) {
        float s = 0.0f;
        for (int c = 0; c < n_chunks; ++c) s += w.rsum[((size_t)job * n_chunks + c) * kH + row];
        return s;
    };
    if (i < kOffB1) {                       // W1 [128][8], shared by the hi and lo inputs
        g = part(2, i / kMlpIn, i % kMlpIn, 16) + part(2, i / kMlpIn, kMlpIn + i % kMlpIn, 16);
    } else if (i < kOffW2) {
        g = rsum(2, i - kOffB1);
    } else if (i < kOffB2) {
        const int j = i - kOffW2;
        g = part(1, j / kH, j % kH, kH);
    } else if (i < kOffW3) {
        g = rsum(1, i - kOffB2);
    } else if (i < kOffB3) {
        const int j = i - kOffW3;
        g = part(0, j / kH, j % kH, kH);
    } else if (i < kOffW4) {
        g = rsum(0, i - kOffB3);
    } else if (i < kOffB4) {
        g = part(3, i - kOffW4, 0, 16);
    } else {
        // db4 = sum of g over the batch (per-chunk sums from k_mlp_gsum)
        for (int c = 0; c < n_chunks; ++c) g += w.gsum[c];
    }
    if (grad) {
        grad[i] = g;
        return;
    }
    const float a = 0.9f * m1[i] + 0.1f * g;
    const float b = 0.999f * m2[i] + 0.001f * g * g;
    m1[i] = a;
    m2[i] = b;
    const float pnew = P[i] - lr * (a / bc1) / (sqrtf(b / bc2) + 1e-8f);
    P[i] = pnew;
    const bf16 pb = __float2bfloat16_rn(pnew);
    if (i < kOffB1) {
        const int o = i / kMlpIn, in = i % kMlpIn;
        W1b[o * kInP + in] = pb;
        W1b[o * kInP + kMlpIn + in] = pb;
    } else if (i >= kOffW2 && i < kOffB2) {
        const int j = i - kOffW2, o = j / kH, in = j % kH;
        W2b[o * kH + in] = pb;
        W2Tb[in * kH + o] = pb;
    } else if (i >= kOffW3 && i < kOffB3) {
        const int j = i - kOffW3, o = j / kH, in = j % kH;
        W3b[o * kH + in] = pb;
        W3Tb[in * kH + o] = pb;
    }
}

// Column sums of g over each chunk (for db4).
__global__ void k_mlp_gsum(MlpWork w, int B, int n_chunks)
{
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int k = c * kWgradChunk + threadIdx.x; k < min(B, (c + 1) * kWgradChunk); k += blockDim.x)
        s += __bfloat162float(w.g[k]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) w.gsum[c] = red[0];
}

// Per-material maximum of L over n rows (atomicMax on the float bits of
// non-negative values).
__global__ void k_mlp_lmax(const float *L, long long n, int n_mat, unsigned int *mx)
{
    __shared__ unsigned int sm[kMaxMat];
    if (threadIdx.x < kMaxMat) sm[threadIdx.x] = 0u;
    __syncthreads();
    unsigned int loc[kMaxMat] = {0u};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        for (int m = 0; m < n_mat; ++m) loc[m] = max(loc[m], __float_as_uint(fmaxf(L[i * n_mat + m], 0.0f)));
    for (int m = 0; m < n_mat; ++m) atomicMax(&sm[m], loc[m]);
    __syncthreads();
    if (threadIdx.x < n_mat) atomicMax(&mx[threadIdx.x], sm[threadIdx.x]);
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_mlp_eval(const SurrogateParams &p, const float *L, long long n, float *lnT,
                            unsigned int *n_fallback, int *err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kInfSmem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (n + 127) / 128;
    const long long want = (ntiles + kInfGroups - 1) / kInfGroups;
    const int sms = sm_count();
    const int grid = (int)(want < sms ? want : sms);   // one CTA per SM (208 KB smem)
    k_mlp_eval<<<grid, kInfGroupThreads * kInfGroups, kInfSmem, s>>>(p, L, n, lnT, n_fallback, err);
    return cudaGetLastError();
}

__global__ void k_exp(const float *__restrict__ x, float *__restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = expf(x[i]);
}

cudaError_t launch_exp(const float *x, float *y, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    k_exp<<<(int)blocks, 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_energy_sum_lengths(const SurrogateParams &p, const float *L, long long n,
                                      float *lnT, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    k_energy_sum_lengths<<<(int)blocks, 256, 0, s>>>(p, L, n, lnT);
    return cudaGetLastError();
}

cudaError_t launch_mlp_lmax(const float *L, long long n, int n_mat, unsigned int *mx, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    k_mlp_lmax<<<(int)blocks, 256, 0, s>>>(L, n, n_mat, mx);
    return cudaGetLastError();
}

cudaError_t launch_mlp_step(const SurrogateParams &p, const float *L, const float *y, long long n,
                            int B, int sample, unsigned long long seed, int step, const MlpWork &w,
                            float *loss, int *err, float *P, float *m1, float *m2, float lr,
                            float bc1, float bc2, float *grad, bf16 *W1b, bf16 *W2b, bf16 *W3b,
                            bf16 *W2Tb, bf16 *W3Tb, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTrSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    if (e != cudaSuccess) return e;
    const int ntiles = (B + 127) / 128;
    const int sms = sm_count();
    k_mlp_train<<<ntiles < sms ? ntiles : sms, 128, kTrSmem, s>>>(p, L, y, n, B, sample, seed, step,
                                                                  w, loss, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n_chunks = (B + kWgradChunk - 1) / kWgradChunk;
    k_mlp_wgrad<<<dim3(n_chunks, 4), 128, 65536, s>>>(w, B, n_chunks, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_gsum<<<n_chunks, 256, 0, s>>>(w, B, n_chunks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w, n_chunks, P, m1, m2, lr, bc1, bc2, grad,
                                                         W1b, W2b, W3b, W2Tb, W3Tb);
    return cudaGetLastError();
}

}  // namespace fc

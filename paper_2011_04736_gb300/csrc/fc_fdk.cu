// FDK reconstruction (paper Sec. II.G: projections recovered with the flood
// field, reconstructed with FDK [Feldkamp, Davis, Kress 1984], HU
// normalised on the water region).
//
//   q  = ln(I_flood / max(K, 1)) * SAD / sqrt(SAD^2 + u_i^2 + v_i^2)
//   f  = tau * (h * q),  Ram-Lak h[0] = 1/(4 tau^2), h[odd n] = -1/(pi n tau)^2
//   mu = arc / (2 N) * sum_k (SAD / U)^2 * bilinear(f_k; u(x), v(x))
//
// Filter: the weighted rows the backprojector can sample (a conservative
// bound on the rows the voxel slab projects onto), two rows per CTA as the
// real and imaginary parts of one FFT of a power-of-two length in shared
// memory, times the Ram-Lak spectrum, inverse FFT; stored in a zero-padded
// layout of (value, next value - value) pairs so the bilinear taps need no
// bounds tests.  The adjoint's transposed filter sums the taps directly.
// Backprojection: one thread per (x, y) column and chunk of z; per angle
// the column's detector abscissa and weight are computed once and the z
// loop walks the detector column linearly.  Partial sums over 256 angles are
// kept in binary32 and folded into binary64 accumulators.
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {
constexpr int kFiltOut = 16;
constexpr int kFiltThreads = 128;
constexpr int kMaxFiltTaps = 8192;        // odd taps for rows up to 8192 pixels
__constant__ float c_ramp_odd[kMaxFiltTaps];   // -1 / (pi^2 j^2) for j = 1, 3, 5, ...

}  // namespace

// Upload the tau-free odd Ram-Lak taps once per process.
cudaError_t upload_ramp_taps()
{
    static bool done = false;
    static float h[kMaxFiltTaps];
    if (done) return cudaSuccess;
    for (int m = 0; m < kMaxFiltTaps; ++m) {
        const double j = 2.0 * m + 1.0;
        h[m] = (float)(-1.0 / (M_PI * M_PI * j * j));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_ramp_odd, h, sizeof(h));
    if (e == cudaSuccess) done = true;
    return e;
}

// Padded row for the filter: position P = j + off holds sample j (zeros
// elsewhere; off = jm, the largest odd offset, or 1 for a one-pixel row, so
// that P is even for even outputs at every odd offset), stored as pairs
// (P even, P + 1) with one spare pair after every 8 (a warp's 8-byte loads at
// a pair stride of 8 then hit distinct banks).
__host__ __device__ __forceinline__ int pidx(int P) { return 2 * ((P >> 1) + (P >> 4)) + (P & 1); }

// Padded positions the filter reads: up to the last output's window end,
// (n - 1) + 2 ntap + 16 with ntap = jm + 1 <= n (even count).
__host__ __device__ __forceinline__ int filt_span(int n) { return (n + 2 * n + kFiltOut + 2 + 1) & ~1; }

__device__ __forceinline__ int filt_off(int jm) { return jm >= 1 ? jm : 1; }

// Ram-Lak filtered row from the pair-skewed row sp: calls out(i, v) for i in
// [0, n) with v = (x[i] / 4 + sum over odd j of -x[i + j] / (pi j)^2) / tau,
// each output summed in binary32 from x[i] / 4 through the odd offsets in
// ascending order (-jm, ..., jm).  16 outputs per thread as 8 pairs updated
// by packed binary32 FMAs (each element rounded as a scalar fma), a window
// of 8 sample pairs advancing one pair per odd offset, and per warp only the
// offsets at which some output of the warp meets a sample inside the row
// (the others would add h * 0, leaving every output unchanged).
template <class Out>
__device__ __forceinline__ void ramp_row_pairs(const float *sp, int n, float inv_tau, Out out)
{
    const int jm = ((n - 1) & 1) ? n - 1 : n - 2;
    const int ntap = jm >= 1 ? (jm + 1) : 0;
    const int off = filt_off(jm);
    const float2 *sp2 = reinterpret_cast<const float2 *>(sp);
    const int lane = threadIdx.x & 31;
    for (int i0 = threadIdx.x * kFiltOut; i0 < n; i0 += blockDim.x * kFiltOut) {
        float2 acc[kFiltOut / 2];
#pragma unroll
        for (int k = 0; k < kFiltOut / 2; ++k)
            acc[k] = make_float2(0.25f * sp[pidx(i0 + 2 * k + off)], 0.25f * sp[pidx(i0 + 2 * k + 1 + off)]);
        // offsets j = -jm + 2 m, m in [m_lo, m_hi): some output of the warp
        // (outputs [iw0, iw1]) meets a sample j' in [0, n)
        const int iw0 = i0 - kFiltOut * lane;
        const int iw1 = min(iw0 + 32 * kFiltOut - 1, n - 1);
        const int m_lo = max(0, (jm - iw1 + 1) >> 1);
        const int m_hi = min(ntap, ((n - 1 - iw0 + jm) >> 1) + 1);
        if (m_lo < m_hi) {
            // window pair k holds samples at P = i0 + 2 (m + k), + 1 (off = jm
            // here: ntap > 0 needs jm >= 1)
            const int pb = (i0 >> 1) + m_lo;            // pair index of window pair 0
            float2 win[kFiltOut / 2];
#pragma unroll
            for (int k = 0; k < kFiltOut / 2; ++k) win[k] = sp2[(pb + k) + ((pb + k) >> 3)];
            int m = m_lo;
            for (; m + kFiltOut / 2 <= m_hi; m += kFiltOut / 2) {
#pragma unroll
                for (int q = 0; q < kFiltOut / 2; ++q) {
                    const int j = -jm + 2 * (m + q);
                    const int aj = j < 0 ? -j : j;
                    const float h = c_ramp_odd[aj >> 1];
                    const float2 h2 = make_float2(h, h);
#pragma unroll
                    for (int k = 0; k < kFiltOut / 2; ++k)
                        acc[k] = __ffma2_rn(h2, win[(k + q) % (kFiltOut / 2)], acc[k]);
                    const int pn = pb + (m - m_lo) + q + kFiltOut / 2;
                    win[q] = sp2[pn + (pn >> 3)];
                }
            }
#pragma unroll
            for (int q = 0; q < kFiltOut / 2; ++q) {
                if (m + q < m_hi) {
                    const int j = -jm + 2 * (m + q);
                    const int aj = j < 0 ? -j : j;
                    const float h = c_ramp_odd[aj >> 1];
                    const float2 h2 = make_float2(h, h);
#pragma unroll
                    for (int k = 0; k < kFiltOut / 2; ++k)
                        acc[k] = __ffma2_rn(h2, win[(k + q) % (kFiltOut / 2)], acc[k]);
                    const int pn = pb + (m - m_lo) + q + kFiltOut / 2;
                    win[q] = sp2[pn + (pn >> 3)];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kFiltOut / 2; ++k) {
            if (i0 + 2 * k < n) out(i0 + 2 * k, acc[k].x * inv_tau);
            if (i0 + 2 * k + 1 < n) out(i0 + 2 * k + 1, acc[k].y * inv_tau);
        }
    }
}

// DIF butterfly: (u, v) -> (u + v, (u - v) w)
__device__ __forceinline__ void cbfly_dif(float2 &u, float2 &v, float2 w)
{
    const float dx = u.x - v.x, dy = u.y - v.y;
    u = make_float2(u.x + v.x, u.y + v.y);
    v = make_float2(dx * w.x - dy * w.y, dx * w.y + dy * w.x);
}

// DIT butterfly with the conjugate twiddle: (u, v) -> (u + v conj(w), u - v conj(w))
__device__ __forceinline__ void cbfly_dit_conj(float2 &u, float2 &v, float2 w)
{
    const float vx = v.x * w.x + v.y * w.y, vy = v.y * w.x - v.x * w.y;
    v = make_float2(u.x - vx, u.y - vy);
    u = make_float2(u.x + vx, u.y + vy);
}

// Projection and reachable-row index of row `row` of the filters' flattened
// row order: (projection, row) in the plain layout; (k mod Q, row, k div Q)
// in the quarter-interleaved one, so the two rows of a CTA (ra even) are
// quarters b and b + 1 (b even) of the same cell row.
__device__ __forceinline__ void filt_row(const FdkParams &p, long row, int nrows, int *k, int *r)
{
    if (p.filt_quad) {
        const long cell = row >> 2;
        *k = (int)(row & 3) * p.sym_quarter + (int)(cell / nrows);
        *r = (int)(cell % nrows);
    } else {
        *k = (int)(row / nrows);
        *r = (int)(row % nrows);
    }
}

// (value, next value - value) pairs over padded columns 0..n of the CTA's
// rows ra (z[].x) and ra + 1 (z[].y): column c holds output c - 1, columns 0
// and n + 1 are zero.  Quarter-interleaved: both rows go to one 16-byte half
// of each cell, (v_b, v_b+1, d_b, d_b+1).
__device__ __forceinline__ void filt_store(const FdkParams &p, const float2 *z, long ra, long R, int nrows,
                                           int n, float2 *filt)
{
    if (p.filt_quad) {
        const long cell = ra >> 2;
        const int kq = (int)(cell / nrows), r = (int)(cell % nrows);
        float4 *dst = reinterpret_cast<float4 *>(filt) + 2 * (((size_t)kq * p.ph + (r + 1)) * p.pw) +
                      ((ra >> 1) & 1);
        for (int c = threadIdx.x; c <= n; c += blockDim.x) {
            const float2 y0 = c >= 1 ? z[c - 1] : make_float2(0.0f, 0.0f);
            const float2 y1 = c < n ? z[c] : make_float2(0.0f, 0.0f);
            dst[2 * c] = make_float4(y0.x, y0.y, y1.x - y0.x, y1.y - y0.y);
        }
        return;
    }
    for (int half = 0; half < 2; ++half) {
        const long row = ra + half;
        if (row >= R) break;
        const int k = (int)(row / nrows), r = (int)(row % nrows);
        float2 *dst = filt + ((size_t)k * p.ph + (r + 1)) * p.pw;
        for (int c = threadIdx.x; c <= n; c += blockDim.x) {
            const float y0 = c >= 1 ? (half ? z[c - 1].y : z[c - 1].x) : 0.0f;
            const float y1 = c < n ? (half ? z[c].y : z[c].x) : 0.0f;
            dst[c] = make_float2(y0, y1 - y0);
        }
    }
}

__global__ void __launch_bounds__(256)
k_fdk_filter_fft(const __grid_constant__ FdkParams p, const float *__restrict__ counts,
                 float2 *__restrict__ filt)
{
    extern __shared__ float2 z[];
    const DevGeom &g = p.g;
    const int n = g.n_u, L = 1 << p.fft_log2, H = L >> 1;
    const int nrows = p.v_hi - p.v_lo + 1;
    const long R = (long)g.n_angles * nrows;
    const long ra = 2L * blockIdx.x;   // rows ra and ra + 1 of this CTA (the second may be past the end)
    const float *src[2];
    float d2[2];                        // SAD^2 + v^2 of each row
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const long row = ra + t < R ? ra + t : ra;
        int k, r;
        filt_row(p, row, nrows, &k, &r);
        const int iv = p.v_lo + r;
        const float vi = ((float)iv - g.cv) * g.dv * p.mag;
        src[t] = counts + ((size_t)k * g.n_v + iv) * n;
        d2[t] = g.sad * g.sad + vi * vi;
    }
    const bool two = ra + 1 < R;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        float a = 0.0f, b = 0.0f;
        if (j < n) {
            const float ui = ((float)j - g.cu) * g.du * p.mag, u2 = ui * ui;
            a = (p.log_flood - logf(fmaxf(__ldg(src[0] + j), 1.0f))) * (g.sad * rsqrtf(d2[0] + u2));
            if (two) b = (p.log_flood - logf(fmaxf(__ldg(src[1] + j), 1.0f))) * (g.sad * rsqrtf(d2[1] + u2));
        }
        z[j] = make_float2(a, b);
    }
    __syncthreads();
    const float2 *tw = p.fft_tw;
    // forward, decimation in frequency: stages of half-width h = H, H/2, ..., 1,
    // two at a time (h and h/2 on the four elements a, a + h/2, a + h, a + 3h/2)
    int h = H;
    for (; h >= 2; h >>= 2) {
        const int h2 = h >> 1, s1 = H / h;
        for (int q = threadIdx.x; q < (L >> 2); q += blockDim.x) {
            const int pos = q & (h2 - 1);
            const int a = ((q - pos) << 2) + pos;
            float2 x0 = z[a], x1 = z[a + h2], x2 = z[a + h], x3 = z[a + h + h2];
            cbfly_dif(x0, x2, __ldg(tw + pos * s1));
            cbfly_dif(x1, x3, __ldg(tw + (pos + h2) * s1));
            const float2 w2 = __ldg(tw + 2 * pos * s1);
            cbfly_dif(x0, x1, w2);
            cbfly_dif(x2, x3, w2);
            z[a] = x0;
            z[a + h2] = x1;
            z[a + h] = x2;
            z[a + h + h2] = x3;
        }
        __syncthreads();
    }
    if (h == 1) {   // odd log2 L: the last radix-2 stage (twiddle 1)
        for (int q = threadIdx.x; q < H; q += blockDim.x) {
            float2 x0 = z[2 * q], x1 = z[2 * q + 1];
            z[2 * q] = make_float2(x0.x + x1.x, x0.y + x1.y);
            z[2 * q + 1] = make_float2(x0.x - x1.x, x0.y - x1.y);
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < L; r += blockDim.x) {
        const float k = __ldg(p.fft_k + r);
        const float2 v = z[r];
        z[r] = make_float2(v.x * k, v.y * k);
    }
    __syncthreads();
    // inverse, decimation in time with conjugate twiddles: half-widths
    // h = 1, 2, ..., H, two at a time (h and 2h on a, a + h, a + 2h, a + 3h)
    h = 1;
    if (p.fft_log2 & 1) {
        for (int q = threadIdx.x; q < H; q += blockDim.x) {
            float2 x0 = z[2 * q], x1 = z[2 * q + 1];
            z[2 * q] = make_float2(x0.x + x1.x, x0.y + x1.y);
            z[2 * q + 1] = make_float2(x0.x - x1.x, x0.y - x1.y);
        }
        __syncthreads();
        h = 2;
    }
    for (; h < L; h <<= 2) {
        const int s1 = H / h, s2 = s1 >> 1;
        for (int q = threadIdx.x; q < (L >> 2); q += blockDim.x) {
            const int pos = q & (h - 1);
            const int a = ((q - pos) << 2) + pos;
            float2 x0 = z[a], x1 = z[a + h], x2 = z[a + 2 * h], x3 = z[a + 3 * h];
            const float2 w1 = __ldg(tw + pos * s1);
            cbfly_dit_conj(x0, x1, w1);
            cbfly_dit_conj(x2, x3, w1);
            cbfly_dit_conj(x0, x2, __ldg(tw + pos * s2));
            cbfly_dit_conj(x1, x3, __ldg(tw + (pos + h) * s2));
            z[a] = x0;
            z[a + h] = x1;
            z[a + 2 * h] = x2;
            z[a + 3 * h] = x3;
        }
        __syncthreads();
    }
    filt_store(p, z, ra, R, nrows, n, filt);
}

// One pass of R radix-2 stages on groups of 2^R points at stride q (q =
// 2^lq) held in registers, 8 points per thread: forward (decimation in
// frequency, stages of half-width q 2^(R-1) down to q) or inverse
// (decimation in time with conjugate twiddles, half-widths q up to
// q 2^(R-1)).  Group g holds the points grp (q 2^R) + pos + m q, pos = g mod q.
template <int R, bool INV>
__device__ __forceinline__ void fft_pass(float2 *z, int t, int q, int lq, const float2 *__restrict__ tw, int H)
{
    constexpr int NG = 8 >> R, SZ = 1 << R;
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
        const int g = t * NG + gi, pos = g & (q - 1), base = ((g >> lq) << (lq + R)) + pos;
        float2 x[SZ];
#pragma unroll
        for (int m = 0; m < SZ; ++m) x[m] = z[base + m * q];
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
            const int j = INV ? jj : R - 1 - jj;
            const int span = 1 << j, st = H >> (lq + j);     // st = H / (half-width)
#pragma unroll
            for (int m = 0; m < SZ; ++m) {
                if (m & span) continue;
                const float2 w = __ldg(tw + (pos + (m & (2 * span - 1)) * q) * st);
                if (INV)
                    cbfly_dit_conj(x[m], x[m + span], w);
                else
                    cbfly_dif(x[m], x[m + span], w);
            }
        }
#pragma unroll
        for (int m = 0; m < SZ; ++m) z[base + m * q] = x[m];
    }
}

// The last three forward stages (half-widths 4, 2, 1), the product with the
// spectrum (bit-reversed order) and the first three inverse stages on the 8
// consecutive points of one thread, in registers.
__device__ __forceinline__ void fft_mid(float2 *z, int t, const float2 *__restrict__ tw,
                                        const float *__restrict__ kbr, int H)
{
    const int base = t * 8;
    float2 x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = z[base + m];
#pragma unroll
    for (int j = 2; j >= 0; --j) {
        const int span = 1 << j;
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (!(m & span)) cbfly_dif(x[m], x[m + span], __ldg(tw + (m & (2 * span - 1)) * (H >> j)));
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const float k = __ldg(kbr + base + m);
        x[m] = make_float2(x[m].x * k, x[m].y * k);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int span = 1 << j;
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (!(m & span)) cbfly_dit_conj(x[m], x[m + span], __ldg(tw + (m & (2 * span - 1)) * (H >> j)));
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) z[base + m] = x[m];
}

// The FFT filter for 64 <= L <= 2048 (rows of 17 to 1024 samples), L / 8
// threads each holding 8 points per pass: passes of up to three stages in
// registers, the middle one fused with the spectrum product, so a row pair
// costs about 2 (log2 L - 3) / 3 + 3 barriers instead of one per two stages.
// Same operator, weighting, twiddles and output layout as k_fdk_filter_fft.
__global__ void __launch_bounds__(256)
k_fdk_filter_fft8(const __grid_constant__ FdkParams p, const float *__restrict__ counts,
                  float2 *__restrict__ filt)
{
    extern __shared__ float2 z[];
    const DevGeom &g = p.g;
    const int n = g.n_u, lg = p.fft_log2, L = 1 << lg, H = L >> 1;
    const int nrows = p.v_hi - p.v_lo + 1;
    const long R = (long)g.n_angles * nrows;
    const long ra = 2L * blockIdx.x;
    const float *src[2];
    float d2[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const long row = ra + t < R ? ra + t : ra;
        int k, r;
        filt_row(p, row, nrows, &k, &r);
        const int iv = p.v_lo + r;
        const float vi = ((float)iv - g.cv) * g.dv * p.mag;
        src[t] = counts + ((size_t)k * g.n_v + iv) * n;
        d2[t] = g.sad * g.sad + vi * vi;
    }
    const bool two = ra + 1 < R;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        float a = 0.0f, b = 0.0f;
        if (j < n) {
            const float ui = ((float)j - g.cu) * g.du * p.mag, u2 = ui * ui;
            a = (p.log_flood - logf(fmaxf(__ldg(src[0] + j), 1.0f))) * (g.sad * rsqrtf(d2[0] + u2));
            if (two) b = (p.log_flood - logf(fmaxf(__ldg(src[1] + j), 1.0f))) * (g.sad * rsqrtf(d2[1] + u2));
        }
        z[j] = make_float2(a, b);
    }
    __syncthreads();
    const float2 *tw = p.fft_tw;
    const int t = threadIdx.x;
    // forward stages of half-width H down to 8, three per pass from the top
    int F = lg - 3, lq = lg - 1;                 // lq: log2 of the top stage's half-width
    while (F > 0) {
        const int Rs = F < 3 ? F : 3;
        lq -= Rs - 1;
        const int q = 1 << lq;
        if (Rs == 3) fft_pass<3, false>(z, t, q, lq, tw, H);
        else if (Rs == 2) fft_pass<2, false>(z, t, q, lq, tw, H);
        else fft_pass<1, false>(z, t, q, lq, tw, H);
        __syncthreads();
        lq -= 1;
        F -= Rs;
    }
    fft_mid(z, t, tw, p.fft_k, H);
    __syncthreads();
    // inverse stages of half-width 8 up to H, three per pass from the bottom
    F = lg - 3;
    lq = 3;
    while (F > 0) {
        const int Rs = F < 3 ? F : 3;
        const int q = 1 << lq;
        if (Rs == 3) fft_pass<3, true>(z, t, q, lq, tw, H);
        else if (Rs == 2) fft_pass<2, true>(z, t, q, lq, tw, H);
        else fft_pass<1, true>(z, t, q, lq, tw, H);
        __syncthreads();
        lq += Rs;
        F -= Rs;
    }
    filt_store(p, z, ra, R, nrows, n, filt);
}

int fdk_fft_log2(int n_u)
{
    int l = 1;
    while ((1 << l) < 2 * n_u - 1) ++l;
    return l;
}

void fdk_fft_tables(int n_u, double tau, std::vector<float2> *tw, std::vector<float> *kbr)
{
    const int lg = fdk_fft_log2(n_u), L = 1 << lg;
    std::vector<double> cs(L);
    for (int t = 0; t < L; ++t) cs[t] = cos(2.0 * M_PI * t / L);
    tw->resize(L / 2);
    for (int t = 0; t < L / 2; ++t) (*tw)[t] = make_float2((float)cs[t], (float)-sin(2.0 * M_PI * t / L));
    const int jm = ((n_u - 1) & 1) ? n_u - 1 : n_u - 2;
    kbr->resize(L);
    for (int r = 0; r < L; ++r) {
        unsigned m = 0;   // frequency at bit-reversed position r
        for (int b = 0; b < lg; ++b)
            if (r >> b & 1) m |= 1u << (lg - 1 - b);
        double K = 0.25;
        for (int j = 1; j <= jm; j += 2) K -= 2.0 * cs[(size_t)j * m % L] / (M_PI * M_PI * (double)j * j);
        (*kbr)[r] = (float)(K / ((double)L * tau));
    }
}

cudaError_t launch_fdk_filter(const FdkParams &p, const float *counts, float2 *filt, cudaStream_t s)
{
    const int nrows = p.v_hi - p.v_lo + 1;
    if (nrows <= 0 || p.g.n_angles <= 0) return cudaSuccess;
    if (p.g.n_u > kMaxFiltTaps) return cudaErrorInvalidValue;
    if (!p.fft_k || !p.fft_tw) return cudaErrorInvalidValue;
    const int L = 1 << p.fft_log2;
    const size_t smem = (size_t)L * sizeof(float2);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_fdk_filter_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long rows = (long)p.g.n_angles * nrows;
    if (p.fft_log2 >= 6 && p.fft_log2 <= 11) {
        k_fdk_filter_fft8<<<(unsigned)((rows + 1) / 2), L / 8, smem, s>>>(p, counts, filt);
        return cudaGetLastError();
    }
    const int threads = L / 2 < 256 ? L / 2 : 256;
    k_fdk_filter_fft<<<(unsigned)((rows + 1) / 2), threads, smem, s>>>(p, counts, filt);
    return cudaGetLastError();
}

// Ram-Lak transpose (the kernel is symmetric, so it is the same row filter)
// and the chain rule down to dJ/dI:  q = ln(I_flood / max(K, 1)) cosw,
// K = I + sqrt(I) z.  One CTA per reachable detector row of a projection
// (gf in the padded layout of the filtered rows); gI elsewhere is left as is.
__global__ void __launch_bounds__(kFiltThreads)
k_filter_adjoint(const __grid_constant__ FdkParams p, const float *__restrict__ gf,
                 const float *__restrict__ I, const float *__restrict__ K,
                 const float *__restrict__ z, float *__restrict__ gI)
{
    extern __shared__ float sx[];
    const DevGeom &g = p.g;
    const int n = g.n_u;
    const int nrows = p.v_hi - p.v_lo + 1;
    const int k = blockIdx.x / nrows;
    const int r = (int)(blockIdx.x % nrows);
    const int iv = p.v_lo + r;
    const float *src = gf + ((size_t)k * p.ph + (r + 1)) * p.pw + 1;
    const int off = filt_off(((n - 1) & 1) ? n - 1 : n - 2);
    const int span = filt_span(n);
    for (int i = threadIdx.x; i < span; i += blockDim.x) {
        const int j = i - off;
        sx[pidx(i)] = j >= 0 && j < n ? src[j] : 0.0f;
    }
    __syncthreads();
    const float vi = ((float)iv - g.cv) * g.dv * p.mag;
    const size_t row = ((size_t)k * g.n_v + iv) * n;
    ramp_row_pairs(sx, n, 1.0f / p.tau, [&](int iu, float gq) {
        const float ui = ((float)iu - g.cu) * g.du * p.mag;
        const float cosw = g.sad * rsqrtf(g.sad * g.sad + ui * ui + vi * vi);
        const size_t idx = row + iu;
        const float Kv = K[idx];
        const float gK = Kv > 1.0f ? -gq * cosw / Kv : 0.0f;
        float dKdI = 1.0f;
        if (z) {
            const float Iv = I[idx];
            dKdI = Iv > 0.0f ? 1.0f + 0.5f * z[idx] * rsqrtf(Iv) : 1.0f;
        }
        gI[idx] = gK * dKdI;
    });
}

cudaError_t launch_filter_adjoint(const FdkParams &p, const float *gf, const float *I, const float *K,
                                  const float *z, float *gI, cudaStream_t s)
{
    const int nrows = p.v_hi - p.v_lo + 1;
    if (nrows <= 0 || p.g.n_angles <= 0) return cudaSuccess;
    if (p.g.n_u > kMaxFiltTaps) return cudaErrorInvalidValue;
    cudaError_t e = upload_ramp_taps();
    if (e != cudaSuccess) return e;
    const int span = filt_span(p.g.n_u);
    const size_t smem = (size_t)(2 * ((span >> 1) + (span >> 4)) + 4) * sizeof(float);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_filter_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
    }
    const size_t blocks = (size_t)p.g.n_angles * nrows;
    k_filter_adjoint<<<(unsigned)blocks, kFiltThreads, smem, s>>>(p, gf, I, K, z, gI);
    return cudaGetLastError();
}

// Conservative range of detector rows the backprojector can touch.
void fdk_row_range(const DevGeom &g, int *v_lo, int *v_hi)
{
    const double hx = 0.5 * g.nx * (double)g.dx, hy = 0.5 * g.ny * (double)g.dy;
    const double rmax = sqrt(hx * hx + hy * hy);
    const double zmax = 0.5 * (g.nz - 1) * (double)g.dz;
    const double umin = (double)g.sad - rmax;
    double vmax;
    if (umin <= 0.0) {
        *v_lo = 0;
        *v_hi = g.n_v - 1;
        return;
    }
    vmax = zmax * (double)g.sdd / umin / (double)g.dv;
    int lo = (int)floor((double)g.cv - vmax) - 2;
    int hi = (int)ceil((double)g.cv + vmax) + 2;
    *v_lo = lo < 0 ? 0 : lo;
    *v_hi = hi > g.n_v - 1 ? g.n_v - 1 : hi;
}

namespace {
constexpr int kFold = 256;       // angles per binary32 partial sum
// floor(v) of 0 <= v < 2^22 as the low bits of v + 2^23 rounded toward -inf
constexpr float kTwo23 = 8388608.0f;
constexpr int kSlabMaxNz = 16;   // slices the thin-slab kernel keeps per thread
// largest projected z pitch (detector rows) the thin-slab kernel takes: the
// row index may then advance by at most one per slice, rounding included
constexpr double kSlabMaxStep = 0.98;
constexpr int kSymMaxRun = 5;      // slices per thread of the quarter-turn kernel (more spill)

// Chunked kernel: z values per thread as many as possible (the per-angle
// column set-up is shared by them) while keeping about 48 resident warps
// per SM; the chunks are balanced.
void chunked_launch_shape(const FdkParams &p, int *zc_out, dim3 *grid)
{
    const long cols = (long)p.g.nx * p.g.ny;
    const long want = (long)sm_count() * 1536;
    int zc = 8;
    while (zc > 1 && cols * ((p.g.nz + zc - 1) / zc) < want) --zc;
    const int nchunk = (p.g.nz + zc - 1) / zc;
    zc = (p.g.nz + nchunk - 1) / nchunk;
    *zc_out = zc;
    *grid = dim3((p.g.nx + 31) / 32, (p.g.ny + 7) / 8, (p.g.nz + zc - 1) / zc);
}
}  // namespace

namespace {
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
// a - b, exactly as a binary32 subtraction rounds it (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
}  // namespace

// kZc z values per thread, kZc even: the same arithmetic as the scalar body
// below, issued as packed binary32 pairs over the z values (z, z + kZc / 2)
// (each element rounded as the scalar instruction rounds it, so the volume
// is identical), binary64 sums in shared memory.
template <int kZc>
__device__ __forceinline__ void backproject_body_pairs(const FdkParams &p, const float2 *__restrict__ f,
                                                       double *__restrict__ vol)
{
    constexpr int NA = kZc / 2;
    __shared__ double accd[kZc][256];
    const DevGeom &g = p.g;
    const int t = threadIdx.y * 32 + threadIdx.x;
    // a warp covers 8 x 4 voxels of the CTA's 32 x 8 (its taps then span
    // fewer detector columns and, through the perspective, fewer rows)
    const int ix = blockIdx.x * 32 + (threadIdx.y % 4) * 8 + threadIdx.x % 8;
    const int iy = blockIdx.y * 8 + (threadIdx.y / 4) * 4 + threadIdx.x / 8;
    const int iz0 = blockIdx.z * kZc;
#pragma unroll
    for (int z = 0; z < kZc; ++z) accd[z][t] = 0.0;
    if (ix >= g.nx || iy >= g.ny) return;   // no block-wide barrier follows
    const float x = ((float)ix - 0.5f * (float)(g.nx - 1)) * g.dx;
    const float y = ((float)iy - 0.5f * (float)(g.ny - 1)) * g.dy;
    const float z0 = ((float)iz0 - 0.5f * (float)(g.nz - 1)) * g.dz;
    const int nzc = min(kZc, g.nz - iz0);
    const unsigned plane = (unsigned)p.ph * (unsigned)p.pw;
    const float cu1 = g.cu + 1.0f, cv1 = g.cv - (float)p.v_lo + 1.0f;
    const float umax = (float)(p.pw - 2), vmaxp = (float)(p.ph - 2);
    const float sdd_du = g.sdd / g.du, sdd_dv = g.sdd / g.dv;
    const int two23 = __float_as_int(kTwo23);
    for (int kb = 0; kb < g.n_angles; kb += kFold) {
        const int ke = min(g.n_angles, kb + kFold);
        float2 acc[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) acc[i] = make_float2(0.0f, 0.0f);
#pragma unroll 2
        for (int k = kb; k < ke; ++k) {
            const float2 cs = p.trig[k];
            const float U = g.sad - (x * cs.x + y * cs.y);
            const float ru = y * cs.x - x * cs.y;
            float iU;                                   // hardware reciprocal + one Newton step
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iU) : "f"(U));
            iU = fmaf(iU, fmaf(-U, iU, 1.0f), iU);
            const float fu = fminf(fmaxf(fmaf(ru * iU, sdd_du, cu1), 0.0f), umax);
            const float2 w2 = f2((g.sad * iU) * (g.sad * iU));
            const float2 fv0 = f2(fmaf(z0 * iU, sdd_dv, cv1));
            const float2 dfv = f2(g.dz * iU * sdd_dv);
            const float tu = __fadd_rd(fu, kTwo23);     // 2^23 + floor(fu)
            const float au = fu - (tu - kTwo23);
            const unsigned cofs = (unsigned)k * (unsigned)plane + (unsigned)(__float_as_int(tu) - two23);
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                // z values past a ragged last chunk are computed on clamped,
                // in-buffer coordinates and never stored
                float2 fv = __ffma2_rn(make_float2((float)i, (float)(i + NA)), dfv, fv0);
                fv.x = fminf(fmaxf(fv.x, 0.0f), vmaxp);
                fv.y = fminf(fmaxf(fv.y, 0.0f), vmaxp);
                const float2 tv = __fadd2_rd(fv, f2(kTwo23));
                const float2 av = sub2(fv, __fadd2_rn(tv, f2(-kTwo23)));
                const unsigned oa = (unsigned)(__float_as_int(tv.x) - two23) * (unsigned)p.pw + cofs;
                const unsigned ob = (unsigned)(__float_as_int(tv.y) - two23) * (unsigned)p.pw + cofs;
                const float2 a0 = __ldg(f + oa), a1 = __ldg(f + (oa + (unsigned)p.pw));
                const float2 b0 = __ldg(f + ob), b1 = __ldg(f + (ob + (unsigned)p.pw));
                const float2 top = make_float2(fmaf(au, a0.y, a0.x), fmaf(au, b0.y, b0.x));
                const float2 bot = make_float2(fmaf(au, a1.y, a1.x), fmaf(au, b1.y, b1.x));
                acc[i] = __ffma2_rn(w2, __ffma2_rn(av, sub2(bot, top), top), acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            accd[i][t] += (double)acc[i].x;
            accd[i + NA][t] += (double)acc[i].y;
        }
    }
#pragma unroll
    for (int z = 0; z < kZc; ++z)
        if (z < nzc) vol[((size_t)(iz0 + z) * g.ny + iy) * g.nx + ix] = accd[z][t] * p.scale;
}

// kZc z values per thread (the launcher balances the z chunks).
template <int kZc>
__device__ __forceinline__ void backproject_body(const FdkParams &p, const float2 *__restrict__ f,
                                                 double *__restrict__ vol)
{
    if constexpr (kZc % 2 == 0) {
        backproject_body_pairs<kZc>(p, f, vol);
        return;
    }
    const DevGeom &g = p.g;
    // a warp covers 8 x 4 voxels of the CTA's 32 x 8 (its taps then span
    // fewer detector columns and, through the perspective, fewer rows)
    const int ix = blockIdx.x * 32 + (threadIdx.y % 4) * 8 + threadIdx.x % 8;
    const int iy = blockIdx.y * 8 + (threadIdx.y / 4) * 4 + threadIdx.x / 8;
    const int iz0 = blockIdx.z * kZc;
    if (ix >= g.nx || iy >= g.ny) return;
    const float x = ((float)ix - 0.5f * (float)(g.nx - 1)) * g.dx;
    const float y = ((float)iy - 0.5f * (float)(g.ny - 1)) * g.dy;
    const float z0 = ((float)iz0 - 0.5f * (float)(g.nz - 1)) * g.dz;
    const int nzc = min(kZc, g.nz - iz0);
    const unsigned plane = (unsigned)p.ph * (unsigned)p.pw;
    // padded coordinates: column c + 1 holds detector column c, row r + 1
    // holds detector row v_lo + r; clamping to [0, pw - 2] x [0, ph - 2]
    // keeps both taps inside the buffer and only ever lands on zero padding
    // where the true sample lies outside the detector (columns) or is never
    // requested (rows).
    const float cu1 = g.cu + 1.0f, cv1 = g.cv - (float)p.v_lo + 1.0f;
    const float umax = (float)(p.pw - 2), vmaxp = (float)(p.ph - 2);
    const float sdd_du = g.sdd / g.du, sdd_dv = g.sdd / g.dv;
    const int two23 = __float_as_int(kTwo23);
    double accd[kZc];
#pragma unroll
    for (int z = 0; z < kZc; ++z) accd[z] = 0.0;
    for (int kb = 0; kb < g.n_angles; kb += kFold) {
        const int ke = min(g.n_angles, kb + kFold);
        float accf[kZc];
#pragma unroll
        for (int z = 0; z < kZc; ++z) accf[z] = 0.0f;
#pragma unroll 2
        for (int k = kb; k < ke; ++k) {
            const float2 cs = p.trig[k];
            const float U = g.sad - (x * cs.x + y * cs.y);
            const float ru = y * cs.x - x * cs.y;
            float iU;                                   // hardware reciprocal + one Newton step
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iU) : "f"(U));
            iU = fmaf(iU, fmaf(-U, iU, 1.0f), iU);
            const float fu = fminf(fmaxf(fmaf(ru * iU, sdd_du, cu1), 0.0f), umax);
            const float w = (g.sad * iU) * (g.sad * iU);
            const float fv0 = fmaf(z0 * iU, sdd_dv, cv1);
            const float dfv = g.dz * iU * sdd_dv;
            const float tu = __fadd_rd(fu, kTwo23);     // 2^23 + floor(fu)
            const float au = fu - (tu - kTwo23);
            // element offset of the column in projection k (the buffer holds
            // fewer than 2^31 elements: 32-bit offsets from the kernel's pointer)
            const unsigned cofs = (unsigned)k * (unsigned)plane + (unsigned)(__float_as_int(tu) - two23);
#pragma unroll
            for (int z = 0; z < kZc; ++z) {
                if (z < nzc) {
                    const float fv = fminf(fmaxf(fmaf((float)z, dfv, fv0), 0.0f), vmaxp);
                    const float tv = __fadd_rd(fv, kTwo23);
                    const float av = fv - (tv - kTwo23);
                    const unsigned o = (unsigned)(__float_as_int(tv) - two23) * (unsigned)p.pw + cofs;
                    const float2 t0 = __ldg(f + o), t1 = __ldg(f + (o + (unsigned)p.pw));
                    const float top = fmaf(au, t0.y, t0.x);
                    const float bot = fmaf(au, t1.y, t1.x);
                    accf[z] = fmaf(w, fmaf(av, bot - top, top), accf[z]);
                }
            }
        }
#pragma unroll
        for (int z = 0; z < kZc; ++z) accd[z] += (double)accf[z];
    }
#pragma unroll
    for (int z = 0; z < kZc; ++z)
        if (z < nzc) vol[((size_t)(iz0 + z) * g.ny + iy) * g.nx + ix] = accd[z] * p.scale;
}

// The body as compiled with the default register budget (40 registers, 6
// CTAs per SM, no spill) and capped for 8 CTAs per SM (32 registers, a few
// bytes of the binary64 sums spilled).
template <int kZc>
__global__ void __launch_bounds__(256) k_backproject(const __grid_constant__ FdkParams p,
                                                     const float2 *__restrict__ f,
                                                     double *__restrict__ vol)
{
    backproject_body<kZc>(p, f, vol);
}

template <int kZc>
// (6 resident CTAs for the packed bodies of 6 or 8 z values: at 8 their
// binary32 pairs spill)
__global__ void __launch_bounds__(256, (kZc % 2 == 0 && kZc >= 6) ? 6 : 8)
k_backproject_dense(const __grid_constant__ FdkParams p,
                                                              const float2 *__restrict__ f,
                                                              double *__restrict__ vol)
{
    backproject_body<kZc>(p, f, vol);
}

// Thin slabs: the z pitch projects to less than one detector row at every
// voxel (dz SDD / U < dv), which holds for the paper-scale 10-slice volumes
// with a fine voxel pitch.  One thread per (x, y) column then walks all NZ
// slices of its column for each angle.  Slice z samples rows j_z and j_z + 1
// with j_z - j_{z-1} in {0, 1}, so the u-interpolated value of each row is
// formed once: slice z loads only row j_z + 1 (two taps) and takes row j_z
// from the slice before (the same row, or the one it loaded).  Per update
// that is two tap loads instead of four and one u interpolation instead of
// two.  The slices run as two interleaved halves (z and z + NA), so the
// binary32 arithmetic of the v coordinate, the v interpolation and the sums
// issues as packed pairs (Blackwell f32x2 FMA / add instructions: two lanes'
// worth of binary32 work per instruction, each element rounded exactly as the
// scalar instruction would); the u interpolation of the loaded taps stays
// scalar (fewer registers); floors come from adding 2^23 with rounding toward
// -inf (exact for 0 <= v < 2^22); tap addresses are 32-bit element offsets
// from the kernel's pointer, one multiply-add each.
// Binary32 partial sums over kFold angles are folded into binary64 sums
// kept in shared memory.  CLAMP: clamp the detector coordinates into the
// stored rows and columns (needed only when a voxel can project outside them:
// rows cut at a detector edge, or a detector narrower than the volume's
// shadow).  The reciprocal of U is the hardware approximation refined by one
// Newton-Raphson step, r' = r (2 - U r), within an ulp or so of 1 / U.

template <int NZ, bool CLAMP>
__global__ void __launch_bounds__(256)
k_backproject_slab(const __grid_constant__ FdkParams p, const float2 *__restrict__ f,
                   double *__restrict__ vol)
{
    constexpr int NA = (NZ + 1) / 2;     // slices per half: z = i and z = i + NA
    __shared__ double accd[NZ][256];
    const DevGeom &g = p.g;
    const int t = threadIdx.y * 32 + threadIdx.x;
    // a warp covers 8 x 4 voxel columns of the CTA's 32 x 8
    const int ix = blockIdx.x * 32 + (threadIdx.y % 4) * 8 + threadIdx.x % 8;
    const int iy = blockIdx.y * 8 + (threadIdx.y / 4) * 4 + threadIdx.x / 8;
#pragma unroll
    for (int z = 0; z < NZ; ++z) accd[z][t] = 0.0;
    if (ix >= g.nx || iy >= g.ny) return;   // no block-wide barrier follows
    const float x = ((float)ix - 0.5f * (float)(g.nx - 1)) * g.dx;
    const float y = ((float)iy - 0.5f * (float)(g.ny - 1)) * g.dy;
    const float z0 = -0.5f * (float)(g.nz - 1) * g.dz;
    const unsigned plane = (unsigned)p.ph * (unsigned)p.pw;
    const float cu1 = g.cu + 1.0f, cv1 = g.cv - (float)p.v_lo + 1.0f;
    const float umax = (float)(p.pw - 2), vmaxp = (float)(p.ph - 2);
    const float sdd_du = g.sdd / g.du, sdd_dv = g.sdd / g.dv, dz_dv = g.dz * (g.sdd / g.dv);
    const float2 zz_step = make_float2(0.0f, (float)NA);   // (z_a, z_b) at i = 0
    const int two23 = __float_as_int(kTwo23);
    for (int kb = 0; kb < g.n_angles; kb += kFold) {
        const int ke = min(g.n_angles, kb + kFold);
        float2 acc[NA];
#pragma unroll
        for (int i = 0; i < NA; ++i) acc[i] = make_float2(0.0f, 0.0f);
#pragma unroll 2
        for (int k = kb; k < ke; ++k) {
            const float2 cs = p.trig[k];
            const float U = g.sad - (x * cs.x + y * cs.y);
            const float ru = y * cs.x - x * cs.y;
            float iU;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iU) : "f"(U));
            iU = fmaf(iU, fmaf(-U, iU, 1.0f), iU);
            float fu = fmaf(ru * iU, sdd_du, cu1);
            if (CLAMP) fu = fminf(fmaxf(fu, 0.0f), umax);
            const float tu = __fadd_rd(fu, kTwo23);          // 2^23 + floor(fu)
            const float au = fu - (tu - kTwo23);
            const float2 w2 = f2((g.sad * iU) * (g.sad * iU));
            const float2 fv0 = f2(fmaf(z0 * iU, sdd_dv, cv1));
            const float2 dfv = f2(dz_dv * iU);
            const float2 au2 = f2(au);
            // element offset of row r + 1 of the column: (2^23 + r) pw + cofs,
            // in 32-bit modular arithmetic (the true offset is below 2^31), so
            // each tap address is one multiply-add off the kernel's pointer
            const unsigned cofs = (unsigned)k * (unsigned)plane + (unsigned)(__float_as_int(tu) - two23) +
                                  (unsigned)(1 - two23) * (unsigned)p.pw;
            float2 lo, hi;
            int2 jp;
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                const float2 zz = make_float2((float)i + zz_step.x, (float)i + zz_step.y);
                float2 fv = __ffma2_rn(zz, dfv, fv0);
                if (CLAMP) {
                    fv.x = fminf(fmaxf(fv.x, 0.0f), vmaxp);
                    fv.y = fminf(fmaxf(fv.y, 0.0f), vmaxp);
                }
                const float2 tv = __fadd2_rd(fv, f2(kTwo23));    // 2^23 + floor(fv)
                const float2 av = sub2(fv, __fadd2_rn(tv, f2(-kTwo23)));
                const int2 j = make_int2(__float_as_int(tv.x), __float_as_int(tv.y));
                const float2 *ra = f + ((unsigned)j.x * (unsigned)p.pw + cofs);
                const float2 *rb = f + ((unsigned)j.y * (unsigned)p.pw + cofs);
                const float2 qa = __ldg(ra), qb = __ldg(rb);
                const float2 nh = make_float2(fmaf(au2.x, qa.y, qa.x), fmaf(au2.x, qb.y, qb.x));
                if (i == 0) {
                    const float2 pa = __ldg(ra - p.pw), pb = __ldg(rb - p.pw);
                    lo = make_float2(fmaf(au2.x, pa.y, pa.x), fmaf(au2.x, pb.y, pb.x));
                } else {
                    lo.x = j.x == jp.x ? lo.x : hi.x;
                    lo.y = j.y == jp.y ? lo.y : hi.y;
                }
                hi = nh;
                jp = j;
                acc[i] = __ffma2_rn(w2, __ffma2_rn(av, sub2(hi, lo), lo), acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            accd[i][t] += (double)acc[i].x;
            if (i + NA < NZ) accd[i + NA][t] += (double)acc[i].y;
        }
    }
#pragma unroll
    for (int z = 0; z < NZ; ++z) vol[((size_t)z * g.ny + iy) * g.nx + ix] = accd[z][t] * p.scale;
}

// Thin slabs of a full-circle scan of a square grid centred on the axis:
// turning a voxel column by a quarter turn about the axis while the gantry
// turns by a quarter turn leaves its geometry unchanged (U = SAD - (x cos +
// y sin) and the detector abscissa y cos - x sin are invariant under
// (x, y, theta) -> (-y, x, theta + pi/2)).  With N projections equally
// spaced over 2 pi and N a multiple of 4, projection k + N/4 is projection k
// turned by a quarter turn, so the column set-up of base column c at
// projection k (U, 1 / U, the detector abscissa and its fraction, the
// weight) and every slice's row index and row fraction also hold for the
// turned columns R^t c at projections k + t N / 4 (mod N), t = 1, 2, 3, with
// R (ix, iy) = (n-1-iy, ix).  One thread takes a base column of the quadrant
// ix, iy < n / 2 (the four quadrants are the orbits of an even n); per
// projection it computes that geometry once and then loads, interpolates
// and sums the taps of the four columns, the sums as packed binary32 pairs
// (each element rounded as the scalar instruction rounds it).  QUAD (thin
// slabs whose voxel pitch projects to at most a detector column): the
// filtered rows are quarter-interleaved, so the four columns' taps at one
// detector position are one 32-byte cell, two 16-byte loads from one
// address whose (value, difference) halves feed the packed interpolations
// directly (otherwise four 8-byte loads from four projections, each
// interpolated on its own).  THIN (the
// z pitch projects to less than one detector row): a slice whose row index
// equals the previous slice's reuses both interpolated rows and loads
// nothing, one whose row advanced loads only the new row j + 1; otherwise
// every slice loads rows j and j + 1.  FULL: every run holds NS slices (R
// divides nz), so the slice loop carries no run-length test (paper-scale
// thin slab 3.98 -> 3.64 ms).  A thread takes one of R balanced runs of consecutive
// slices (at most NS) and one half of the projections (grid z = 2 R; the
// halves on separate CTAs make more, shorter CTAs, so the last round of
// resident CTAs is less empty).  The projections are walked in segments of
// at most kFold in which no turned projection index wraps past N, so each
// column's projection is a fixed offset from k there; binary32 sums over a
// segment are folded into binary64 sums in shared memory.  Every voxel then
// receives exactly two atomic binary64 adds onto a zeroed volume, whose sum
// x + y does not depend on their order.  Floors, reciprocal and clamps as
// in k_backproject_slab.
template <int NS, bool CLAMP, bool THIN, bool FULL, bool QUAD>
__global__ void __launch_bounds__(256, 4)
k_backproject_sym(const __grid_constant__ FdkParams p, const float2 *__restrict__ f,
                  double *__restrict__ vol)
{
    __shared__ double accd[4 * NS][256];
    const DevGeom &g = p.g;
    const int n = g.nx, NZ = g.nz;
    const int t = threadIdx.y * 32 + threadIdx.x;
    const int ix = blockIdx.x * 32 + (threadIdx.y % 4) * 8 + threadIdx.x % 8;
    const int iy = blockIdx.y * 8 + (threadIdx.y / 4) * 4 + threadIdx.x / 8;
#pragma unroll
    for (int i = 0; i < 4 * NS; ++i) accd[i][t] = 0.0;
    if (ix >= n / 2 || iy >= n / 2) return;   // no block-wide barrier follows
    // grid z = (half of the projections) x (run of slices); run r of R holds
    // slices [r NZ / R, (r + 1) NZ / R)
    const int R = (int)gridDim.z / 2;
    const int run = (int)blockIdx.z % R, half = (int)blockIdx.z / R;
    const int zb = run * NZ / R;
    const int ns = (run + 1) * NZ / R - zb;
    const float x = ((float)ix - 0.5f * (float)(n - 1)) * g.dx;
    const float y = ((float)iy - 0.5f * (float)(n - 1)) * g.dy;
    const float zc = (-0.5f * (float)(NZ - 1) + (float)zb) * g.dz;   // the run's first slice
    const unsigned plane = (unsigned)p.ph * (unsigned)p.pw;
    const float cu1 = g.cu + 1.0f, cv1 = g.cv - (float)p.v_lo + 1.0f;
    const float umax = (float)(p.pw - 2), vmaxp = (float)(p.ph - 2);
    const float sdd_du = g.sdd / g.du, sdd_dv = g.sdd / g.dv, dz_dv = g.dz * (g.sdd / g.dv);
    const int two23 = __float_as_int(kTwo23);
    const int N = g.n_angles, Q = N / 4;     // projections per quarter turn
    const int kend = (half + 1) * (N / 2);
    const float4 *fq = reinterpret_cast<const float4 *>(f);   // two per cell
    // segments of at most kFold projections in which no turned projection
    // index k + u Q wraps past N (k within one quarter [b Q, (b + 1) Q))
    for (int kb = half * (N / 2); kb < kend;) {
        const int blk = kb / Q;
        const int ke = min(min(kend, kb + kFold), (blk + 1) * Q);
        // column u reads projection k + u Q (mod N): QUAD, slot (blk + u) mod 4
        // of the cells of k mod Q (the sums are kept by slot); otherwise
        // (u Q - N [blk + u >= 4]) planes from projection k
        const unsigned d1 = (unsigned)(Q - (blk >= 3 ? N : 0)) * plane;
        const unsigned d2 = (unsigned)(2 * Q - (blk >= 2 ? N : 0)) * plane;
        const unsigned d3 = (unsigned)(3 * Q - (blk >= 1 ? N : 0)) * plane;
        float2 a01[NS], a23[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) a01[i] = a23[i] = make_float2(0.0f, 0.0f);
        for (int k = kb; k < ke; ++k) {
            const float2 cs = p.trig[k];
            const float U = g.sad - (x * cs.x + y * cs.y);
            const float ru = y * cs.x - x * cs.y;
            float iU;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iU) : "f"(U));
            iU = fmaf(iU, fmaf(-U, iU, 1.0f), iU);
            float fu = fmaf(ru * iU, sdd_du, cu1);
            if (CLAMP) fu = fminf(fmaxf(fu, 0.0f), umax);
            const float tu = __fadd_rd(fu, kTwo23);          // 2^23 + floor(fu)
            const float au = fu - (tu - kTwo23);
            const float2 w2 = f2((g.sad * iU) * (g.sad * iU));
            const float2 au2 = f2(au);
            const float fv0 = fmaf(zc * iU, sdd_dv, cv1);
            const float dfv = dz_dv * iU;
            // offset of row r + 1 of the column (QUAD: in cells of k mod Q;
            // otherwise in pairs of projection k): (2^23 + r) pw + o in 32-bit
            // modular arithmetic (the true offsets are below 2^31)
            const unsigned o = (unsigned)(QUAD ? k - blk * Q : k) * plane +
                               (unsigned)(__float_as_int(tu) - two23) + (unsigned)(1 - two23) * (unsigned)p.pw;
            float2 lo01, lo23, hi01, hi23;
            int jp = 0;
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                if (FULL || i < ns) {
                    float fv = fmaf((float)i, dfv, fv0);
                    if (CLAMP) fv = fminf(fmaxf(fv, 0.0f), vmaxp);
                    const float tv = __fadd_rd(fv, kTwo23);      // 2^23 + floor(fv)
                    const float2 av = f2(fv - (tv - kTwo23));
                    const int j = __float_as_int(tv);
                    const unsigned r = (unsigned)j * (unsigned)p.pw;
                    if (!QUAD && (i == 0 || !THIN)) {
                        // rows j and j + 1 of each column
                        const unsigned rl = r - (unsigned)p.pw + o;
                        const float2 p0 = __ldg(f + rl), p1 = __ldg(f + (rl + d1));
                        const float2 p2 = __ldg(f + (rl + d2)), p3 = __ldg(f + (rl + d3));
                        const float2 q0 = __ldg(f + (r + o)), q1 = __ldg(f + (r + o + d1));
                        const float2 q2 = __ldg(f + (r + o + d2)), q3 = __ldg(f + (r + o + d3));
                        lo01.x = fmaf(au, p0.y, p0.x);
                        lo01.y = fmaf(au, p1.y, p1.x);
                        lo23.x = fmaf(au, p2.y, p2.x);
                        lo23.y = fmaf(au, p3.y, p3.x);
                        hi01.x = fmaf(au, q0.y, q0.x);
                        hi01.y = fmaf(au, q1.y, q1.x);
                        hi23.x = fmaf(au, q2.y, q2.x);
                        hi23.y = fmaf(au, q3.y, q3.x);
                    } else if (!QUAD && j != jp) {
                        // the row advanced: the old row j + 1 is row j; load the new row j + 1
                        const float2 q0 = __ldg(f + (r + o)), q1 = __ldg(f + (r + o + d1));
                        const float2 q2 = __ldg(f + (r + o + d2)), q3 = __ldg(f + (r + o + d3));
                        lo01 = hi01;
                        lo23 = hi23;
                        hi01.x = fmaf(au, q0.y, q0.x);
                        hi01.y = fmaf(au, q1.y, q1.x);
                        hi23.x = fmaf(au, q2.y, q2.x);
                        hi23.y = fmaf(au, q3.y, q3.x);
                    } else if (QUAD && (i == 0 || !THIN)) {
                        // rows j and j + 1 of each slot: value + au difference
                        const float4 *cl = fq + 2u * (r - (unsigned)p.pw + o), *ch = fq + 2u * (r + o);
                        const float4 pa = __ldg(cl), pb = __ldg(cl + 1);
                        const float4 qa = __ldg(ch), qb = __ldg(ch + 1);
                        lo01 = __ffma2_rn(au2, make_float2(pa.z, pa.w), make_float2(pa.x, pa.y));
                        lo23 = __ffma2_rn(au2, make_float2(pb.z, pb.w), make_float2(pb.x, pb.y));
                        hi01 = __ffma2_rn(au2, make_float2(qa.z, qa.w), make_float2(qa.x, qa.y));
                        hi23 = __ffma2_rn(au2, make_float2(qb.z, qb.w), make_float2(qb.x, qb.y));
                    } else if (QUAD && j != jp) {
                        // the row advanced: the old row j + 1 is row j; load the new row j + 1
                        const float4 *ch = fq + 2u * (r + o);
                        const float4 qa = __ldg(ch), qb = __ldg(ch + 1);
                        lo01 = hi01;
                        lo23 = hi23;
                        hi01 = __ffma2_rn(au2, make_float2(qa.z, qa.w), make_float2(qa.x, qa.y));
                        hi23 = __ffma2_rn(au2, make_float2(qb.z, qb.w), make_float2(qb.x, qb.y));
                    }
                    jp = j;
                    a01[i] = __ffma2_rn(w2, __ffma2_rn(av, sub2(hi01, lo01), lo01), a01[i]);
                    a23[i] = __ffma2_rn(w2, __ffma2_rn(av, sub2(hi23, lo23), lo23), a23[i]);
                }
            }
        }
        // QUAD: slot s holds column (s - blk) mod 4; one sum at a time (the
        // compiler otherwise hoists every shared load and conversion of the
        // fold and spills)
        const int c0 = QUAD ? (4 - blk) & 3 : 0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            accd[4 * i + c0][t] += (double)a01[i].x;
            asm volatile("" ::: "memory");
            accd[4 * i + ((c0 + 1) & 3)][t] += (double)a01[i].y;
            asm volatile("" ::: "memory");
            accd[4 * i + ((c0 + 2) & 3)][t] += (double)a23[i].x;
            asm volatile("" ::: "memory");
            accd[4 * i + ((c0 + 3) & 3)][t] += (double)a23[i].y;
            asm volatile("" ::: "memory");
        }
        kb = ke;
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        if (i < ns) {
            const size_t zo = (size_t)(zb + i) * n;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // the orbit's columns c, R c, R^2 c, R^3 c
                const int cx = u == 0 ? ix : u == 1 ? n - 1 - iy : u == 2 ? n - 1 - ix : iy;
                const int cy = u == 0 ? iy : u == 1 ? ix : u == 2 ? n - 1 - iy : n - 1 - ix;
                atomicAdd(vol + (zo + cy) * n + cx, accd[4 * i + u][t] * p.scale);
                asm volatile("" ::: "memory");
            }
        }
    }
}

// Whether a voxel can project outside the stored filtered rows (fdk_row_range
// cut them at a detector edge) or outside the detector columns with less
// than two pixels to spare (|u| <= SDD r_max / (SAD - r_max) at the voxels).
static bool slab_needs_clamp(const DevGeom &g)
{
    const double hx = 0.5 * g.nx * (double)g.dx, hy = 0.5 * g.ny * (double)g.dy;
    const double rmax = sqrt(hx * hx + hy * hy);
    const double umin = (double)g.sad - rmax;
    if (umin <= 0.0) return true;
    const double vmax = 0.5 * (g.nz - 1) * (double)g.dz * (double)g.sdd / umin / (double)g.dv;
    const double uext = (double)g.sdd * rmax / umin / (double)g.du;
    return (int)floor((double)g.cv - vmax) - 2 < 0 || (int)ceil((double)g.cv + vmax) + 2 > g.n_v - 1 ||
           uext + 2.0 > (double)g.cu;
}

// Largest projected z pitch, in detector rows, over the voxels of the
// volume (U >= SAD - r_max); +inf when the volume reaches the source.
double fdk_slab_row_step(const DevGeom &g)
{
    const double hx = 0.5 * g.nx * (double)g.dx, hy = 0.5 * g.ny * (double)g.dy;
    const double umin = (double)g.sad - sqrt(hx * hx + hy * hy);
    if (umin <= 0.0) return INFINITY;
    return (double)g.dz * (double)g.sdd / umin / (double)g.dv;
}

template <int S, bool THIN>
static int sym_occupancy(bool clamp)
{
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n,
        clamp ? (const void *)k_backproject_sym<S, true, THIN, false, false>
              : (const void *)k_backproject_sym<S, false, THIN, false, false>,
        256, 0);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

// Slice runs of the quarter-turn kernel: the number of balanced runs (at
// most kSymMaxRun slices each) whose grid, in whole rounds of resident
// CTAs, issues the fewest instructions per SM (a column set-up of about 30
// instructions per projection and run, about 28 per slice on thin slabs and
// 40 otherwise; a short last round costs as much as a full one; on thin
// slabs runs of equal length, which need no run-length test, cost 10% less:
// paper-scale 3.98 -> 3.64 ms, while on the head-like 256^3 scan 64 equal
// runs of 4 measured 6.95 ms against 4.88 ms for 52 runs of up to 5).
static void sym_launch_shape(const FdkParams &p, bool clamp, bool thin, int *ns_out, bool *full, dim3 *grid)
{
    const int tx = (p.g.nx / 2 + 31) / 32, ty = (p.g.nx / 2 + 7) / 8;
    const long tiles = (long)tx * ty;
    double best = 0.0;
    int br = 0;
    for (int runs = (p.g.nz + kSymMaxRun - 1) / kSymMaxRun; runs <= p.g.nz; ++runs) {
        const int ns = (p.g.nz + runs - 1) / runs;
        int occ = 1;
#define FC_OCC(S) \
    case S: occ = thin ? sym_occupancy<S, true>(clamp) : sym_occupancy<S, false>(clamp); break;
        switch (ns) {
        FC_OCC(1) FC_OCC(2) FC_OCC(3) FC_OCC(4)
        default: occ = thin ? sym_occupancy<5, true>(clamp) : sym_occupancy<5, false>(clamp); break;
        }
#undef FC_OCC
        const long slots = (long)occ * sm_count();
        const long rounds = (tiles * runs * 2 + slots - 1) / slots;
        const double cost = (double)rounds * (30.0 + (thin ? 28.0 : 40.0) * ns) *
                            (thin && p.g.nz % runs == 0 ? 0.9 : 1.0);
        if (br == 0 || cost < best) {
            best = cost;
            br = runs;
        }
    }
    *ns_out = (p.g.nz + br - 1) / br;
    *full = p.g.nz % br == 0;
    *grid = dim3(tx, ty, 2 * br);
}

int backproject_variant(const FdkParams &p, int request)
{
    // every kernel addresses the filtered rows with 32-bit element offsets
    if ((double)p.g.n_angles * p.ph * p.pw >= 2147483648.0) return -1;
    const bool slab_ok = p.g.nz <= kSlabMaxNz && fdk_slab_row_step(p.g) <= kSlabMaxStep;
    const bool quarter = p.sym_quarter > 0 && 4 * p.sym_quarter == p.g.n_angles && p.g.nx == p.g.ny &&
                         p.g.nx % 2 == 0;
    const bool sym_ok = slab_ok && quarter;
    if (request == FC_BP_SLAB_SYM) return sym_ok ? FC_BP_SLAB_SYM : -1;
    if (request == FC_BP_CHUNKED_SYM) return quarter ? FC_BP_CHUNKED_SYM : -1;
    if (request == FC_BP_SLAB) return slab_ok ? FC_BP_SLAB : -1;
    if (request == FC_BP_CHUNKED || request == FC_BP_CHUNKED_DENSE) return request;
    if (request != FC_BP_AUTO) return -1;
    if (sym_ok) return FC_BP_SLAB_SYM;
    if (slab_ok) return FC_BP_SLAB;
    // thick volumes of a full-circle scan: catphan_kv 0.327 -> 0.278 ms,
    // the head-like 256^3 scan 6.25 -> 4.88 ms against the chunked kernels
    if (quarter) return FC_BP_CHUNKED_SYM;
    int zc;
    dim3 grid;
    chunked_launch_shape(p, &zc, &grid);
    // A grid of two or more waves at 6 CTAs per SM runs faster with 8
    // resident CTAs (more warps to hide the tap latency; 512^2 x 10 voxels
    // with 180 projections: 1.087 -> 0.872 ms); a grid of about one wave
    // (256^2 x 10: 1024 CTAs) runs faster with the unspilled 40-register
    // kernel.
    return (long)grid.x * grid.y * grid.z >= 2L * sm_count() * 6 ? FC_BP_CHUNKED_DENSE : FC_BP_CHUNKED;
}

// The thin-slab quarter-turn kernel reads quarter-interleaved filtered rows
// where the in-plane voxel pitch projects to at most one detector column at
// the axis: a warp's 8 x 4 columns then sample few distinct cells, and the
// packed loads save instructions (paper-scale MV case, 0.6 columns per
// voxel: 3.65 -> 3.08 ms).  Where the pitch projects to ~2 columns, each
// lane reads its own 32-byte cell and the L1 sectors per tap row outnumber
// those of four 8-byte loads from four projections (the thick-volume form
// measured 0.278 -> 0.434 ms on catphan_kv, 2.3 columns per voxel, and
// 4.88 -> 7.15 ms on the head-like scan, 1.9), so those read the plain rows.
bool backproject_reads_quad(const FdkParams &p, int variant)
{
    return variant == FC_BP_SLAB_SYM && (double)p.g.dx * p.g.sdd <= (double)p.g.du * p.g.sad;
}

cudaError_t launch_backproject(const FdkParams &p, const float2 *filt, double *vol, int variant,
                               cudaStream_t s)
{
    if (variant == FC_BP_SLAB_SYM || variant == FC_BP_CHUNKED_SYM) {
        const bool clamp = slab_needs_clamp(p.g), thin = variant == FC_BP_SLAB_SYM;
        // the filter wrote the layout this variant reads
        if ((p.filt_quad != 0) != backproject_reads_quad(p, variant)) return cudaErrorInvalidValue;
        const bool quad = p.filt_quad != 0;
        int ns;
        bool full;
        dim3 grid;
        sym_launch_shape(p, clamp, thin, &ns, &full, &grid);
        const dim3 block(32, 8);
        // the two halves add onto zero
        const cudaError_t e = cudaMemsetAsync(vol, 0, sizeof(double) * (size_t)p.g.nx * p.g.ny * p.g.nz, s);
        if (e != cudaSuccess) return e;
#define FC_BPY_F(S, C, T, Q)                                                                  \
    (full ? (k_backproject_sym<S, C, T, true, Q><<<grid, block, 0, s>>>(p, filt, vol), 0)        \
          : (k_backproject_sym<S, C, T, false, Q><<<grid, block, 0, s>>>(p, filt, vol), 0))
#define FC_BPY(S)                                                                             \
    case S:                                                                                   \
        if (thin && quad) (void)(clamp ? FC_BPY_F(S, true, true, true) : FC_BPY_F(S, false, true, true)); \
        else if (thin) (void)(clamp ? FC_BPY_F(S, true, true, false) : FC_BPY_F(S, false, true, false)); \
        else (void)(clamp ? FC_BPY_F(S, true, false, false) : FC_BPY_F(S, false, false, false)); \
        break;
        switch (ns) {
        FC_BPY(1) FC_BPY(2) FC_BPY(3) FC_BPY(4) FC_BPY(5)
        default:
            return cudaErrorInvalidValue;
        }
#undef FC_BPY
#undef FC_BPY_F
        return cudaGetLastError();
    }
    if (variant == FC_BP_SLAB) {
        dim3 block(32, 8);
        dim3 grid((p.g.nx + 31) / 32, (p.g.ny + 7) / 8);
        // the stored rows [v_lo, v_hi] hold every row a voxel projects onto
        // (with two rows of margin) unless the range was cut at a detector
        // edge; only then can a row coordinate leave the stored rows
        const bool clamp = slab_needs_clamp(p.g);
#define FC_BPS(Z)                                                              \
    case Z:                                                                    \
        if (clamp)                                                             \
            k_backproject_slab<Z, true><<<grid, block, 0, s>>>(p, filt, vol);  \
        else                                                                   \
            k_backproject_slab<Z, false><<<grid, block, 0, s>>>(p, filt, vol); \
        break;
        switch (p.g.nz) {
        FC_BPS(1) FC_BPS(2) FC_BPS(3) FC_BPS(4) FC_BPS(5) FC_BPS(6) FC_BPS(7) FC_BPS(8)
        FC_BPS(9) FC_BPS(10) FC_BPS(11) FC_BPS(12) FC_BPS(13) FC_BPS(14) FC_BPS(15) FC_BPS(16)
        default:
            return cudaErrorInvalidValue;
        }
#undef FC_BPS
        return cudaGetLastError();
    }
    if (variant != FC_BP_CHUNKED && variant != FC_BP_CHUNKED_DENSE) return cudaErrorInvalidValue;
    const bool dense = variant == FC_BP_CHUNKED_DENSE;
    dim3 block(32, 8);
    int zc;
    dim3 grid;
    chunked_launch_shape(p, &zc, &grid);
#define FC_BP(Z)                                                                  \
    case Z:                                                                       \
        if (dense)                                                                \
            k_backproject_dense<Z><<<grid, block, 0, s>>>(p, filt, vol);          \
        else                                                                      \
            k_backproject<Z><<<grid, block, 0, s>>>(p, filt, vol);                \
        break;
    switch (zc) {
    FC_BP(1)
    FC_BP(2)
    FC_BP(3)
    FC_BP(4)
    FC_BP(5)
    FC_BP(6)
    FC_BP(7)
    default:
    FC_BP(8)
    }
#undef FC_BP
    return cudaGetLastError();
}

// ---- HU: mu_w = mean over the water region; HU = 1000 (mu - mu_w) / mu_w
namespace {
constexpr int kRoiBlocks = 256;
}

__global__ void k_roi_partial(DevGeom g, const double *__restrict__ vol, double *partials,
                              float r2, int zcut)
{
    __shared__ double ssum[256];
    __shared__ double scnt[256];
    // one (x, y) column per thread and pass, its z range in an inner loop
    // (32-bit index arithmetic: nx ny < 2^31)
    const int nxy = g.nx * g.ny;
    double s = 0.0, c = 0.0;
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < nxy; col += gridDim.x * blockDim.x) {
        const float x = ((float)(col % g.nx) - 0.5f * (float)(g.nx - 1)) * g.dx;
        const float y = ((float)(col / g.nx) - 0.5f * (float)(g.ny - 1)) * g.dy;
        if (x * x + y * y > r2) continue;
        for (int iz = zcut; iz < g.nz - zcut; ++iz) {
            s += vol[(size_t)iz * nxy + col];
            c += 1.0;
        }
    }
    ssum[threadIdx.x] = s;
    scnt[threadIdx.x] = c;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            ssum[threadIdx.x] += ssum[threadIdx.x + st];
            scnt[threadIdx.x] += scnt[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = ssum[0];
        partials[2 * blockIdx.x + 1] = scnt[0];
    }
}

__global__ void k_hu(DevGeom g, const double *__restrict__ vol, const double *__restrict__ partials,
                     float *__restrict__ hu)
{
    // every CTA folds the partials the same way (thread b takes block b's,
    // then a fixed tree), so all obtain the same mu_w
    __shared__ double ssum[kRoiBlocks], scnt[kRoiBlocks];
    static_assert(kRoiBlocks == 256, "one partial per thread");
    ssum[threadIdx.x] = partials[2 * threadIdx.x];
    scnt[threadIdx.x] = partials[2 * threadIdx.x + 1];
    __syncthreads();
    for (int st = kRoiBlocks / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            ssum[threadIdx.x] += ssum[threadIdx.x + st];
            scnt[threadIdx.x] += scnt[threadIdx.x + st];
        }
        __syncthreads();
    }
    const double m = scnt[0] > 0.0 ? ssum[0] / scnt[0] : 0.0;
    const double k = m != 0.0 ? 1000.0 / m : 0.0;    // HU = 1000 (mu - mu_w) / mu_w
    // per voxel in binary32, HU = mu k - mu_w k as one fma: the result is
    // binary32 anyway, and the rounding of mu and of the two products moves
    // it by ~1e-4 HU, while GB300's binary64 rate made the binary64 form the
    // kernel's bound
    const float kf = (float)k, bf = (float)(-m * k);
    // four voxels per thread and pass (two 16-byte loads, one 16-byte store:
    // more bytes in flight per warp than one 8-byte load), then the tail;
    // both buffers are the handle's (256-byte aligned)
    const size_t n = (size_t)g.nx * g.ny * g.nz, n4 = n / 4;
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
    const double2 *v2 = reinterpret_cast<const double2 *>(vol);
    float4 *h4 = reinterpret_cast<float4 *>(hu);
    for (size_t i = i0; i < n4; i += step) {
        const double2 a = __ldg(v2 + 2 * i), b = __ldg(v2 + 2 * i + 1);
        h4[i] = make_float4(fmaf((float)a.x, kf, bf), fmaf((float)a.y, kf, bf), fmaf((float)b.x, kf, bf),
                            fmaf((float)b.y, kf, bf));
    }
    for (size_t i = 4 * n4 + i0; i < n; i += step) hu[i] = fmaf((float)vol[i], kf, bf);
}

cudaError_t launch_hu(const DevGeom &g, const double *vol, float *hu, double *partials, float radius,
                      int zcut, cudaStream_t s)
{
    k_roi_partial<<<kRoiBlocks, 256, 0, s>>>(g, vol, partials, radius * radius, zcut);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_hu<<<sm_count() * 4, 256, 0, s>>>(g, vol, partials, hu);
    return cudaGetLastError();
}

}  // namespace fc

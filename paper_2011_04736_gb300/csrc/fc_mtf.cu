// Detector MTF by the slanted-slit method (Sec. II.C): the detector PSF
// (each energy group's optical spread weighted by the group's share of the
// flood, or the single optical-spread kernel) is applied to an ideal slit
// tilted across the pixel grid, the line spread function is presampled on a
// grid d / os fine, and the MTF is its Fourier magnitude.  The problem is
// small (a 192 x 192 image, 32 os bins), so every kernel works in binary64
// and in fixed orders (results reproducible bit for bit).
//   k_mtf_slit  area fraction of each pixel inside |n . (x - c)| <= w / 2
//               (the pixel's distribution of n . x is the convolution of two
//               uniforms of widths d |cos a| and d |sin a|: a trapezoid);
//   k_mtf_blur  I = sum_g c_g G_g (x) S, clamp-to-edge sampled Gaussians;
//   k_mtf_bins  the presampling bin of every pixel of rows [N/4, 3N/4);
//   k_mtf_lsf   one CTA per bin: mean of I over that bin's pixels;
//   k_mtf_dft   one CTA per frequency k / (32 d), k = 0 .. 16 os.
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

// CDF at t of the sum of two centred uniforms of widths a >= b >= 0.
__device__ double trap_cdf(double t, double a, double b)
{
    if (b == 0.0) return fmin(fmax(__ddiv_rn(__dadd_rn(t, 0.5 * a), a), 0.0), 1.0);
    double x = __dadd_rn(t, 0.5 * (a + b));
    x = fmin(fmax(x, 0.0), a + b);
    if (x <= b) return __ddiv_rn(__dmul_rn(x, x), 2.0 * a * b);
    if (x <= a) return __ddiv_rn(__dsub_rn(x, 0.5 * b), a);
    const double y = __dsub_rn(a + b, x);
    return __dsub_rn(1.0, __ddiv_rn(__dmul_rn(y, y), 2.0 * a * b));
}

// signed distance of pixel (row i, column j) from the slit's centre line
__device__ __forceinline__ double dist(const MtfParams &p, int i, int j)
{
    const double x = __dmul_rn((double)j - 0.5 * (p.n - 1), p.pitch);
    const double y = __dmul_rn((double)i - 0.5 * (p.n - 1), p.pitch);
    return __dadd_rn(__dmul_rn(x, p.ca), __dmul_rn(y, p.sa));
}

}  // namespace

__global__ void k_mtf_slit(const __grid_constant__ MtfParams p, double *S)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.n * p.n) return;
    const double s = dist(p, e / p.n, e % p.n);
    const double a = p.pitch * fmax(fabs(p.ca), fabs(p.sa));
    const double b = p.pitch * fmin(fabs(p.ca), fabs(p.sa));
    S[e] = trap_cdf(__dadd_rn(-s, 0.5 * p.width), a, b) - trap_cdf(__dsub_rn(-s, 0.5 * p.width), a, b);
}

__global__ void k_mtf_blur(const __grid_constant__ MtfParams p, const double *S, double *I)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.n * p.n) return;
    const int i = e / p.n, j = e % p.n;
    double acc = 0.0;
    for (int g = 0; g < p.n_groups; ++g) {
        const int R = p.r[g];
        double sg = 0.0;
        for (int jv = -R; jv <= R; ++jv) {
            const double *row = S + (size_t)clampi(i + jv, p.n) * p.n;
            double sr = 0.0;
            for (int ju = -R; ju <= R; ++ju) sr = fma(p.taps[g][ju + R], row[clampi(j + ju, p.n)], sr);
            sg = fma(p.taps[g][jv + R], sr, sg);
        }
        acc = fma(p.wgt[g], sg, acc);
    }
    I[e] = acc;
}

// bin of every pixel of rows [row0, row1) (-1 outside the bins)
__global__ void k_mtf_bins(const __grid_constant__ MtfParams p, int *bins)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nr = p.row1 - p.row0;
    if (e >= nr * p.n) return;
    const int i = p.row0 + e / p.n, j = e % p.n;
    const double q = floor(__dadd_rn(__ddiv_rn(dist(p, i, j), p.delta), 0.5 * p.nb));
    bins[e] = (q >= 0.0 && q < (double)p.nb) ? (int)q : -1;
}

// mean of I over each bin: one CTA per bin; thread t sums the bin's pixels
// t, t + 256, ... (row-major), then a fixed tree (reproducible bits)
constexpr int kLsfThreads = 256;
__global__ void __launch_bounds__(kLsfThreads)
k_mtf_lsf(const __grid_constant__ MtfParams p, const double *I, const int *bins, double *lsf)
{
    __shared__ double st[kLsfThreads];
    __shared__ int sc[kLsfThreads];
    const int b = blockIdx.x;
    const int nr = p.row1 - p.row0;
    double tot = 0.0;
    int cnt = 0;
    for (int e = threadIdx.x; e < nr * p.n; e += kLsfThreads)
        if (bins[e] == b) {
            tot += I[(size_t)(p.row0 + e / p.n) * p.n + e % p.n];
            ++cnt;
        }
    st[threadIdx.x] = tot;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int h = kLsfThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            st[threadIdx.x] += st[threadIdx.x + h];
            sc[threadIdx.x] += sc[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) lsf[b] = sc[0] ? st[0] / sc[0] : 0.0;
}

// one CTA per frequency: thread t takes bins t, t + 128, ..., then a fixed
// tree of the real part, the imaginary part and the LSF sum
constexpr int kDftThreads = 128;
__global__ void __launch_bounds__(kDftThreads)
k_mtf_dft(const __grid_constant__ MtfParams p, const double *lsf, double *freq, double *mtf)
{
    __shared__ double sre[kDftThreads], sim[kDftThreads], ssum[kDftThreads];
    const int k = blockIdx.x;
    const double f = k / (p.nb * p.delta);           // 1/cm
    double re = 0.0, im = 0.0, sum = 0.0;
    for (int b = threadIdx.x; b < p.nb; b += kDftThreads) {
        const double sb = (b - 0.5 * p.nb + 0.5) * p.delta;
        double sn, cs;
        sincospi(2.0 * f * sb, &sn, &cs);
        re = fma(lsf[b], cs, re);
        im = fma(-lsf[b], sn, im);
        sum += lsf[b];
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    ssum[threadIdx.x] = sum;
    __syncthreads();
    for (int h = kDftThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sre[threadIdx.x] += sre[threadIdx.x + h];
            sim[threadIdx.x] += sim[threadIdx.x + h];
            ssum[threadIdx.x] += ssum[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        freq[k] = f / 10.0;
        mtf[k] = sqrt(sre[0] * sre[0] + sim[0] * sim[0]) / fabs(ssum[0]);
    }
}

cudaError_t launch_mtf(const MtfParams &p, double *work, double *freq, double *mtf, cudaStream_t s)
{
    const int np = p.n * p.n;
    double *S = work, *I = work + np, *lsf = work + 2 * (size_t)np;
    int *bins = reinterpret_cast<int *>(S);       // S is no longer needed after the blur
    const int nb_px = (p.row1 - p.row0) * p.n;
    k_mtf_slit<<<(np + 255) / 256, 256, 0, s>>>(p, S);
    k_mtf_blur<<<(np + 255) / 256, 256, 0, s>>>(p, S, I);
    k_mtf_bins<<<(nb_px + 255) / 256, 256, 0, s>>>(p, bins);
    k_mtf_lsf<<<p.nb, kLsfThreads, 0, s>>>(p, I, bins, lsf);
    k_mtf_dft<<<p.nb / 2 + 1, kDftThreads, 0, s>>>(p, lsf, freq, mtf);
    return cudaGetLastError();
}

}  // namespace fc

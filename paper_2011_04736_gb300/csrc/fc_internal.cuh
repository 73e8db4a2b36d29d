// Internal declarations shared by the CUDA translation units of libfastcat.
#pragma once
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fastcat.h"

namespace fc {

// 2^x by the hardware approximation (ex2.approx.ftz; subnormal results are
// flushed to zero), the energy integral's exponential.  Its error enters T
// through the parity tests against the binary64 oracle (<= 1e-4 relative).
__device__ __forceinline__ float exp2_hw(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kMaxMat = FC_MAX_MATERIALS;
constexpr int kMaxBins = FC_MAX_BINS;
constexpr int kMaxTaps = 2 * 256 + 1;  // 2 * ceil(4 * FC_MAX_SIGMA_PX) + 1
constexpr int kBrick = 8;              // x and y edge of the label bricks the projector skips
constexpr int kBrickZ = 16;            // their depth along z (the rotation axis)
constexpr int kMixed = 255;            // brick-map value of a brick with several labels

// Geometry in the precision the kernels use (binary32), derived on the host
// from the binary64 fc_geometry.
struct DevGeom {
    float sad, sdd;
    float du, dv;
    float cu, cv;           // (n_u - 1) / 2, (n_v - 1) / 2
    int n_u, n_v, n_angles;
    int nx, ny, nz;
    float dx, dy, dz;
    float lox, loy, loz;    // lower box corner = -N d / 2
    float idx, idy, idz;    // 1 / voxel pitch
};

// Projector launch parameters (passed as a __grid_constant__ kernel argument;
// the tables are read with warp-uniform indices).
struct ProjParams {
    DevGeom g;
    const float2 *trig;     // [n_angles] (cos, sin) of each angle
    const uint8_t *labels;  // [nz][ny][nx]
    const uint8_t *labels_zf;  // the same labels z fastest: [ny][nx][nz] (the walk reads these)
    const uint8_t *bricks;  // [ceil(nz/kBrickZ)][ceil(ny/kBrick)][ceil(nx/kBrick)]: uniform label or kMixed
    int angle0;             // absolute index of the first angle of the launch
    int n_angles_launch;
    int v_hit_lo, v_hit_hi; // detector rows whose rays can meet the voxel slab
    int compact;            // trace the band with its rays compacted (most miss the voxels)
    int n_mat, n_e;
    int n_groups;                   // energy-group output (k_project<kModeGroups>)
    int grp_end[FC_MAX_GROUPS];     // exclusive end bin of each group
    float grp_flood[FC_MAX_GROUPS]; // compensated sum of wd over each group (rays that miss)
    size_t grp_stride;              // elements between group planes of the output
    float wd[kMaxBins];             // w D / sum(w D)
    float mu2[kMaxBins][kMaxMat];   // mu * log2(e), zero padded
};

// Energy-group detector model: per-group optical spread and scatter profile.
constexpr int kMaxGroupR = 16;      // ceil(4 * FC_MAX_GROUP_SIGMA_PX)
struct GroupParams {
    int n_u, n_v, n_groups;
    size_t grp_stride;              // elements between group planes of P
    int r[FC_MAX_GROUPS];
    float taps[FC_MAX_GROUPS][2 * kMaxGroupR + 1];   // index j + r[g]
    float tpad[FC_MAX_GROUPS][2 * kMaxGroupR + 1];   // index j + max r (zero padded)
    float amp[FC_MAX_GROUPS], a_cm[FC_MAX_GROUPS], b[FC_MAX_GROUPS];
    float du, cu;                   // detector pitch (cm) and centre column
    float n0;
};

// Richardson-Lucy deconvolution (fc_deconvolve.cu): blur radius <= 16.
struct RlParams {
    int n_u, n_v, R;
    float taps[2 * kMaxGroupR + 1];
    float cl[kMaxGroupR + 1];       // cl[k] = sum of taps j < -k (mass clamped onto index 0)
    float floor_;                   // lower bound of H u before the division
};

// Slanted-slit detector MTF (fc_mtf.cu), binary64 throughout.
struct MtfParams {
    int n;                          // image size (pixels per side)
    double pitch, width, ca, sa;    // cm, cm, slit normal (cos, sin)
    int n_groups;
    double wgt[FC_MAX_GROUPS];      // share of the flood per group, sum 1
    int r[FC_MAX_GROUPS];
    double taps[FC_MAX_GROUPS][2 * kMaxGroupR + 1];
    int nb, row0, row1;             // presampling bins, rows used
    double delta;                   // bin width, cm
};

// Final reduction of the dose estimate (Sec. II.H).
constexpr int kDoseBlocks = 2048;            // most blocks of the per-bin partial sums
constexpr double kGyGramPerKev = 1.602176634e-13;  // 1 keV per gram, in Gy

struct DoseParams {
    int n_e, n_mat, n_part;
    double n_rays;                 // N_i: rays the sums run over
    double voxel_cm3;              // dx dy dz
    double e_kev[kMaxBins];        // bin energies
    double muen[kMaxBins];         // (mu_en / mu) of water
    double phi[kMaxBins];          // fluence spectrum, sum 1
    double rho[kMaxMat];           // material densities, g/cm^3
};

struct BlurParams {
    int n_u, n_v;
    int rp, rs;             // tap radii of the PSF and scatter kernels
    int inject_timeout;     // testing: tensor-core passes give up their first epilogue wait
    float n0, spr;
    float gp[kMaxTaps];     // PSF taps, index j + rp
    float gs[kMaxTaps];     // scatter taps, index j + rs
};

// Tensor-core blur (fc_blur_tc.cu): one band = one sampled-Gaussian kernel
// applied along the pass's axis as a banded Toeplitz product.
struct TcBand {
    const float *src;   // [img][n_v][n_u]
    uint32_t h_off;     // bf16 offset of the band's Hankel hi array (lo follows)
    int pad;            // P = 8 ceil(R / 8)
    int kw;             // window 128 + 2 P
    int ncore;          // Hankel cores 15 + kw / 8
};

// Radii the tensor-core blur takes: the optical spread of the column pass
// runs on the CUDA cores from a staged tile of 128 + 2 R rows, and the scatter
// band matrix of the column pass lives in TMEM beside two accumulators
// (128 + 2 P <= 384 columns).  Larger radii use the direct f32 kernels.
constexpr int kTcMaxPsfR = 16;
constexpr int kTcMaxScR = 128;

struct TcBlurParams {
    TcBand band[2];
    int n_band;
    const uint16_t *H;  // Hankel arrays, bf16 bits
    float *out0, *out1;
    const float *tp;    // column pass: row-blurred optical-spread input
    int n_u, n_v, n_img;
    float n0, spr;
    int rp;                          // column pass: optical-spread radius
    float gp[2 * kTcMaxPsfR + 1];    // and taps
    unsigned int *err;  // set on a bounded-wait timeout
    int x_off, x_cnt;   // rows pass: the 64-line tiles [x_off, x_off + x_cnt) are computed
    int ts_lo, ts_hi;   // columns pass: rows of ts outside [ts_lo, ts_hi) equal ts_const
    float ts_const;
    int tp_lo, tp_hi;   // columns pass: rows of tp outside [tp_lo, tp_hi) equal tp_const
    float tp_const;
    int m_off, m_cnt;   // columns pass: output rows [m_off + 128 i, +128), i < m_cnt, are computed
    unsigned int epi_polls;   // bound of the epilogue's accumulator waits
};

constexpr size_t kBlurTcHankelMax = 2 * 2 * 64 * (15 + (128 + 2 * 256) / 8);  // bf16 elements

// Filtered projections are stored only for the detector rows the
// backprojector can reach, [v_lo, v_hi], in a zero-padded layout
// [angle][1 + (v_hi - v_lo + 1) + 2][1 + n_u + 2] of (value, next value -
// value) pairs: one zero row / column before and two after, so bilinear taps
// need no bounds tests and a tap pair is one 8-byte load.  For the
// quarter-turn backprojectors (filt_quad = 1) the four projections k, k + Q,
// k + 2Q, k + 3Q (Q = n_angles / 4) share one 32-byte cell per padded
// (row, column): [k mod Q][row][column] of (v_0, v_1, d_0, d_1, v_2, v_3,
// d_2, d_3), v_b the value and d_b the difference of projection
// (k mod Q) + b Q, so the four taps of one detector position are two
// 16-byte loads from one address.
struct FdkParams {
    DevGeom g;
    const float2 *trig;
    float log_flood;        // ln(I_flood)
    float tau;              // du * SAD / SDD
    float mag;              // SAD / SDD
    double scale;           // arc / (2 n_angles)
    int v_lo, v_hi;         // reachable detector rows
    int pw, ph;             // padded row length (n_u + 3 rounded up to 4), padded rows (v_hi - v_lo + 1) + 3
    const float2 *fft_tw;   // FFT filter: twiddles exp(-2 pi i k / L), k < L / 2
    const float *fft_k;     // FFT filter: Ram-Lak response / (L tau) at bit-reversed frequency index
    int fft_log2;           // log2 L, L the transform length (>= 2 n_u - 1)
    int sym_quarter;        // n_angles / 4 for a full-circle scan of n_angles divisible by 4 over a
                            // square grid with an even side and dx = dy (quarter-turn symmetry), else 0
    int filt_quad;          // 1: filtered rows in the quarter-interleaved cells (needs sym_quarter > 0)
};

// Whether a backprojector variant reads the quarter-interleaved filtered
// rows for this geometry (the filter then writes them so).
bool backproject_reads_quad(const FdkParams &p, int variant);

void fdk_row_range(const DevGeom &g, int *v_lo, int *v_hi);

// Sets the message fc_last_error() returns on this thread.
void set_last_error(const char *msg);

// Streaming multiprocessors of the current device (queried once per device
// ordinal; 1 if the query fails).  Launchers size persistent and grid-stride
// grids from it.
int sm_count();

// FDK backprojector variants (FC_BP_* in fastcat.h).  backproject_variant
// resolves a request for the geometry (-1: not applicable);
// fdk_slab_row_step is the largest projected z pitch in detector rows.
double fdk_slab_row_step(const DevGeom &g);
int backproject_variant(const FdkParams &p, int request);

// ---- learned surrogate of the energy integral (fc_mlp.cu) ----
constexpr int kMlpHidden = 128;
constexpr int kMlpIn = 8;
// packed fp32 parameter vector: W1 [128][8], b1, W2 [128][128], b2, W3, b3,
// w4 [128], b4, then input scale [8], the spectral-group baseline (weights
// a[4], attenuation mu[4][8]) and the training box [8]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHidden * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpHidden;
constexpr int kOffB2 = kOffW2 + kMlpHidden * kMlpHidden;
constexpr int kOffW3 = kOffB2 + kMlpHidden;
constexpr int kOffB3 = kOffW3 + kMlpHidden * kMlpHidden;
constexpr int kOffW4 = kOffB3 + kMlpHidden;
constexpr int kOffB4 = kOffW4 + kMlpHidden;
constexpr int kMlpParams = kOffB4 + 1;
constexpr int kMlpGroups = 4;
constexpr int kOffScale = kMlpParams;
constexpr int kOffGa = kOffScale + kMaxMat;
constexpr int kOffGmu = kOffGa + kMlpGroups;
constexpr int kOffBox = kOffGmu + kMlpGroups * kMaxMat;
constexpr int kMlpPacked = kOffBox + kMaxMat;
constexpr int kWgradChunk = 1024;   // batch columns per split-K weight-gradient CTA

struct SurrogateParams {
    const __nv_bfloat16 *W1b;   // [128][16] (columns 8..15 repeat 0..7: lo parts of the inputs)
    const __nv_bfloat16 *W2b, *W3b;    // [out][in]
    const __nv_bfloat16 *W2Tb, *W3Tb;  // [in][out]
    const float *P;             // packed fp32 parameters
    int n_mat, n_e;
    float guard;                // rays whose baseline attenuation reaches it are evaluated exactly
    float wd[kMaxBins];
    float mu2[kMaxBins][kMaxMat];
};

// Training workspace for a batch of B samples (feature-major [rows][B]).
struct MlpWork {
    __nv_bfloat16 *xt;          // [16][B]
    __nv_bfloat16 *h1t, *h2t, *h3t, *dz1t, *dz2t, *dz3t;  // [128][B]
    __nv_bfloat16 *g;           // [16][B], row 0 = dLoss / dy_hat, rows 1..15 zero
    float *part;                // [4][n_chunks][128][128] split-K partials
    float *rsum;                // [4][n_chunks][128]
    float *gsum;                // [n_chunks]
};

cudaError_t launch_mlp_eval(const SurrogateParams &p, const float *L, long long n, float *lnT,
                            unsigned int *n_fallback, int *err, cudaStream_t s);
cudaError_t launch_energy_sum_lengths(const SurrogateParams &p, const float *L, long long n,
                                      float *lnT, cudaStream_t s);
// Smallest baseline attenuation among the rays whose surrogate ln T (ys)
// misses the exact y by more than tol, as an order-preserving integer
// atomically minimised into *best (set it to 0x7fffffff first).
cudaError_t launch_guard_scan(const SurrogateParams &p, const float *L, const float *y,
                              const float *ys, long long n, float tol, int *best, cudaStream_t s);
cudaError_t launch_sigma_probe(const float *z, float *s, long long n, cudaStream_t st);
cudaError_t launch_exp(const float *x, float *y, long long n, cudaStream_t s);
cudaError_t launch_mlp_lmax(const float *L, long long n, int n_mat, unsigned int *mx,
                            cudaStream_t s);
cudaError_t launch_mlp_step(const SurrogateParams &p, const float *L, const float *y, long long n,
                            int B, int sample, unsigned long long seed, int step, const MlpWork &w,
                            float *loss, int *err, float *P, float *m1, float *m2, float lr,
                            float bc1, float bc2, float *grad, __nv_bfloat16 *W1b,
                            __nv_bfloat16 *W2b, __nv_bfloat16 *W3b, __nv_bfloat16 *W2Tb,
                            __nv_bfloat16 *W3Tb, cudaStream_t s);

// ---- adjoint of the CNR objective (fc_adjoint.cu) ----
constexpr int kMaxRoi = 8;

struct AdjParams {
    DevGeom g;
    const float2 *trig;
    const uint8_t *labels;      // [nz][ny][nx]
    int n_e;
    float inv_csum;             // 1 / sum_E (w D)_E before normalisation
    float irho0[kMaxMat];       // 1 / nominal density of each material
    float wd[kMaxBins];         // (w D)_E / sum (w D)
    float mu[kMaxBins][kMaxMat];  // attenuation at nominal density, 1/cm
};

struct CnrParams {
    DevGeom g;
    double water_r;
    int zcut, n_roi;
    double cx[kMaxRoi], cy[kMaxRoi], rad[kMaxRoi];
};

cudaError_t launch_project_density(const AdjParams &p, const float *rho, float *T, cudaStream_t s);
cudaError_t launch_project_density_adjoint(const AdjParams &p, const float *rho, const float *gT,
                                           float *grho, double *gwd, cudaStream_t s);
cudaError_t launch_noise_gauss(const float *I, const float *z, float *K, size_t n, cudaStream_t s);
cudaError_t launch_cnr(const CnrParams &c, const double *mu, float *gmu, double *out, double *work,
                       cudaStream_t s);
size_t cnr_work_doubles();
cudaError_t launch_backproject_adjoint(const FdkParams &p, const float *gmu, float *gf,
                                       cudaStream_t s);
cudaError_t launch_filter_adjoint(const FdkParams &p, const float *gf, const float *I,
                                  const float *K, const float *z, float *gI, cudaStream_t s);
// launchers (return cudaError_t of the launch)
// T output: rows [f_lo, f_hi) that no ray of the traced band covers get
// T = 1 (f_hi < 0: every row); L_out: path lengths of every ray.
cudaError_t launch_project(const ProjParams &p, float *T, float *L_out, cudaStream_t s, int f_lo = 0,
                           int f_hi = -1);
int project_launches(const ProjParams &p, int f_lo = 0, int f_hi = -1);
cudaError_t launch_project_groups(const ProjParams &p, float *P, cudaStream_t s);
cudaError_t launch_group_blur(const GroupParams &g, const float *P, float *prof, float *out,
                              int angle0, int n_img, cudaStream_t s);
cudaError_t launch_blur_rows(const BlurParams &p, const float *T, float *tp, float *ts,
                             int n_img, cudaStream_t s);
// whether the direct f32 row / column pass fits its shared-memory staging
// (a row of n_u + 2R samples; a tile of columns over all n_v rows)
bool blur_rows_fit(const BlurParams &p);
bool blur_cols_fit(const BlurParams &p);
cudaError_t launch_blur_cols(const BlurParams &p, const float *tp, const float *ts, float *out,
                             int n_img, cudaStream_t s);
// transposed blur: gout = n0 (G_psf^T + spr G_scatter^T) gin (tp, ts scratch)
cudaError_t launch_blur_transpose(const BlurParams &p, const float *gin, float *tp, float *ts,
                                  float *gout, int n_img, cudaStream_t s);
// Poisson counts of rates lam; with c_hi >= 0, the rows outside [c_lo, c_hi)
// of every image take the rate cst instead of reading lam (out is written
// everywhere).
cudaError_t launch_poisson(const float *lam, float *out, int n_img, int n_v, int n_u,
                           int angle0, uint64_t seed, cudaStream_t s, int c_lo = 0, int c_hi = -1,
                           float cst = 0.0f);
// Tables of the FFT ramp filter for rows of n_u samples: log2 of the
// transform length L (the smallest power of two >= 2 n_u - 1), the L / 2
// twiddles and the L values of the Ram-Lak response / (L tau) in the
// bit-reversed order the forward transform leaves the spectrum in.
int fdk_fft_log2(int n_u);
void fdk_fft_tables(int n_u, double tau, std::vector<float2> *tw, std::vector<float> *kbr);

cudaError_t launch_fdk_filter(const FdkParams &p, const float *counts, float2 *filt,
                              cudaStream_t s);
cudaError_t launch_backproject(const FdkParams &p, const float2 *filt, double *vol, int variant,
                               cudaStream_t s);
cudaError_t launch_hu(const DevGeom &g, const double *vol, float *hu, double *partials,
                      float radius, int zcut, cudaStream_t s);
bool blur_tc_supported(const BlurParams &bp);
cudaError_t launch_blur_tc_rows(const BlurParams &bp, const float *in, float *tp, float *ts,
                                uint16_t *hankel, unsigned int *err, int n_img, cudaStream_t s,
                                int one_lo = 0, int one_hi = -1);
int blur_tc_rows_launches(const BlurParams &bp, int one_lo, int one_hi);
// rows [lo, hi) of the input that launch_blur_tc_rows reads (with one_hi < 0:
// every row)
void blur_tc_rows_read(const BlurParams &bp, int one_lo, int one_hi, int *lo, int *hi);
int blur_tc_cols_launches(const BlurParams &bp, int one_lo, int one_hi);
// Blur of an input that is 1 outside the rows [b_lo, b_hi) (fc_blur_band.cu):
// one kernel reading only those rows and writing every output pixel, or,
// with write_const false, only the rows [c_lo, c_hi) near the band, the
// others holding the constant cst (blur_band_rows gives both).
bool blur_band_supported(const BlurParams &bp, int b_lo, int b_hi);
void blur_band_rows(const BlurParams &bp, int b_lo, int b_hi, int *c_lo, int *c_hi, float *cst);
cudaError_t launch_blur_band(const BlurParams &bp, const float *T, float *out, int n_img, int b_lo,
                             int b_hi, cudaStream_t s, bool write_const = true);
cudaError_t launch_blur_tc_cols(const BlurParams &bp, const float *tp, const float *ts, float *out,
                                const uint16_t *hankel, unsigned int *err, int n_img, cudaStream_t s,
                                int one_lo = 0, int one_hi = -1);
cudaError_t launch_rl(const RlParams &p, const float *d, float *ua, float *ub, float *norm,
                      int n_img, int n_iter, float **result, cudaStream_t s);
cudaError_t launch_mtf(const MtfParams &p, double *work, double *freq, double *mtf, cudaStream_t s);
cudaError_t launch_dose(const ProjParams &p, const DoseParams &d, double *part,
                        unsigned long long *count, double *out, cudaStream_t s);
int dose_blocks(const ProjParams &p);
cudaError_t launch_labels_zfast(const uint8_t *labels, uint8_t *labels_zf, int nx, int ny, int nz,
                                cudaStream_t s);
cudaError_t launch_brick_map(const uint8_t *labels, uint8_t *bricks, int nx, int ny, int nz,
                             int n_mat, unsigned int *bad, cudaStream_t s);

}  // namespace fc

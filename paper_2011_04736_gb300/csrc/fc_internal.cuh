// Internal declarations shared by the CUDA translation units of libfastcat.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fastcat.h"

namespace fc {

constexpr int kMaxMat = FC_MAX_MATERIALS;
constexpr int kMaxBins = FC_MAX_BINS;
constexpr int kMaxTaps = 2 * 256 + 1;  // 2 * ceil(4 * FC_MAX_SIGMA_PX) + 1
constexpr int kBrick = 8;              // edge of the label bricks the projector skips
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
    const uint8_t *bricks;  // [nz/8][ny/8][nx/8] (rounded up): uniform label or kMixed
    int angle0;             // absolute index of the first angle of the launch
    int n_angles_launch;
    int v_hit_lo, v_hit_hi; // detector rows whose rays can meet the voxel slab
    int n_mat, n_e;
    float wd[kMaxBins];             // w D / sum(w D)
    float mu2[kMaxBins][kMaxMat];   // mu * log2(e), zero padded
};

struct BlurParams {
    int n_u, n_v;
    int rp, rs;             // tap radii of the PSF and scatter kernels
    float n0, spr;
    float gp[kMaxTaps];     // PSF taps, index j + rp
    float gs[kMaxTaps];     // scatter taps, index j + rs
};

// Filtered projections are stored only for the detector rows the
// backprojector can reach, [v_lo, v_hi], in a zero-padded layout
// [angle][1 + (v_hi - v_lo + 1) + 2][1 + n_u + 2]: one zero row / column
// before and two after, so bilinear taps need no bounds tests.
struct FdkParams {
    DevGeom g;
    const float2 *trig;
    float log_flood;        // ln(I_flood)
    float tau;              // du * SAD / SDD
    float mag;              // SAD / SDD
    double scale;           // arc / (2 n_angles)
    int v_lo, v_hi;         // reachable detector rows
    int pw, ph;             // padded row length n_u + 3, padded rows (v_hi - v_lo + 1) + 3
};

void fdk_row_range(const DevGeom &g, int *v_lo, int *v_hi);

// Sets the message fc_last_error() returns on this thread.
void set_last_error(const char *msg);

// launchers (return cudaError_t of the launch)
cudaError_t launch_project(const ProjParams &p, float *T, float *L_out, cudaStream_t s);
cudaError_t launch_blur_rows(const BlurParams &p, const float *T, float *tp, float *ts,
                             int n_img, cudaStream_t s);
cudaError_t launch_blur_cols(const BlurParams &p, const float *tp, const float *ts, float *out,
                             int n_img, cudaStream_t s);
cudaError_t launch_poisson(const float *lam, float *out, int n_img, int n_v, int n_u,
                           int angle0, uint64_t seed, cudaStream_t s);
cudaError_t launch_fdk_filter(const FdkParams &p, const float *counts, float *filt,
                              cudaStream_t s);
cudaError_t launch_backproject(const FdkParams &p, const float *filt, double *vol,
                               cudaStream_t s);
cudaError_t launch_hu(const DevGeom &g, const double *vol, float *hu, double *partials,
                      float radius, int zcut, cudaStream_t s);
cudaError_t launch_brick_map(const uint8_t *labels, uint8_t *bricks, int nx, int ny, int nz,
                             int n_mat, unsigned int *bad, cudaStream_t s);

}  // namespace fc

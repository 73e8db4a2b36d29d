// Allocation-free variant of the detector blur (fc_detector_blur_static).
//
// Some callers cannot allocate device memory once they are running: their
// device memory is owned by another allocator (a pool that reserved the whole
// GPU at start-up) or fixed by a budget that forbids allocation after
// initialisation.  This entry point runs the same row and column blur kernels
// as fc_project, but keeps the two row-pass intermediates in a file-scope
// device array instead of handle-owned buffers, so it needs no handle and
// calls no cudaMalloc / cudaFree (or anything that allocates).
//
// The array is part of the library image: every GPU on which the library is
// loaded holds FC_STATIC_SCRATCH_FLOATS floats of it until the process exits.
// All calls share it and it keeps the contents of the last call, so calls
// whose kernels overlap on the GPU (different streams, or different host
// threads without ordering) race on it.  The row pass overwrites every
// scratch element the column pass then reads, so nothing needs clearing.
// The array's device address is looked up once per device and kept for the
// life of the process; a device reset (cudaDeviceReset, or anything else
// that destroys the primary context) invalidates it and is not supported
// while this library is loaded.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fc_internal.cuh"

namespace {

static __device__ __align__(256) float g_blur_scratch[FC_STATIC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch[kMaxDevices] = {nullptr};

// Device address of g_blur_scratch on the current device.  In host code the
// array's name is a host-side stand-in, not a device address, so it is looked
// up once per device with cudaGetSymbolAddress (that device current).
cudaError_t scratch_for(int dev, float **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_blur_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = (float *)p;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

// Sampled Gaussian, |j| <= ceil(4 sigma), normalised; no heap use.
bool taps_no_alloc(double sigma, float *taps, int *radius)
{
    if (!(sigma >= 0.0) || sigma > FC_MAX_SIGMA_PX) return false;
    const int R = sigma > 0.0 ? (int)ceil(4.0 * sigma) : 0;
    double g[fc::kMaxTaps];
    double sum = 0.0;
    for (int j = -R; j <= R; ++j) {
        g[j + R] = R == 0 ? 1.0 : exp(-(double)j * j / (2.0 * sigma * sigma));
        sum += g[j + R];
    }
    for (int j = 0; j < 2 * R + 1; ++j) taps[j] = (float)(g[j] / sum);
    *radius = R;
    return true;
}

int fail(int code, const char *msg)
{
    fc::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" {

int fc_detector_blur_static(const float *T, float *I, int n_img, int n_v, int n_u,
                            double psf_sigma_px, double scatter_sigma_px, double spr, double n0,
                            void *stream)
{
    if (!T || !I) return fail(FC_EINVAL, "fc_detector_blur_static: null pointer");
    if (n_img <= 0 || n_v <= 0 || n_u <= 0)
        return fail(FC_EINVAL, "fc_detector_blur_static: sizes must be positive");
    const size_t n = (size_t)n_img * n_v * n_u;
    if (2 * n > (size_t)FC_STATIC_SCRATCH_FLOATS)
        return fail(FC_EINVAL, "fc_detector_blur_static: 2 * n_img * n_v * n_u exceeds "
                               "FC_STATIC_SCRATCH_FLOATS; blur fewer projections per call");
    if (!(spr >= 0.0) || !(n0 > 0.0) || !isfinite(spr) || !isfinite(n0))
        return fail(FC_EINVAL, "fc_detector_blur_static: need spr >= 0 and n0 > 0");
    fc::BlurParams b;
    memset(&b, 0, sizeof(b));
    if (!taps_no_alloc(psf_sigma_px, b.gp, &b.rp) || !taps_no_alloc(scatter_sigma_px, b.gs, &b.rs))
        return fail(FC_EINVAL, "fc_detector_blur_static: sigma outside [0, FC_MAX_SIGMA_PX]");
    b.n_u = n_u;
    b.n_v = n_v;
    b.n0 = (float)n0;
    b.spr = (float)spr;
    // both passes stage their inputs in shared memory: a row of n_u + 2R
    // samples (row pass), a tile of columns over all n_v rows (column pass)
    if (!fc::blur_rows_fit(b))
        return fail(FC_EINVAL, "fc_detector_blur_static: detector too wide for the row blur "
                               "(n_u + 2 * blur radius)");
    if (!fc::blur_cols_fit(b))
        return fail(FC_EINVAL, "fc_detector_blur_static: detector too tall for the column blur "
                               "(n_v + blur radii)");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(FC_ECUDA, "fc_detector_blur_static: no device");
    float *scratch = nullptr;
    cudaError_t e = scratch_for(dev, &scratch);
    if (e != cudaSuccess) return fail(FC_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    e = fc::launch_blur_rows(b, T, scratch, scratch + n, n_img, s);
    if (e != cudaSuccess) return fail(FC_ECUDA, cudaGetErrorString(e));
    e = fc::launch_blur_cols(b, scratch, scratch + n, I, n_img, s);
    if (e != cudaSuccess) return fail(FC_ECUDA, cudaGetErrorString(e));
    return FC_OK;
}

}  // extern "C"

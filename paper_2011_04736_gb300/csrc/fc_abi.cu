// C ABI of libfastcat (declarations and conventions in include/fastcat.h).
//
// The handle owns device copies of the phantom and the per-angle
// trigonometry, plus the projection-sized and volume-sized buffers of the
// pipeline (primary signal, the two row-blur intermediates, counts, filtered
// projections, volume, HU).  Geometry and spectrum are reduced here, once,
// to the binary32 tables the kernels read; every per-ray, per-pixel and
// per-voxel step runs in the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include "fc_internal.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define FC_CK(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? FC_ENOMEM : FC_ECUDA,       \
                        "%s: %s", #call, cudaGetErrorString(e_));                     \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Fault injection for tests (fc_inject_fault): device allocations left
// before one fails (-1: none), and whether the next tensor-core blur gives up
// its epilogue waits at once.
std::atomic<long long> g_alloc_fail_in{-1};
std::atomic<int> g_blur_timeout{0};

// cudaMalloc, or the injected failure.
cudaError_t dev_malloc(void **p, size_t bytes)
{
    long long c = g_alloc_fail_in.load();
    while (c >= 0 && !g_alloc_fail_in.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// Padded filtered-projection row: one zero column before the detector row,
// at least two after, rounded up to 16 bytes (tensor-map row stride).
int fdk_row_pitch(int n_u) { return (n_u + 3 + 3) & ~3; }

template <class T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

}  // namespace

void fc::set_last_error(const char *msg) { g_err = msg; }

int fc::sm_count()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kMaxDev) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    if (dev >= 0 && dev < kMaxDev) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

struct fc_handle {
    int device = 0;
    bool has_geom = false, has_phantom = false, has_spec = false, has_counts = false;
    fc_geometry g{};
    fc::DevGeom dg{};
    int phantom_mat = 0;
    // spectrum / detector
    int n_e = 0, n_mat = 0;
    std::vector<float> wd;     // [n_e]
    std::vector<double> phi;   // [n_e] fluence spectrum w / sum w
    std::vector<float> mu2;    // [n_e][kMaxMat]
    double psf = 0.0, sc = 0.0, spr = 0.0, n0 = 1.0;
    uint64_t seed = 0;
    int noise = 0;
    int noise_order = FC_NOISE_AFTER_BLUR;
    int bp_request = FC_BP_AUTO;   // FDK backprojector variant (fc_set_backprojector)
    double band_hit_frac = 1.0;    // share of the traced band's rays that meet the voxels
    // energy-group detector model (off when n_groups == 0)
    int n_groups = 0;
    int grp_end[FC_MAX_GROUPS] = {0};
    double grp_psf[FC_MAX_GROUPS] = {0}, grp_amp[FC_MAX_GROUPS] = {0};
    double grp_a[FC_MAX_GROUPS] = {0}, grp_b[FC_MAX_GROUPS] = {0};
    float *d_grp = nullptr, *d_prof = nullptr;   // group primaries, scatter profile
    float *d_rlnorm = nullptr;                   // deconvolution: H^T 1 per axis
    int grp_alloc = 0;
    double water_r = 1.0, zmargin = 0.1;
    // device buffers
    float2 *d_trig = nullptr;
    uint8_t *d_labels = nullptr;   // caller layout [nz][ny][nx]
    uint8_t *d_labels_zf = nullptr;   // the same, z fastest [ny][nx][nz] (projector walk)
    uint8_t *d_bricks = nullptr;   // 8x8x16 brick map: uniform label or mixed
    float *d_T = nullptr, *d_tp = nullptr, *d_ts = nullptr, *d_counts = nullptr;
    float2 *d_filt = nullptr;   // filtered rows as (value, next - value) pairs
    int filt_quad = -1;         // their layout (FdkParams::filt_quad) since the last zeroing; -1: none yet
    double *d_vol = nullptr;
    float *d_hu = nullptr;
    double *d_part = nullptr;
    unsigned int *d_flag = nullptr;
    size_t proj_elems = 0, vol_elems = 0, filt_elems = 0;
    // kernel-time tracing
    struct Rec {
        int id;
        int launches;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[FC_K_COUNT] = {0};
    int64_t prof_n[FC_K_COUNT] = {0};
    // adjoint of the CNR objective
    float *d_I = nullptr, *d_gI = nullptr, *d_gT = nullptr, *d_gtmp = nullptr, *d_gf = nullptr;
    float *d_gmu = nullptr;
    double *d_gwd = nullptr;
    double *d_cnr_work = nullptr;   // CNR stage partials
    // learned surrogate of the energy integral
    bool has_sur = false, sur_fitted = false;
    double sur_guard = INFINITY;   // fc_surrogate_guard threshold (baseline attenuation)
    int sur_step = 0;
    float *d_P = nullptr, *d_m1 = nullptr, *d_m2 = nullptr, *d_grad = nullptr;
    __nv_bfloat16 *d_W1b = nullptr, *d_W2b = nullptr, *d_W3b = nullptr, *d_W2Tb = nullptr,
                  *d_W3Tb = nullptr;
    fc::MlpWork work{};
    int work_B = 0;
    void *work_mem = nullptr;
    int *d_err = nullptr;
    unsigned int *d_cnt = nullptr;
    float *d_loss = nullptr;
    int loss_cap = 0;
    float *d_sL = nullptr, *d_slnT = nullptr;   // fc_surrogate_project scratch
    size_t sL_rays = 0;
    double *d_dose = nullptr;   // dose estimate: partial sums, result, label counts
    uint16_t *d_hankel = nullptr;   // tensor-core blur band matrices
    unsigned int *d_blur_err = nullptr;
    // FC_HOST_ASYNC outputs of fc_reconstruct: copied on the handle's own
    // stream after ev_done; ev_copied marks the last queued copy's end
    cudaStream_t copy_s = nullptr;
    cudaEvent_t ev_done = nullptr, ev_copied = nullptr;
    bool copy_pending = false;
    // FFT ramp filter tables (twiddles, Ram-Lak response) for fft_n samples
    float2 *d_fft_tw = nullptr;
    float *d_fft_k = nullptr;
    int fft_n = 0;

    void free_all()
    {
        dfree(d_trig);
        dfree(d_labels);
        dfree(d_labels_zf);
        dfree(d_bricks);
        dfree(d_T);
        dfree(d_tp);
        dfree(d_ts);
        dfree(d_counts);
        dfree(d_filt);
        dfree(d_vol);
        dfree(d_hu);
        dfree(d_part);
        dfree(d_flag);
        dfree(d_dose);
        dfree(d_cnr_work);
        dfree(d_grp);
        dfree(d_prof);
        dfree(d_rlnorm);
        dfree(d_hankel);
        dfree(d_blur_err);
        for (auto &r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        pending.clear();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
        dfree(d_I);
        dfree(d_gI);
        dfree(d_gT);
        dfree(d_gtmp);
        dfree(d_gf);
        dfree(d_gmu);
        dfree(d_gwd);
        dfree(d_P);
        dfree(d_m1);
        dfree(d_m2);
        dfree(d_grad);
        dfree(d_W1b);
        dfree(d_W2b);
        dfree(d_W3b);
        dfree(d_W2Tb);
        dfree(d_W3Tb);
        if (work_mem) cudaFree(work_mem);
        work_mem = nullptr;
        dfree(d_err);
        dfree(d_cnt);
        dfree(d_loss);
        dfree(d_sL);
        dfree(d_slnT);
        dfree(d_fft_tw);
        dfree(d_fft_k);
        fft_n = 0;
        if (copy_s) cudaStreamDestroy(copy_s);
        if (ev_done) cudaEventDestroy(ev_done);
        if (ev_copied) cudaEventDestroy(ev_copied);
        copy_s = nullptr;
        ev_done = ev_copied = nullptr;
        copy_pending = false;
    }

    // Before the device volume or HU image is written again: make `s` wait
    // for the queued asynchronous copy-out of the previous results.
    cudaError_t order_after_copy(cudaStream_t s) const
    {
        return copy_pending ? cudaStreamWaitEvent(s, ev_copied, 0) : cudaSuccess;
    }

    // Host wait for the queued copy-out (before buffers are freed).
    cudaError_t drain_copy()
    {
        if (!copy_pending) return cudaSuccess;
        copy_pending = false;
        return cudaEventSynchronize(ev_copied);
    }
};

namespace {

// Each buffer is allocated on its own, so a call that failed part-way (out
// of memory) leaves the handle consistent and the next call allocates the rest.
int ensure_proj_buffers(fc_handle *h)
{
    const size_t b = h->proj_elems * sizeof(float);
    if (!h->d_T) FC_CK(dev_malloc((void **)&h->d_T, b));
    if (!h->d_tp) FC_CK(dev_malloc((void **)&h->d_tp, b));
    if (!h->d_ts) FC_CK(dev_malloc((void **)&h->d_ts, b));
    if (!h->d_counts) FC_CK(dev_malloc((void **)&h->d_counts, b));
    if (!h->d_hankel) FC_CK(dev_malloc((void **)&h->d_hankel, fc::kBlurTcHankelMax * sizeof(uint16_t)));
    if (!h->d_blur_err) {
        FC_CK(dev_malloc((void **)&h->d_blur_err, sizeof(unsigned int)));
        const cudaError_t e = cudaMemset(h->d_blur_err, 0, sizeof(unsigned int));
        if (e != cudaSuccess) {
            dfree(h->d_blur_err);
            FC_CK(e);
        }
    }
    return FC_OK;
}

// Read and clear the tensor-core blur's timeout word (synchronises `s`).
int check_blur_err(fc_handle *h, cudaStream_t s, const char *fn)
{
    if (!h->d_blur_err) return FC_OK;
    unsigned int e = 0;
    FC_CK(cudaMemcpyAsync(&e, h->d_blur_err, sizeof(e), cudaMemcpyDeviceToHost, s));
    FC_CK(cudaStreamSynchronize(s));
    if (!e) return FC_OK;
    FC_CK(cudaMemsetAsync(h->d_blur_err, 0, sizeof(unsigned int), s));
    return fail(FC_ETIMEOUT, "%s: a detector-blur kernel timed out waiting for its copies or MMAs", fn);
}

int ensure_recon_buffers(fc_handle *h, cudaStream_t s)
{
    if (!h->d_filt) {
        int lo, hi;
        fc::fdk_row_range(h->dg, &lo, &hi);
        h->filt_elems = (size_t)h->g.n_angles * (hi - lo + 1 + 3) * fdk_row_pitch(h->g.n_u);
        FC_CK(dev_malloc((void **)&h->d_filt, h->filt_elems * sizeof(float2)));
        FC_CK(cudaMemsetAsync(h->d_filt, 0, h->filt_elems * sizeof(float2), s));
        h->filt_quad = -1;
    }
    if (!h->d_counts) FC_CK(dev_malloc((void **)&h->d_counts, h->proj_elems * sizeof(float)));
    if (!h->d_vol) FC_CK(dev_malloc((void **)&h->d_vol, h->vol_elems * sizeof(double)));
    if (!h->d_hu) FC_CK(dev_malloc((void **)&h->d_hu, h->vol_elems * sizeof(float)));
    if (!h->d_part) FC_CK(dev_malloc((void **)&h->d_part, 2 * 256 * sizeof(double)));
    return FC_OK;
}

// Before filtering in `quad` layout: the zero padding of one layout is data
// in the other, so a change of layout re-zeroes the buffer.
int filt_layout(fc_handle *h, int quad, cudaStream_t s)
{
    if (h->filt_quad == quad) return FC_OK;
    if (h->filt_quad >= 0) FC_CK(cudaMemsetAsync(h->d_filt, 0, h->filt_elems * sizeof(float2), s));
    h->filt_quad = quad;
    return FC_OK;
}

int copy_out(void *dst, int where, const void *src, size_t bytes, cudaStream_t s)
{
    if (where == FC_DEVICE) {
        FC_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    } else {
        FC_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        FC_CK(cudaStreamSynchronize(s));
    }
    return FC_OK;
}

cudaEvent_t take_event(fc_handle *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records the start event of a traced launch; Trace::end records the stop.
struct Trace {
    fc_handle *h;
    int id, launches;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Trace(fc_handle *h_, int id_, int n_, cudaStream_t s_) : h(h_), id(id_), launches(n_), s(s_)
    {
        if (h->prof && (a = take_event(h))) cudaEventRecord(a, s);
    }
    void end()
    {
        if (!a) return;
        cudaEvent_t b = take_event(h);
        if (!b) {
            h->pool.push_back(a);
            a = nullptr;
            return;
        }
        cudaEventRecord(b, s);
        h->pending.push_back({id, launches, a, b});
        a = nullptr;
    }
    ~Trace()
    {
        if (a) h->pool.push_back(a);
    }
};

int gauss_taps(double sigma, float *taps, int *radius)
{
    if (!(sigma >= 0.0) || sigma > FC_MAX_SIGMA_PX)
        return fail(FC_EINVAL, "blur sigma %g outside [0, %g]", sigma, (double)FC_MAX_SIGMA_PX);
    const int R = sigma > 0.0 ? (int)ceil(4.0 * sigma) : 0;
    double sum = 0.0;
    std::vector<double> g(2 * R + 1);
    for (int j = -R; j <= R; ++j) {
        g[j + R] = R == 0 ? 1.0 : exp(-(double)j * j / (2.0 * sigma * sigma));
        sum += g[j + R];
    }
    for (int j = 0; j < 2 * R + 1; ++j) taps[j] = (float)(g[j] / sum);
    *radius = R;
    return FC_OK;
}

// Detector rows whose rays can meet the voxel slab: a ray through row v lies
// at height z = v * s along the central direction, s = distance from the
// source / SDD; inside the voxel box s >= (SAD - r_max) / SDD.  It can meet the
// slab |z| <= nz dz / 2 only if |v| (SAD - r_max) / SDD <= nz dz / 2.  Two rows
// of margin.
static void hit_band(const fc_geometry &G, int *lo, int *hi)
{
    const double rmax = sqrt(0.25 * G.nx * G.dx_cm * G.nx * G.dx_cm + 0.25 * G.ny * G.dy_cm * G.ny * G.dy_cm);
    const double vmax = 0.5 * G.nz * G.dz_cm * G.sdd_cm / (G.sad_cm - rmax) / G.dv_cm;
    const double cv = 0.5 * (G.n_v - 1);
    *lo = (int)floor(cv - vmax) - 2;
    *hi = (int)ceil(cv + vmax) + 2;
}

// Fraction of the rays of the traced band that meet the voxel box, from a
// sample (8 projections, every 4th column, up to 64 rows) intersected with
// the box in binary64.  It only chooses how the projector assigns rays to
// threads (compacted when most band rays miss); results do not depend on it.
static double band_hit_fraction(const fc_geometry &G)
{
    int lo, hi;
    hit_band(G, &lo, &hi);
    lo = lo < 0 ? 0 : lo;
    hi = hi > G.n_v - 1 ? G.n_v - 1 : hi;
    if (lo > hi) return 1.0;
    const double box[3] = {0.5 * G.nx * G.dx_cm, 0.5 * G.ny * G.dy_cm, 0.5 * G.nz * G.dz_cm};
    const int rstep = (hi - lo + 1 + 63) / 64;
    long long n = 0, hits = 0;
    for (int ka = 0; ka < 8; ++ka) {
        const double th = G.theta0_rad + G.arc_rad * (double)ka / 8.0;
        const double c = cos(th), sn = sin(th);
        const double S[3] = {G.sad_cm * c, G.sad_cm * sn, 0.0};
        for (int iv = lo; iv <= hi; iv += rstep)
            for (int iu = 0; iu < G.n_u; iu += 4) {
                const double u = (iu - 0.5 * (G.n_u - 1)) * G.du_cm, v = (iv - 0.5 * (G.n_v - 1)) * G.dv_cm;
                const double P[3] = {-(G.sdd_cm - G.sad_cm) * c - u * sn, -(G.sdd_cm - G.sad_cm) * sn + u * c, v};
                double t0 = 0.0, t1 = 1.0;
                for (int a = 0; a < 3; ++a) {
                    const double d = P[a] - S[a];
                    if (d == 0.0) {
                        if (S[a] < -box[a] || S[a] >= box[a]) t1 = -1.0;
                        continue;
                    }
                    const double ta = (-box[a] - S[a]) / d, tb = (box[a] - S[a]) / d;
                    t0 = fmax(t0, fmin(ta, tb));
                    t1 = fmin(t1, fmax(ta, tb));
                }
                ++n;
                hits += t1 > t0;
            }
    }
    return n ? (double)hits / (double)n : 1.0;
}

}  // namespace

extern "C" {

const char *fc_last_error(void) { return g_err.c_str(); }

int fc_inject_fault(int kind, int64_t arg)
{
    switch (kind) {
    case FC_FAULT_NONE:
        g_alloc_fail_in.store(-1);
        g_blur_timeout.store(0);
        return FC_OK;
    case FC_FAULT_ALLOC:
        if (arg < 0) return fail(FC_EINVAL, "fc_inject_fault: allocation count %lld < 0", (long long)arg);
        g_alloc_fail_in.store(arg);
        return FC_OK;
    case FC_FAULT_BLUR_TIMEOUT:
        g_blur_timeout.store(1);
        return FC_OK;
    default:
        return fail(FC_EINVAL, "fc_inject_fault: unknown kind %d", kind);
    }
}

int fc_create(fc_handle **out, int device)
{
    if (!out) return fail(FC_EINVAL, "fc_create: null output pointer");
    *out = nullptr;
    int n = 0;
    FC_CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(FC_EINVAL, "fc_create: device %d of %d", device, n);
    DeviceGuard dgd(device);
    if (!dgd.ok) return fail(FC_ECUDA, "fc_create: cannot select device %d", device);
    fc_handle *h = new fc_handle();
    h->device = device;
    if (dev_malloc((void **)&h->d_flag, sizeof(unsigned int)) != cudaSuccess) {
        delete h;
        return fail(FC_ENOMEM, "fc_create: allocation failed");
    }
    *out = h;
    g_err.clear();
    return FC_OK;
}

int fc_destroy(fc_handle *h)
{
    if (!h) return FC_OK;
    DeviceGuard dgd(h->device);
    (void)h->drain_copy();
    h->free_all();
    delete h;
    return FC_OK;
}

int fc_set_geometry(fc_handle *h, const fc_geometry *g)
{
    if (!h || !g) return fail(FC_EINVAL, "fc_set_geometry: null argument");
    if (g->n_u <= 0 || g->n_v <= 0 || g->n_angles <= 0 || g->nx <= 0 || g->ny <= 0 || g->nz <= 0)
        return fail(FC_EINVAL, "fc_set_geometry: sizes must be positive");
    if (!(g->du_cm > 0) || !(g->dv_cm > 0) || !(g->dx_cm > 0) || !(g->dy_cm > 0) || !(g->dz_cm > 0))
        return fail(FC_EINVAL, "fc_set_geometry: pitches must be positive");
    if (!(g->sad_cm > 0) || !(g->sdd_cm > g->sad_cm) || !(g->arc_rad > 0))
        return fail(FC_EINVAL, "fc_set_geometry: need 0 < SAD < SDD and arc > 0");
    if (g->n_u > 8192) return fail(FC_EINVAL, "fc_set_geometry: n_u %d > 8192", g->n_u);
    if (g->n_v > 65535 || g->n_angles > 65535)
        return fail(FC_EINVAL, "fc_set_geometry: n_v and n_angles must be <= 65535");
    const double hx = 0.5 * g->nx * g->dx_cm, hy = 0.5 * g->ny * g->dy_cm;
    const double rmax = sqrt(hx * hx + hy * hy);
    if (rmax >= g->sad_cm || rmax >= g->sdd_cm - g->sad_cm)
        return fail(FC_EINVAL, "fc_set_geometry: volume (radius %g cm) must lie strictly between "
                               "source and detector", rmax);
    const size_t proj = (size_t)g->n_angles * g->n_v * g->n_u;
    const size_t vox = (size_t)g->nx * g->ny * g->nz;
    if (vox >= ((size_t)1 << 31))
        return fail(FC_EINVAL, "fc_set_geometry: %zu voxels exceed the 2^31 index range", vox);
    DeviceGuard dgd(h->device);
    FC_CK(h->drain_copy());   // buffers below may be freed
    const bool same_vol = h->has_geom && h->g.nx == g->nx && h->g.ny == g->ny && h->g.nz == g->nz;
    if (proj != h->proj_elems || !h->has_geom) {
        dfree(h->d_T);
        dfree(h->d_tp);
        dfree(h->d_ts);
        dfree(h->d_counts);
        h->has_counts = false;
    }
    dfree(h->d_filt);  // its size follows the reachable detector rows
    dfree(h->d_fft_tw);   // the filter tables follow n_u and tau
    dfree(h->d_fft_k);
    h->fft_n = 0;
    dfree(h->d_I);
    dfree(h->d_gI);
    dfree(h->d_gT);
    dfree(h->d_gtmp);
    dfree(h->d_gf);
    dfree(h->d_gmu);
    if (vox != h->vol_elems) {
        dfree(h->d_vol);
        dfree(h->d_hu);
    }
    if (!same_vol) {
        dfree(h->d_labels);
        dfree(h->d_labels_zf);
        dfree(h->d_bricks);
        h->has_phantom = false;
    }
    dfree(h->d_trig);
    h->g = *g;
    h->proj_elems = proj;
    h->vol_elems = vox;
    fc::DevGeom &d = h->dg;
    d.sad = (float)g->sad_cm;
    d.sdd = (float)g->sdd_cm;
    d.du = (float)g->du_cm;
    d.dv = (float)g->dv_cm;
    d.cu = (float)(0.5 * (g->n_u - 1));
    d.cv = (float)(0.5 * (g->n_v - 1));
    d.n_u = g->n_u;
    d.n_v = g->n_v;
    d.n_angles = g->n_angles;
    d.nx = g->nx;
    d.ny = g->ny;
    d.nz = g->nz;
    d.dx = (float)g->dx_cm;
    d.dy = (float)g->dy_cm;
    d.dz = (float)g->dz_cm;
    d.lox = (float)(-0.5 * g->nx * g->dx_cm);
    d.loy = (float)(-0.5 * g->ny * g->dy_cm);
    d.loz = (float)(-0.5 * g->nz * g->dz_cm);
    d.idx = (float)(1.0 / g->dx_cm);
    d.idy = (float)(1.0 / g->dy_cm);
    d.idz = (float)(1.0 / g->dz_cm);
    std::vector<float2> trig(g->n_angles);
    for (int k = 0; k < g->n_angles; ++k) {
        const double th = g->theta0_rad + g->arc_rad * (double)k / (double)g->n_angles;
        trig[k] = make_float2((float)cos(th), (float)sin(th));
    }
    FC_CK(dev_malloc((void **)&h->d_trig, sizeof(float2) * g->n_angles));
    FC_CK(cudaMemcpy(h->d_trig, trig.data(), sizeof(float2) * g->n_angles, cudaMemcpyHostToDevice));
    h->band_hit_frac = band_hit_fraction(*g);
    h->has_geom = true;
    return FC_OK;
}

int fc_set_phantom(fc_handle *h, const uint8_t *labels, int n_mat, int where, void *stream)
{
    if (!h || !labels) return fail(FC_EINVAL, "fc_set_phantom: null argument");
    if (!h->has_geom) return fail(FC_ESTATE, "fc_set_phantom: call fc_set_geometry first");
    if (n_mat < 1 || n_mat > FC_MAX_MATERIALS)
        return fail(FC_EINVAL, "fc_set_phantom: n_mat %d outside [1, %d]", n_mat, FC_MAX_MATERIALS);
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_EINVAL, "fc_set_phantom: bad where");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->d_labels) FC_CK(dev_malloc((void **)&h->d_labels, h->vol_elems));
    if (!h->d_labels_zf) FC_CK(dev_malloc((void **)&h->d_labels_zf, h->vol_elems));
    if (!h->d_bricks)
        FC_CK(dev_malloc((void **)&h->d_bricks,
                         (size_t)((h->g.nx + fc::kBrick - 1) / fc::kBrick) *
                             ((h->g.ny + fc::kBrick - 1) / fc::kBrick) *
                             ((h->g.nz + fc::kBrickZ - 1) / fc::kBrickZ)));
    if (where == FC_HOST) {
        // host labels are checked here, before the copy, so the call need
        // not wait for the device (the copy and kernels stay queued on s)
        uint8_t mx = 0;
        for (size_t i = 0; i < h->vol_elems; ++i) mx = labels[i] > mx ? labels[i] : mx;
        if (mx >= n_mat) {
            h->has_phantom = false;
            return fail(FC_EINVAL, "fc_set_phantom: a label is >= n_mat (%d)", n_mat);
        }
    }
    FC_CK(cudaMemcpyAsync(h->d_labels, labels, h->vol_elems,
                          where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    FC_CK(fc::launch_labels_zfast(h->d_labels, h->d_labels_zf, h->g.nx, h->g.ny, h->g.nz, s));
    FC_CK(cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned int), s));
    FC_CK(fc::launch_brick_map(h->d_labels, h->d_bricks, h->g.nx, h->g.ny, h->g.nz, n_mat,
                               h->d_flag, s));
    if (where == FC_DEVICE) {
        // device labels: the brick-map kernel flags a label >= n_mat
        unsigned int bad = 0;
        FC_CK(cudaMemcpyAsync(&bad, h->d_flag, sizeof(bad), cudaMemcpyDeviceToHost, s));
        FC_CK(cudaStreamSynchronize(s));
        if (bad) {
            h->has_phantom = false;
            return fail(FC_EINVAL, "fc_set_phantom: a label is >= n_mat (%d)", n_mat);
        }
    }
    h->phantom_mat = n_mat;
    h->has_phantom = true;
    return FC_OK;
}

int fc_set_spectrum_detector(fc_handle *h, const fc_spectrum_detector *s)
{
    if (!h || !s || !s->w || !s->d || !s->mu) return fail(FC_EINVAL, "fc_set_spectrum_detector: null argument");
    if (s->n_e < 1 || s->n_e > FC_MAX_BINS)
        return fail(FC_EINVAL, "fc_set_spectrum_detector: n_e %d outside [1, %d]", s->n_e, FC_MAX_BINS);
    if (s->n_mat < 1 || s->n_mat > FC_MAX_MATERIALS)
        return fail(FC_EINVAL, "fc_set_spectrum_detector: n_mat %d outside [1, %d]", s->n_mat,
                    FC_MAX_MATERIALS);
    double den = 0.0;
    for (int e = 0; e < s->n_e; ++e) {
        if (!(s->w[e] >= 0) || !(s->d[e] >= 0))
            return fail(FC_EINVAL, "fc_set_spectrum_detector: negative or NaN w/D at bin %d", e);
        for (int m = 0; m < s->n_mat; ++m)
            if (!(s->mu[(size_t)e * s->n_mat + m] >= 0) || !isfinite(s->mu[(size_t)e * s->n_mat + m]))
                return fail(FC_EINVAL, "fc_set_spectrum_detector: bad mu at bin %d material %d", e, m);
        den += s->w[e] * s->d[e];
    }
    if (!(den > 0) || !isfinite(den)) return fail(FC_EINVAL, "fc_set_spectrum_detector: sum w D must be > 0");
    if (!(s->spr >= 0) || !(s->n0 > 0) || !isfinite(s->n0) || !isfinite(s->spr))
        return fail(FC_EINVAL, "fc_set_spectrum_detector: need spr >= 0 and n0 > 0");
    float tmp[fc::kMaxTaps];
    int r;
    int rc = gauss_taps(s->psf_sigma_px, tmp, &r);
    if (rc) return rc;
    rc = gauss_taps(s->scatter_sigma_px, tmp, &r);
    if (rc) return rc;
    h->n_e = s->n_e;
    h->n_groups = 0;   // energy groups refer to the previous spectrum's bins
    h->n_mat = s->n_mat;
    h->wd.assign(s->n_e, 0.0f);
    h->phi.assign(s->n_e, 0.0);
    double wsum = 0.0;
    for (int e = 0; e < s->n_e; ++e) wsum += s->w[e];
    for (int e = 0; e < s->n_e; ++e) h->phi[e] = s->w[e] / wsum;
    h->mu2.assign((size_t)s->n_e * fc::kMaxMat, 0.0f);
    const double log2e = 1.4426950408889634;
    for (int e = 0; e < s->n_e; ++e) {
        h->wd[e] = (float)(s->w[e] * s->d[e] / den);
        for (int m = 0; m < s->n_mat; ++m)
            h->mu2[(size_t)e * fc::kMaxMat + m] = (float)(s->mu[(size_t)e * s->n_mat + m] * log2e);
    }
    h->psf = s->psf_sigma_px;
    h->sc = s->scatter_sigma_px;
    h->spr = s->spr;
    h->n0 = s->n0;
    h->seed = s->seed;
    h->noise = s->noise ? 1 : 0;
    h->has_spec = true;
    return FC_OK;
}

int fc_set_water_roi(fc_handle *h, double radius_cm, double z_margin)
{
    if (!h) return fail(FC_EINVAL, "fc_set_water_roi: null handle");
    if (!(radius_cm > 0) || !(z_margin >= 0) || !(z_margin < 0.5))
        return fail(FC_EINVAL, "fc_set_water_roi: need radius > 0 and 0 <= margin < 0.5");
    h->water_r = radius_cm;
    h->zmargin = z_margin;
    return FC_OK;
}

static int fill_proj_params(fc_handle *h, int a0, int na, fc::ProjParams *p)
{
    if (!h->has_geom || !h->has_phantom || !h->has_spec)
        return fail(FC_ESTATE, "fc_project: geometry, phantom and spectrum must be set");
    if (h->phantom_mat > h->n_mat)
        return fail(FC_EINVAL, "fc_project: phantom has %d materials, attenuation table %d",
                    h->phantom_mat, h->n_mat);
    if (a0 < 0 || na < 0 || a0 + na > h->g.n_angles)
        return fail(FC_EINVAL, "fc_project: angles [%d, %d) outside [0, %d)", a0, a0 + na, h->g.n_angles);
    memset(p, 0, sizeof(*p));
    p->g = h->dg;
    p->trig = h->d_trig;
    p->labels = h->d_labels;
    p->labels_zf = h->d_labels_zf;
    p->bricks = h->d_bricks;
    p->angle0 = a0;
    p->n_angles_launch = na;
    hit_band(h->g, &p->v_hit_lo, &p->v_hit_hi);
    p->compact = h->band_hit_frac < 0.6;
    p->n_mat = h->n_mat;
    p->n_e = h->n_e;
    for (int e = 0; e < h->n_e; ++e) {
        p->wd[e] = h->wd[e];
        for (int m = 0; m < fc::kMaxMat; ++m) p->mu2[e][m] = h->mu2[(size_t)e * fc::kMaxMat + m];
    }
    return FC_OK;
}

// out = n0 (G_psf (x) in + spr G_sc (x) in) over `n` images starting at
// element `off` of the projection buffers: tensor-core row and column passes
// through the handle's intermediates (direct f32 passes for radii beyond the
// tensor-core path); `in` and `out` may alias.
// one_lo, one_hi: when one_hi >= 0, every row of `in` outside [one_lo,
// one_hi) is all ones (the projector's primary on rows that cannot meet the
// voxels); the tensor-core row pass then skips those rows' tiles.
static int blur_params(const fc_handle *h, double psf, double sc, double n0, double spr, fc::BlurParams *b)
{
    memset(b, 0, sizeof(*b));
    b->n_u = h->g.n_u;
    b->n_v = h->g.n_v;
    int rc = gauss_taps(psf, b->gp, &b->rp);
    if (rc) return rc;
    rc = gauss_taps(sc, b->gs, &b->rs);
    if (rc) return rc;
    b->n0 = (float)n0;
    b->spr = (float)spr;
    return FC_OK;
}

// Rows of a blurred image left unwritten because they hold one constant
// (c_hi < 0: every row written).
struct ConstRows {
    int c_lo = 0, c_hi = -1;
    float cst = 0.0f;
};

// cr != nullptr: the output feeds a consumer that takes the constant rows
// from *cr (the noise draw), so the band kernel need not store them.
static int run_blur(fc_handle *h, const float *in, float *out, size_t off, int n, double psf,
                    double sc, double n0, double spr, cudaStream_t s, int one_lo = 0, int one_hi = -1,
                    ConstRows *cr = nullptr)
{
    fc::BlurParams b;
    int rc = blur_params(h, psf, sc, n0, spr, &b);
    if (rc) return rc;
    if (cr) cr->c_hi = -1;
    if (one_hi >= 0 && in != out && fc::blur_band_supported(b, one_lo, one_hi)) {
        // the input differs from 1 on a narrow band of rows only
        if (cr) fc::blur_band_rows(b, one_lo, one_hi, &cr->c_lo, &cr->c_hi, &cr->cst);
        Trace t(h, FC_K_BLUR_BAND, 1, s);
        FC_CK(fc::launch_blur_band(b, in, out, n, one_lo, one_hi, s, cr == nullptr));
        t.end();
        return FC_OK;
    }
    if (!fc::blur_tc_supported(b)) {
        // radii beyond the tensor-core path: direct f32 passes
        if (!fc::blur_rows_fit(b))
            return fail(FC_EINVAL, "fc_project: detector too wide for the row blur (n_u %d)", h->g.n_u);
        if (!fc::blur_cols_fit(b))
            return fail(FC_EINVAL, "fc_project: detector too tall for the column blur (n_v %d)", h->g.n_v);
        {
            Trace t(h, FC_K_BLUR_ROWS, 1, s);
            FC_CK(fc::launch_blur_rows(b, in, h->d_tp + off, h->d_ts + off, n, s));
            t.end();
        }
        {
            Trace t(h, FC_K_BLUR_COLS, 1, s);
            FC_CK(fc::launch_blur_cols(b, h->d_tp + off, h->d_ts + off, out, n, s));
            t.end();
        }
        return FC_OK;
    }
    b.inject_timeout = g_blur_timeout.exchange(0);
    {
        Trace t(h, FC_K_BLUR_ROWS, fc::blur_tc_rows_launches(b, one_lo, one_hi), s);
        FC_CK(fc::launch_blur_tc_rows(b, in, h->d_tp + off, h->d_ts + off, h->d_hankel,
                                      h->d_blur_err, n, s, one_lo, one_hi));
        t.end();
    }
    {
        Trace t(h, FC_K_BLUR_COLS, fc::blur_tc_cols_launches(b, one_lo, one_hi), s);
        FC_CK(fc::launch_blur_tc_cols(b, h->d_tp + off, h->d_ts + off, out, h->d_hankel,
                                      h->d_blur_err, n, s, one_lo, one_hi));
        t.end();
    }
    return FC_OK;
}

// Energy-group model: group primaries (projector), then the scatter profile
// and the per-group blur into the counts buffer.
static int run_groups(fc_handle *h, int a0, int na, cudaStream_t s)
{
    fc::ProjParams p;
    int rc = fill_proj_params(h, a0, na, &p);
    if (rc) return rc;
    const size_t plane_all = h->proj_elems;
    if (!h->d_grp || h->grp_alloc < h->n_groups) {
        dfree(h->d_grp);
        FC_CK(dev_malloc((void **)&h->d_grp, (size_t)h->n_groups * plane_all * sizeof(float)));
        h->grp_alloc = h->n_groups;
    }
    if (!h->d_prof) FC_CK(dev_malloc((void **)&h->d_prof, (size_t)h->g.n_u * sizeof(float)));
    p.n_groups = h->n_groups;
    for (int i = 0, e = 0; i < h->n_groups; ++i) {
        p.grp_end[i] = h->grp_end[i];
        // the binary32 compensated sum the kernel forms for an unattenuated ray
        float sum = 0.0f, comp = 0.0f;
        for (; e < h->grp_end[i]; ++e) {
            const volatile float y = h->wd[e] - comp;
            const volatile float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        p.grp_flood[i] = sum;
    }
    p.grp_stride = plane_all;
    {
        Trace t(h, FC_K_PROJECT, fc::project_launches(p), s);
        FC_CK(fc::launch_project_groups(p, h->d_grp, s));
        t.end();
    }
    fc::GroupParams gp;
    memset(&gp, 0, sizeof(gp));
    gp.n_u = h->g.n_u;
    gp.n_v = h->g.n_v;
    gp.n_groups = h->n_groups;
    gp.grp_stride = plane_all;
    for (int i = 0; i < h->n_groups; ++i) {
        rc = gauss_taps(h->grp_psf[i], gp.taps[i], &gp.r[i]);
        if (rc) return rc;
        gp.amp[i] = (float)h->grp_amp[i];
        gp.a_cm[i] = (float)h->grp_a[i];
        gp.b[i] = (float)h->grp_b[i];
    }
    gp.du = (float)h->g.du_cm;
    gp.cu = 0.5f * (float)(h->g.n_u - 1);
    gp.n0 = (float)h->n0;
    Trace t(h, FC_K_GROUP_BLUR, 2, s);
    FC_CK(fc::launch_group_blur(gp, h->d_grp, h->d_prof, h->d_counts, a0, na, s));
    t.end();
    return FC_OK;
}

int fc_deconvolve_rl(fc_handle *h, int angle_begin, int angle_count, double psf_sigma_px,
                     int n_iter, float *out, int out_where, void *stream)
{
    if (!h) return fail(FC_EINVAL, "fc_deconvolve_rl: null handle");
    if (!h->has_geom || !h->has_counts || !h->d_counts)
        return fail(FC_ESTATE, "fc_deconvolve_rl: no counts in the handle (run fc_project first)");
    if (angle_begin < 0 || angle_count < 0 || angle_begin + angle_count > h->g.n_angles)
        return fail(FC_EINVAL, "fc_deconvolve_rl: angles [%d, %d) outside [0, %d)", angle_begin,
                    angle_begin + angle_count, h->g.n_angles);
    if (!(psf_sigma_px >= 0) || psf_sigma_px > FC_MAX_GROUP_SIGMA_PX)
        return fail(FC_EINVAL, "fc_deconvolve_rl: sigma outside [0, %g]", (double)FC_MAX_GROUP_SIGMA_PX);
    if (n_iter < 0) return fail(FC_EINVAL, "fc_deconvolve_rl: negative iteration count");
    if (out && out_where != FC_HOST && out_where != FC_DEVICE)
        return fail(FC_EINVAL, "fc_deconvolve_rl: bad out_where");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_proj_buffers(h);
    if (rc) return rc;
    fc::RlParams p;
    memset(&p, 0, sizeof(p));
    p.n_u = h->g.n_u;
    p.n_v = h->g.n_v;
    rc = gauss_taps(psf_sigma_px, p.taps, &p.R);
    if (rc) return rc;
    for (int k = 0; k <= p.R; ++k) {
        double c = 0.0;
        for (int j = 0; j < p.R - k; ++j) c += p.taps[j];   // taps j - R < -k
        p.cl[k] = (float)c;
    }
    p.floor_ = 1e-12f;
    if (!h->d_rlnorm)
        FC_CK(dev_malloc((void **)&h->d_rlnorm, (size_t)(h->g.n_u + h->g.n_v) * sizeof(float)));
    const size_t plane = (size_t)h->g.n_v * h->g.n_u;
    const size_t off = (size_t)angle_begin * plane;
    const size_t bytes = (size_t)angle_count * plane * sizeof(float);
    float *res = nullptr;
    {
        Trace t(h, FC_K_DECONV, n_iter + 1, s);
        FC_CK(fc::launch_rl(p, h->d_counts + off, h->d_tp + off, h->d_ts + off, h->d_rlnorm,
                            angle_count, n_iter, &res, s));
        t.end();
    }
    if (res) FC_CK(cudaMemcpyAsync(h->d_counts + off, res, bytes, cudaMemcpyDeviceToDevice, s));
    if (!out || angle_count == 0) return FC_OK;
    return copy_out(out, out_where, h->d_counts + off, bytes, s);
}

int fc_detector_mtf(fc_handle *h, double slit_width_mm, double slit_angle_deg, int oversample,
                    double *freq_per_mm, double *mtf, int n_cap, int *n_out)
{
    if (!h || !freq_per_mm || !mtf || !n_out) return fail(FC_EINVAL, "fc_detector_mtf: null argument");
    if (!h->has_geom || !h->has_spec) return fail(FC_ESTATE, "fc_detector_mtf: geometry and spectrum must be set");
    if (!(slit_width_mm > 0) || !isfinite(slit_width_mm) || !(fabs(slit_angle_deg) < 45.0))
        return fail(FC_EINVAL, "fc_detector_mtf: need slit width > 0 and |angle| < 45 degrees");
    if (oversample < 1 || oversample > 16) return fail(FC_EINVAL, "fc_detector_mtf: oversample outside [1, 16]");
    const int nb = 32 * oversample, nf = nb / 2 + 1;
    if (n_cap < nf) return fail(FC_EINVAL, "fc_detector_mtf: need room for %d frequencies", nf);
    fc::MtfParams p;
    memset(&p, 0, sizeof(p));
    p.n = 192;
    p.pitch = h->g.du_cm;
    p.width = slit_width_mm / 10.0;
    p.ca = cos(slit_angle_deg * M_PI / 180.0);
    p.sa = sin(slit_angle_deg * M_PI / 180.0);
    p.nb = nb;
    p.delta = p.pitch / oversample;
    p.row0 = p.n / 4;
    p.row1 = 3 * p.n / 4;
    // PSF: each group's optical spread weighted by its share of the flood,
    // or the single optical-spread kernel
    const int ng = h->n_groups ? h->n_groups : 1;
    double tot = 0.0;
    int e0 = 0;
    for (int g = 0; g < ng; ++g) {
        const double sigma = h->n_groups ? h->grp_psf[g] : h->psf;
        if (sigma > FC_MAX_GROUP_SIGMA_PX)
            return fail(FC_EINVAL, "fc_detector_mtf: optical spread sigma %g above %g px", sigma,
                        (double)FC_MAX_GROUP_SIGMA_PX);
        const int e1 = h->n_groups ? h->grp_end[g] : h->n_e;
        double c = 0.0;
        for (int e = e0; e < e1; ++e) c += h->wd[e];
        e0 = e1;
        p.wgt[g] = c;
        tot += c;
        const int R = sigma > 0.0 ? (int)ceil(4.0 * sigma) : 0;
        double sum = 0.0;
        for (int j = -R; j <= R; ++j) {
            p.taps[g][j + R] = R == 0 ? 1.0 : exp(-(double)j * j / (2.0 * sigma * sigma));
            sum += p.taps[g][j + R];
        }
        for (int j = 0; j <= 2 * R; ++j) p.taps[g][j] /= sum;
        p.r[g] = R;
    }
    for (int g = 0; g < ng; ++g) p.wgt[g] /= tot;
    p.n_groups = ng;
    DeviceGuard dgd(h->device);
    double *work = nullptr;
    const size_t nwork = 2 * (size_t)p.n * p.n + nb + 2 * (size_t)nf;
    FC_CK(dev_malloc((void **)&work, nwork * sizeof(double)));
    double *fr = work + 2 * (size_t)p.n * p.n + nb, *mt = fr + nf;
    cudaError_t e = fc::launch_mtf(p, work, fr, mt, 0);
    if (e == cudaSuccess) e = cudaMemcpy(freq_per_mm, fr, nf * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(mtf, mt, nf * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(work);
    FC_CK(e);
    *n_out = nf;
    return FC_OK;
}

int fc_set_energy_groups(fc_handle *h, const fc_energy_groups *g)
{
    if (!h || !g) return fail(FC_EINVAL, "fc_set_energy_groups: null argument");
    if (g->n_groups == 0) {
        h->n_groups = 0;
        return FC_OK;
    }
    if (!h->has_spec) return fail(FC_ESTATE, "fc_set_energy_groups: set the spectrum first");
    if (g->n_groups < 0 || g->n_groups > FC_MAX_GROUPS)
        return fail(FC_EINVAL, "fc_set_energy_groups: n_groups %d outside [0, %d]", g->n_groups, FC_MAX_GROUPS);
    if (!g->bin_end || !g->psf_sigma_px || !g->scatter_amp || !g->scatter_a_cm || !g->scatter_b)
        return fail(FC_EINVAL, "fc_set_energy_groups: null array");
    int prev = 0;
    for (int i = 0; i < g->n_groups; ++i) {
        if (g->bin_end[i] <= prev || g->bin_end[i] > h->n_e)
            return fail(FC_EINVAL, "fc_set_energy_groups: bin_end must increase within (0, n_e]");
        prev = g->bin_end[i];
        if (!(g->psf_sigma_px[i] >= 0) || g->psf_sigma_px[i] > FC_MAX_GROUP_SIGMA_PX)
            return fail(FC_EINVAL, "fc_set_energy_groups: group %d sigma outside [0, %g]", i,
                        (double)FC_MAX_GROUP_SIGMA_PX);
        if (!(g->scatter_amp[i] >= 0) || !isfinite(g->scatter_amp[i]) || !(g->scatter_a_cm[i] > 0) ||
            !isfinite(g->scatter_a_cm[i]) || !(g->scatter_b[i] >= 0) || !isfinite(g->scatter_b[i]))
            return fail(FC_EINVAL, "fc_set_energy_groups: bad scatter parameters for group %d", i);
    }
    if (prev != h->n_e) return fail(FC_EINVAL, "fc_set_energy_groups: last bin_end must equal n_e");
    for (int i = 0; i < g->n_groups; ++i) {
        h->grp_end[i] = g->bin_end[i];
        h->grp_psf[i] = g->psf_sigma_px[i];
        h->grp_amp[i] = g->scatter_amp[i];
        h->grp_a[i] = g->scatter_a_cm[i];
        h->grp_b[i] = g->scatter_b[i];
    }
    h->n_groups = g->n_groups;
    return FC_OK;
}

int fc_project(fc_handle *h, int angle_begin, int angle_count, int out_kind, float *out,
               int out_where, void *stream)
{
    if (!h) return fail(FC_EINVAL, "fc_project: null handle");
    if (out_kind < FC_OUT_NONE || out_kind > FC_OUT_COUNTS) return fail(FC_EINVAL, "fc_project: bad out_kind");
    if (out_kind != FC_OUT_NONE && !out) return fail(FC_EINVAL, "fc_project: null output");
    if (out_kind != FC_OUT_NONE && out_where != FC_HOST && out_where != FC_DEVICE)
        return fail(FC_EINVAL, "fc_project: bad out_where");
    fc::ProjParams p;
    int rc = fill_proj_params(h, angle_begin, angle_count, &p);
    if (rc) return rc;
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    rc = ensure_proj_buffers(h);
    if (rc) return rc;
    const size_t plane = (size_t)h->g.n_v * h->g.n_u;
    const size_t off = (size_t)angle_begin * plane;
    const size_t bytes = (size_t)angle_count * plane * sizeof(float);
    // rows outside [v_hit_lo, v_hit_hi] hold T = 1 exactly (their rays cannot
    // meet the voxels)
    const int one_lo = p.v_hit_lo > 0 ? p.v_hit_lo : 0;
    const int one_hi = (p.v_hit_hi < h->g.n_v - 1 ? p.v_hit_hi : h->g.n_v - 1) + 1;
    if (h->n_groups && out_kind != FC_OUT_PRIMARY) {
        if (h->noise_order == FC_NOISE_BEFORE_PSF)
            return fail(FC_EINVAL, "fc_project: noise before the optical spread is not defined for energy groups");
    } else {
        // T = 1 goes to every row when T is returned; otherwise only to the
        // rows the blur reads (it takes the others as 1): none for the band
        // blur, the 64-row tiles around the band for the tensor-core pass
        int f_lo = 0, f_hi = -1;
        if (out_kind != FC_OUT_PRIMARY) {
            fc::BlurParams b;
            rc = blur_params(h, h->noise_order == FC_NOISE_BEFORE_PSF ? 0.0 : h->psf, h->sc, h->n0, h->spr, &b);
            if (rc) return rc;
            if (fc::blur_band_supported(b, one_lo, one_hi)) {
                f_lo = one_lo;
                f_hi = one_hi;
            } else if (fc::blur_tc_supported(b)) {
                fc::blur_tc_rows_read(b, one_lo, one_hi, &f_lo, &f_hi);
            }
        }
        Trace t(h, FC_K_PROJECT, fc::project_launches(p, f_lo, f_hi), s);
        FC_CK(fc::launch_project(p, h->d_T, nullptr, s, f_lo, f_hi));
        t.end();
    }
    if (out_kind == FC_OUT_PRIMARY) return angle_count ? copy_out(out, out_where, h->d_T + off, bytes, s) : FC_OK;
    const bool noise = (out_kind != FC_OUT_INTENSITY) && h->noise;
    if (h->n_groups) {
        rc = run_groups(h, angle_begin, angle_count, s);
        if (rc) return rc;
        if (noise) {
            Trace t(h, FC_K_NOISE, 1, s);
            FC_CK(fc::launch_poisson(h->d_counts + off, h->d_counts + off, angle_count, h->g.n_v,
                                     h->g.n_u, angle_begin, h->seed, s));
            t.end();
        }
        h->has_counts = true;
        if (out_kind == FC_OUT_NONE || angle_count == 0) return FC_OK;
        return copy_out(out, out_where, h->d_counts + off, bytes, s);
    }
    if (h->noise_order == FC_NOISE_BEFORE_PSF) {
        // Sec. II.G order: counts drawn from the scatter-added rate, then the
        // optical spread applied to the counts
        rc = run_blur(h, h->d_T + off, h->d_counts + off, off, angle_count, 0.0, h->sc, h->n0, h->spr, s,
                      one_lo, one_hi);
        if (rc) return rc;
        if (out_kind == FC_OUT_INTENSITY) {
            h->has_counts = true;
            if (!angle_count) return FC_OK;
            rc = copy_out(out, out_where, h->d_counts + off, bytes, s);
            if (rc || out_where != FC_HOST) return rc;
            return check_blur_err(h, s, "fc_project");
        }
        if (noise) {
            Trace t(h, FC_K_NOISE, 1, s);
            FC_CK(fc::launch_poisson(h->d_counts + off, h->d_counts + off, angle_count, h->g.n_v,
                                     h->g.n_u, angle_begin, h->seed, s));
            t.end();
        }
        rc = run_blur(h, h->d_counts + off, h->d_counts + off, off, angle_count, h->psf, 0.0, 1.0, 0.0, s);
        if (rc) return rc;
    } else {
        // with noise the intensity is an intermediate: the band blur leaves
        // its constant rows to the sampler, which takes that rate there
        ConstRows cr;
        rc = run_blur(h, h->d_T + off, h->d_counts + off, off, angle_count, h->psf, h->sc, h->n0, h->spr, s,
                      one_lo, one_hi, noise ? &cr : nullptr);
        if (rc) return rc;
        if (noise) {
            Trace t(h, FC_K_NOISE, 1, s);
            FC_CK(fc::launch_poisson(h->d_counts + off, h->d_counts + off, angle_count, h->g.n_v,
                                     h->g.n_u, angle_begin, h->seed, s, cr.c_lo, cr.c_hi, cr.cst));
            t.end();
        }
    }
    h->has_counts = true;
    if (out_kind == FC_OUT_NONE || angle_count == 0) return FC_OK;
    rc = copy_out(out, out_where, h->d_counts + off, bytes, s);
    if (rc || out_where != FC_HOST) return rc;
    return check_blur_err(h, s, "fc_project");
}

int fc_set_noise_order(fc_handle *h, int order)
{
    if (!h) return fail(FC_EINVAL, "fc_set_noise_order: null handle");
    if (order != FC_NOISE_AFTER_BLUR && order != FC_NOISE_BEFORE_PSF)
        return fail(FC_EINVAL, "fc_set_noise_order: unknown order %d", order);
    h->noise_order = order;
    return FC_OK;
}

int fc_set_backprojector(fc_handle *h, int variant)
{
    if (!h) return fail(FC_EINVAL, "fc_set_backprojector: null handle");
    if (variant < FC_BP_AUTO || variant > FC_BP_CHUNKED_SYM)
        return fail(FC_EINVAL, "fc_set_backprojector: unknown variant %d", variant);
    h->bp_request = variant;
    return FC_OK;
}

// Projections per half / quarter turn of a full-circle scan (0 when the
// scan is not a full circle or n_angles is not divisible by 2 / 4).
// Whether a quarter turn about the axis maps the voxel grid onto itself.
static bool g_sym_quarter_ok(const fc_geometry &g)
{
    return g.nx == g.ny && g.nx % 2 == 0 && g.dx_cm == g.dy_cm;
}

static int fdk_sym_turn(const fc_geometry &g, int parts)
{
    const double two_pi = 2.0 * M_PI;
    if (g.n_angles < parts || g.n_angles % parts != 0) return 0;
    if (!(fabs(g.arc_rad - two_pi) <= 1e-12 * two_pi)) return 0;
    return g.n_angles / parts;
}

// The FFT ramp filter's tables for the handle's geometry (built on first
// use after fc_set_geometry), pointed to by p.
static int ensure_fft_tables(fc_handle *h, fc::FdkParams *p)
{
    p->fft_log2 = fc::fdk_fft_log2(h->g.n_u);
    if (!h->d_fft_k || h->fft_n != h->g.n_u) {
        std::vector<float2> tw;
        std::vector<float> kbr;
        fc::fdk_fft_tables(h->g.n_u, h->g.du_cm * h->g.sad_cm / h->g.sdd_cm, &tw, &kbr);
        dfree(h->d_fft_tw);
        dfree(h->d_fft_k);
        h->fft_n = 0;
        FC_CK(dev_malloc((void **)&h->d_fft_tw, tw.size() * sizeof(float2)));
        FC_CK(dev_malloc((void **)&h->d_fft_k, kbr.size() * sizeof(float)));
        FC_CK(cudaMemcpy(h->d_fft_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
        FC_CK(cudaMemcpy(h->d_fft_k, kbr.data(), kbr.size() * sizeof(float), cudaMemcpyHostToDevice));
        h->fft_n = h->g.n_u;
    }
    p->fft_tw = h->d_fft_tw;
    p->fft_k = h->d_fft_k;
    return FC_OK;
}

// FdkParams of the handle's geometry (no buffers touched).
static void fill_fdk_params(const fc_handle *h, fc::FdkParams *p)
{
    memset(p, 0, sizeof(*p));
    p->g = h->dg;
    p->trig = h->d_trig;
    p->log_flood = (float)log(h->n_groups ? h->n0 : h->n0 * (1.0 + h->spr));
    p->tau = (float)(h->g.du_cm * h->g.sad_cm / h->g.sdd_cm);
    p->mag = (float)(h->g.sad_cm / h->g.sdd_cm);
    p->scale = h->g.arc_rad / (2.0 * h->g.n_angles);
    fc::fdk_row_range(h->dg, &p->v_lo, &p->v_hi);
    p->pw = fdk_row_pitch(h->g.n_u);
    p->ph = p->v_hi - p->v_lo + 1 + 3;
    p->sym_quarter = g_sym_quarter_ok(h->g) ? fdk_sym_turn(h->g, 4) : 0;
}

int fc_backprojector_in_use(fc_handle *h, int *variant)
{
    if (!h || !variant) return fail(FC_EINVAL, "fc_backprojector_in_use: null argument");
    if (!h->has_geom) return fail(FC_ESTATE, "fc_backprojector_in_use: geometry not set");
    DeviceGuard dgd(h->device);
    fc::FdkParams p;
    fill_fdk_params(h, &p);
    *variant = fc::backproject_variant(p, h->bp_request);
    if (*variant < 0)
        return fail(FC_EINVAL, "fc_backprojector_in_use: variant %d does not apply to this geometry",
                    h->bp_request);
    return FC_OK;
}

int fc_project_lengths(fc_handle *h, int angle_begin, int angle_count, float *L, void *stream)
{
    if (!h || !L) return fail(FC_EINVAL, "fc_project_lengths: null argument");
    fc::ProjParams p;
    int rc = fill_proj_params(h, angle_begin, angle_count, &p);
    if (rc) return rc;
    DeviceGuard dgd(h->device);
    Trace t(h, FC_K_LENGTHS, 1, (cudaStream_t)stream);
    FC_CK(fc::launch_project(p, nullptr, L, (cudaStream_t)stream));
    t.end();
    return FC_OK;
}

int fc_dose_estimate(fc_handle *h, int angle_begin, int angle_count, const double *e_kev,
                     const double *muen_over_mu, const double *rho, double *d0, double *dp,
                     int out_where, void *stream)
{
    if (!h || !e_kev || !muen_over_mu || !rho || !d0 || !dp)
        return fail(FC_EINVAL, "fc_dose_estimate: null argument");
    if (out_where != FC_HOST && out_where != FC_DEVICE)
        return fail(FC_EINVAL, "fc_dose_estimate: bad out_where");
    fc::ProjParams p;
    int rc = fill_proj_params(h, angle_begin, angle_count, &p);
    if (rc) return rc;
    if (angle_count < 1) return fail(FC_EINVAL, "fc_dose_estimate: need at least one projection");
    fc::DoseParams d;
    memset(&d, 0, sizeof(d));
    d.n_e = h->n_e;
    d.n_mat = h->n_mat;
    for (int e = 0; e < h->n_e; ++e) {
        if (!(e_kev[e] > 0) || !isfinite(e_kev[e]))
            return fail(FC_EINVAL, "fc_dose_estimate: bin energy %d must be > 0", e);
        if (!(muen_over_mu[e] >= 0) || !(muen_over_mu[e] <= 1))
            return fail(FC_EINVAL, "fc_dose_estimate: mu_en/mu at bin %d outside [0, 1]", e);
        d.e_kev[e] = e_kev[e];
        d.muen[e] = muen_over_mu[e];
        d.phi[e] = h->phi[e];
    }
    for (int m = 0; m < h->n_mat; ++m) {
        if (!(rho[m] > 0) || !isfinite(rho[m]))
            return fail(FC_EINVAL, "fc_dose_estimate: density of material %d must be > 0", m);
        d.rho[m] = rho[m];
    }
    DeviceGuard dgd(h->device);
    d.n_part = fc::dose_blocks(p);
    d.n_rays = (double)angle_count * h->g.n_u * h->g.n_v;
    d.voxel_cm3 = h->g.dx_cm * h->g.dy_cm * h->g.dz_cm;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n_part = (size_t)fc::kDoseBlocks * fc::kMaxBins, n_out = fc::kMaxBins + 1;
    if (!h->d_dose)
        FC_CK(dev_malloc((void **)&h->d_dose, (n_part + n_out + fc::kMaxMat) * sizeof(double)));
    double *part = h->d_dose, *res = h->d_dose + n_part;
    auto *count = reinterpret_cast<unsigned long long *>(res + n_out);
    {
        Trace t(h, FC_K_DOSE, 4, s);   // label count, partials, fold, final
        FC_CK(fc::launch_dose(p, d, part, count, res, s));
        t.end();
    }
    if (out_where == FC_DEVICE) {
        FC_CK(cudaMemcpyAsync(d0, res, h->n_e * sizeof(double), cudaMemcpyDeviceToDevice, s));
        FC_CK(cudaMemcpyAsync(dp, res + h->n_e, sizeof(double), cudaMemcpyDeviceToDevice, s));
        return FC_OK;
    }
    FC_CK(cudaMemcpyAsync(d0, res, h->n_e * sizeof(double), cudaMemcpyDeviceToHost, s));
    FC_CK(cudaMemcpyAsync(dp, res + h->n_e, sizeof(double), cudaMemcpyDeviceToHost, s));
    FC_CK(cudaStreamSynchronize(s));
    return FC_OK;
}

int fc_fluence_for_dose(const fc_handle *h, double dose_gy, double dp_gy, double *n0)
{
    if (!h || !n0) return fail(FC_EINVAL, "fc_fluence_for_dose: null argument");
    if (!h->has_geom) return fail(FC_ESTATE, "fc_fluence_for_dose: geometry not set");
    if (!(dose_gy >= 0) || !(dp_gy > 0) || !isfinite(dose_gy) || !isfinite(dp_gy))
        return fail(FC_EINVAL, "fc_fluence_for_dose: need dose >= 0 and dose per particle > 0");
    // N_gamma = dose / Dp particles spread over the A / A_p = n_u n_v pixels
    *n0 = dose_gy / dp_gy / ((double)h->g.n_u * h->g.n_v);
    return FC_OK;
}

int fc_reconstruct(fc_handle *h, const float *counts, int counts_where, double *vol_mu,
                   float *vol_hu, int out_where, void *stream)
{
    if (!h) return fail(FC_EINVAL, "fc_reconstruct: null handle");
    if (!h->has_geom || !h->has_spec)
        return fail(FC_ESTATE, "fc_reconstruct: geometry and spectrum/detector must be set");
    if (!counts && !h->has_counts) return fail(FC_ESTATE, "fc_reconstruct: no counts simulated yet");
    if (counts && counts_where != FC_HOST && counts_where != FC_DEVICE)
        return fail(FC_EINVAL, "fc_reconstruct: bad counts_where");
    if ((vol_mu || vol_hu) && out_where != FC_HOST && out_where != FC_DEVICE && out_where != FC_HOST_ASYNC)
        return fail(FC_EINVAL, "fc_reconstruct: bad out_where");
    DeviceGuard dgd(h->device);
    if (out_where == FC_HOST_ASYNC) {
        // the asynchronous copy needs page-locked host memory
        for (const void *ptr : {(const void *)vol_mu, (const void *)vol_hu}) {
            if (!ptr) continue;
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess || a.type != cudaMemoryTypeHost) {
                cudaGetLastError();
                return fail(FC_EINVAL, "fc_reconstruct: FC_HOST_ASYNC needs page-locked host memory");
            }
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_recon_buffers(h, s);
    if (rc) return rc;
    const size_t pbytes = h->proj_elems * sizeof(float);
    const float *src = h->d_counts;
    if (counts && counts_where == FC_DEVICE) {
        src = counts;
    } else if (counts) {
        FC_CK(cudaMemcpyAsync(h->d_counts, counts, pbytes, cudaMemcpyHostToDevice, s));
        h->has_counts = true;
    }
    fc::FdkParams p;
    // flood: T = 1 through the detector model (single kernel: N0 (1 + SPR);
    // energy groups: N0, the scatter profile needing a phantom)
    fill_fdk_params(h, &p);
    rc = ensure_fft_tables(h, &p);
    if (rc) return rc;
    const int bpv = fc::backproject_variant(p, h->bp_request);
    if (bpv < 0)
        return fail(FC_EINVAL, "fc_reconstruct: backprojector variant %d does not apply to this geometry",
                    h->bp_request);
    p.filt_quad = fc::backproject_reads_quad(p, bpv) ? 1 : 0;
    rc = filt_layout(h, p.filt_quad, s);
    if (rc) return rc;
    {
        Trace t(h, FC_K_FDK_FILTER, 1, s);
        FC_CK(fc::launch_fdk_filter(p, src, h->d_filt, s));
        t.end();
    }
    {
        // the previous results may still be on their way to the host
        FC_CK(h->order_after_copy(s));
        Trace t(h, FC_K_BACKPROJECT, 1, s);
        FC_CK(fc::launch_backproject(p, h->d_filt, h->d_vol, bpv, s));
        t.end();
    }
    if (vol_hu) {
        const int zcut = (int)floor(h->g.nz * h->zmargin);
        const int zc = (h->g.nz > 2 * zcut) ? zcut : 0;
        Trace t(h, FC_K_HU, 2, s);
        FC_CK(fc::launch_hu(h->dg, h->d_vol, h->d_hu, h->d_part, (float)h->water_r, zc, s));
        t.end();
    }
    if ((vol_mu || vol_hu) && out_where == FC_HOST_ASYNC) {
        if (!h->copy_s) FC_CK(cudaStreamCreateWithFlags(&h->copy_s, cudaStreamNonBlocking));
        if (!h->ev_done) FC_CK(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
        if (!h->ev_copied) FC_CK(cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming));
        FC_CK(cudaEventRecord(h->ev_done, s));
        FC_CK(cudaStreamWaitEvent(h->copy_s, h->ev_done, 0));
        if (vol_mu)
            FC_CK(cudaMemcpyAsync(vol_mu, h->d_vol, h->vol_elems * sizeof(double), cudaMemcpyDeviceToHost,
                                  h->copy_s));
        if (vol_hu)
            FC_CK(cudaMemcpyAsync(vol_hu, h->d_hu, h->vol_elems * sizeof(float), cudaMemcpyDeviceToHost,
                                  h->copy_s));
        FC_CK(cudaEventRecord(h->ev_copied, h->copy_s));
        h->copy_pending = true;
        return FC_OK;
    }
    if (vol_mu) {
        rc = copy_out(vol_mu, out_where, h->d_vol, h->vol_elems * sizeof(double), s);
        if (rc) return rc;
    }
    if (vol_hu) {
        rc = copy_out(vol_hu, out_where, h->d_hu, h->vol_elems * sizeof(float), s);
        if (rc) return rc;
    }
    if ((vol_mu || vol_hu) && out_where == FC_HOST) return check_blur_err(h, s, "fc_reconstruct");
    return FC_OK;
}

int fc_wait_outputs(fc_handle *h)
{
    if (!h) return fail(FC_EINVAL, "fc_wait_outputs: null handle");
    if (!h->copy_pending) return FC_OK;
    DeviceGuard dgd(h->device);
    FC_CK(h->drain_copy());
    return check_blur_err(h, h->copy_s, "fc_wait_outputs");
}

int fc_profile_enable(fc_handle *h, int enable)
{
    if (!h) return fail(FC_EINVAL, "fc_profile_enable: null handle");
    DeviceGuard dgd(h->device);
    for (auto &r : h->pending) {
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->pending.clear();
    for (int i = 0; i < FC_K_COUNT; ++i) {
        h->prof_ms[i] = 0.0;
        h->prof_n[i] = 0;
    }
    h->prof = enable != 0;
    return FC_OK;
}

int fc_profile_read(fc_handle *h, double *ms, int64_t *launches)
{
    if (!h) return fail(FC_EINVAL, "fc_profile_read: null handle");
    DeviceGuard dgd(h->device);
    for (auto &r : h->pending) {
        FC_CK(cudaEventSynchronize(r.b));
        float t = 0.0f;
        FC_CK(cudaEventElapsedTime(&t, r.a, r.b));
        h->prof_ms[r.id] += t;
        h->prof_n[r.id] += r.launches;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->pending.clear();
    for (int i = 0; i < FC_K_COUNT; ++i) {
        if (ms) ms[i] = h->prof_ms[i];
        if (launches) launches[i] = h->prof_n[i];
        h->prof_ms[i] = 0.0;
        h->prof_n[i] = 0;
    }
    return FC_OK;
}

static_assert(fc::kMlpParams == FC_SURROGATE_PARAMS, "surrogate parameter count");
static_assert(fc::kMlpPacked + 2 * fc::kMlpParams + 1 == FC_SURROGATE_STATE, "surrogate state size");

static void fill_sur_params(fc_handle *h, fc::SurrogateParams *p)
{
    memset(p, 0, sizeof(*p));
    p->W1b = h->d_W1b;
    p->W2b = h->d_W2b;
    p->W3b = h->d_W3b;
    p->W2Tb = h->d_W2Tb;
    p->W3Tb = h->d_W3Tb;
    p->P = h->d_P;
    p->n_mat = h->n_mat;
    p->n_e = h->n_e;
    p->guard = (float)h->sur_guard;
    for (int e = 0; e < h->n_e; ++e) {
        p->wd[e] = h->wd[e];
        for (int m = 0; m < fc::kMaxMat; ++m) p->mu2[e][m] = h->mu2[(size_t)e * fc::kMaxMat + m];
    }
}

// Upload a packed parameter vector and rebuild the bf16 operand copies.
static int sur_upload(fc_handle *h, const float *packed)
{
    using fc::kMlpHidden;
    const int H = kMlpHidden;
    std::vector<__nv_bfloat16> w1((size_t)H * 16), w2((size_t)H * H), w3((size_t)H * H),
        w2t((size_t)H * H), w3t((size_t)H * H);
    for (int o = 0; o < H; ++o)
        for (int i = 0; i < 16; ++i)
            w1[(size_t)o * 16 + i] = __float2bfloat16(packed[fc::kOffW1 + o * fc::kMlpIn + i % fc::kMlpIn]);
    for (int o = 0; o < H; ++o)
        for (int i = 0; i < H; ++i) {
            w2[(size_t)o * H + i] = w2t[(size_t)i * H + o] = __float2bfloat16(packed[fc::kOffW2 + o * H + i]);
            w3[(size_t)o * H + i] = w3t[(size_t)i * H + o] = __float2bfloat16(packed[fc::kOffW3 + o * H + i]);
        }
    FC_CK(cudaMemcpy(h->d_P, packed, sizeof(float) * fc::kMlpPacked, cudaMemcpyHostToDevice));
    FC_CK(cudaMemcpy(h->d_W1b, w1.data(), w1.size() * 2, cudaMemcpyHostToDevice));
    FC_CK(cudaMemcpy(h->d_W2b, w2.data(), w2.size() * 2, cudaMemcpyHostToDevice));
    FC_CK(cudaMemcpy(h->d_W3b, w3.data(), w3.size() * 2, cudaMemcpyHostToDevice));
    FC_CK(cudaMemcpy(h->d_W2Tb, w2t.data(), w2t.size() * 2, cudaMemcpyHostToDevice));
    FC_CK(cudaMemcpy(h->d_W3Tb, w3t.data(), w3t.size() * 2, cudaMemcpyHostToDevice));
    return FC_OK;
}

static int sur_alloc(fc_handle *h)
{
    const int H = fc::kMlpHidden;
    if (!h->d_P) FC_CK(dev_malloc((void **)&h->d_P, sizeof(float) * fc::kMlpPacked));
    if (!h->d_m1) FC_CK(dev_malloc((void **)&h->d_m1, sizeof(float) * fc::kMlpParams));
    if (!h->d_m2) FC_CK(dev_malloc((void **)&h->d_m2, sizeof(float) * fc::kMlpParams));
    if (!h->d_grad) FC_CK(dev_malloc((void **)&h->d_grad, sizeof(float) * fc::kMlpParams));
    if (!h->d_W1b) FC_CK(dev_malloc((void **)&h->d_W1b, 2 * H * 16));
    if (!h->d_W2b) FC_CK(dev_malloc((void **)&h->d_W2b, 2 * H * H));
    if (!h->d_W3b) FC_CK(dev_malloc((void **)&h->d_W3b, 2 * H * H));
    if (!h->d_W2Tb) FC_CK(dev_malloc((void **)&h->d_W2Tb, 2 * H * H));
    if (!h->d_W3Tb) FC_CK(dev_malloc((void **)&h->d_W3Tb, 2 * H * H));
    if (!h->d_cnt) FC_CK(dev_malloc((void **)&h->d_cnt, sizeof(unsigned int) * 16));
    if (!h->d_err) {
        FC_CK(dev_malloc((void **)&h->d_err, sizeof(int)));
        const cudaError_t e = cudaMemset(h->d_err, 0, sizeof(int));
        if (e != cudaSuccess) {
            dfree(h->d_err);
            FC_CK(e);
        }
    }
    return FC_OK;
}

static uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int fc_surrogate_init(fc_handle *h, uint64_t seed)
{
    if (!h) return fail(FC_EINVAL, "fc_surrogate_init: null handle");
    if (!h->has_spec) return fail(FC_ESTATE, "fc_surrogate_init: set the spectrum first");
    DeviceGuard dgd(h->device);
    int rc = sur_alloc(h);
    if (rc) return rc;
    const int H = fc::kMlpHidden;
    std::vector<float> P(fc::kMlpPacked, 0.0f);
    uint64_t st = seed;
    auto unif = [&](double a) {
        return (float)(a * (2.0 * ((splitmix64(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    };
    for (int i = 0; i < H * fc::kMlpIn; ++i) P[fc::kOffW1 + i] = unif(sqrt(3.0 / fc::kMlpIn));
    for (int i = 0; i < H * H; ++i) P[fc::kOffW2 + i] = unif(sqrt(3.0 / H));
    for (int i = 0; i < H * H; ++i) P[fc::kOffW3 + i] = unif(sqrt(3.0 / H));
    for (int i = 0; i < H; ++i) P[fc::kOffW4 + i] = unif(0.1 * sqrt(3.0 / H));
    // Spectral groups: consecutive energy bins split where the cumulative
    // weight w D crosses 1/4, 1/2, 3/4; each group keeps its total weight and
    // its weight-averaged attenuation.
    const double log2e = 1.4426950408889634;
    double tot = 0.0;
    for (int e = 0; e < h->n_e; ++e) tot += h->wd[e];
    double ga[fc::kMlpGroups] = {0}, gm[fc::kMlpGroups][fc::kMaxMat] = {{0}};
    double cum = 0.0;
    for (int e = 0; e < h->n_e; ++e) {
        const double mid = (cum + 0.5 * h->wd[e]) / tot;
        cum += h->wd[e];
        int k = (int)(mid * fc::kMlpGroups);
        k = k < 0 ? 0 : (k >= fc::kMlpGroups ? fc::kMlpGroups - 1 : k);
        ga[k] += h->wd[e];
        for (int m = 0; m < fc::kMaxMat; ++m)
            gm[k][m] += (double)h->wd[e] * h->mu2[(size_t)e * fc::kMaxMat + m] / log2e;
    }
    for (int k = 0; k < fc::kMlpGroups; ++k) {
        P[fc::kOffGa + k] = (float)(ga[k] / tot);
        for (int m = 0; m < fc::kMaxMat; ++m)
            P[fc::kOffGmu + k * fc::kMaxMat + m] = ga[k] > 0.0 ? (float)(gm[k][m] / ga[k]) : 0.0f;
    }
    for (int m = 0; m < fc::kMaxMat; ++m) {
        P[fc::kOffScale + m] = 1.0f;
        P[fc::kOffBox + m] = INFINITY;
    }
    rc = sur_upload(h, P.data());
    if (rc) return rc;
    FC_CK(cudaMemset(h->d_m1, 0, sizeof(float) * fc::kMlpParams));
    FC_CK(cudaMemset(h->d_m2, 0, sizeof(float) * fc::kMlpParams));
    h->sur_step = 0;
    h->has_sur = true;
    h->sur_fitted = false;
    return FC_OK;
}

static int sur_work(fc_handle *h, int B)
{
    if (h->work_mem && h->work_B == B) return FC_OK;
    if (h->work_mem) cudaFree(h->work_mem);
    h->work_mem = nullptr;
    const int H = fc::kMlpHidden;
    const int n_chunks = (B + fc::kWgradChunk - 1) / fc::kWgradChunk;
    const size_t nb = (size_t)B;
    const size_t bytes = 2 * (16 * nb + 6 * (size_t)H * nb + 16 * nb) +
                         4 * (4 * (size_t)n_chunks * H * H + 4 * (size_t)n_chunks * H + n_chunks) +
                         16 * 256;  // each of the 11 pieces is rounded up to 256 bytes
    FC_CK(dev_malloc((void **)&h->work_mem, bytes));
    FC_CK(cudaMemset(h->work_mem, 0, bytes));
    char *q = (char *)h->work_mem;
    auto take = [&](size_t b) { char *r = q; q += (b + 255) / 256 * 256; return r; };
    fc::MlpWork &w = h->work;
    w.xt = (__nv_bfloat16 *)take(2 * 16 * nb);
    w.h1t = (__nv_bfloat16 *)take(2 * H * nb);
    w.h2t = (__nv_bfloat16 *)take(2 * H * nb);
    w.h3t = (__nv_bfloat16 *)take(2 * H * nb);
    w.dz1t = (__nv_bfloat16 *)take(2 * H * nb);
    w.dz2t = (__nv_bfloat16 *)take(2 * H * nb);
    w.dz3t = (__nv_bfloat16 *)take(2 * H * nb);
    w.g = (__nv_bfloat16 *)take(2 * 16 * nb);
    w.part = (float *)take(4 * 4 * (size_t)n_chunks * H * H);
    w.rsum = (float *)take(4 * 4 * (size_t)n_chunks * H);
    w.gsum = (float *)take(4 * (size_t)n_chunks);
    h->work_B = B;
    return FC_OK;
}

static int sur_check_data(fc_handle *h, const char *fn, const float *L, const float *y,
                          bool need_y, int64_t n)
{
    if (!h) return fail(FC_EINVAL, "%s: null handle", fn);
    if (!L || (need_y && !y)) return fail(FC_EINVAL, "%s: null data", fn);
    if (n <= 0) return fail(FC_EINVAL, "%s: n must be positive", fn);
    if (!h->has_sur) return fail(FC_ESTATE, "%s: call fc_surrogate_init first", fn);
    return FC_OK;
}

// Per-material maximum of the training path lengths -> input scale and the
// box outside which evaluation falls back to the exact sum (first fit only).
static int sur_fit_box(fc_handle *h, const float *L, int64_t n, cudaStream_t s)
{
    if (h->sur_fitted) return FC_OK;
    FC_CK(cudaMemsetAsync(h->d_cnt, 0, sizeof(unsigned int) * 16, s));
    FC_CK(fc::launch_mlp_lmax(L, n, h->n_mat, h->d_cnt, s));
    unsigned int mx[fc::kMaxMat] = {0};
    FC_CK(cudaMemcpyAsync(mx, h->d_cnt, sizeof(mx), cudaMemcpyDeviceToHost, s));
    FC_CK(cudaStreamSynchronize(s));
    float tail[2 * fc::kMaxMat];
    for (int m = 0; m < fc::kMaxMat; ++m) {
        float v;
        memcpy(&v, &mx[m], 4);
        if (m >= h->n_mat) v = 0.0f;
        tail[m] = (float)(1.0 / (v > 1e-3f ? v : 1e-3f));         // scale
        tail[fc::kMaxMat + m] = m < h->n_mat ? v : 0.0f;           // box
    }
    FC_CK(cudaMemcpyAsync(h->d_P + fc::kOffScale, tail, sizeof(float) * fc::kMaxMat,
                          cudaMemcpyHostToDevice, s));
    FC_CK(cudaMemcpyAsync(h->d_P + fc::kOffBox, tail + fc::kMaxMat, sizeof(float) * fc::kMaxMat,
                          cudaMemcpyHostToDevice, s));
    FC_CK(cudaStreamSynchronize(s));
    h->sur_fitted = true;
    return FC_OK;
}

static int sur_read_err(fc_handle *h, cudaStream_t s, const char *fn)
{
    int err = 0;
    FC_CK(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FC_CK(cudaStreamSynchronize(s));
    if (err) {
        FC_CK(cudaMemset(h->d_err, 0, sizeof(int)));
        return fail(FC_ETIMEOUT, "%s: a tensor-core wait exceeded its bound", fn);
    }
    return FC_OK;
}

int fc_surrogate_train(fc_handle *h, const float *L, const float *lnT, int64_t n, int steps,
                       int batch, float lr, uint64_t seed, float *loss_hist, void *stream)
{
    int rc = sur_check_data(h, "fc_surrogate_train", L, lnT, true, n);
    if (rc) return rc;
    if (steps < 0 || batch <= 0 || batch % 128 != 0 || !(lr > 0.0f))
        return fail(FC_EINVAL, "fc_surrogate_train: need steps >= 0, batch a positive multiple of 128, lr > 0");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    rc = sur_fit_box(h, L, n, s);
    if (rc) return rc;
    rc = sur_work(h, batch);
    if (rc) return rc;
    if (h->loss_cap < steps || !h->d_loss) {
        dfree(h->d_loss);
        h->loss_cap = 0;
        FC_CK(dev_malloc((void **)&h->d_loss, sizeof(float) * (steps > 0 ? steps : 1)));
        h->loss_cap = steps;
    }
    if (steps > 0) FC_CK(cudaMemsetAsync(h->d_loss, 0, sizeof(float) * steps, s));
    fc::SurrogateParams p;
    fill_sur_params(h, &p);
    Trace t(h, FC_K_SURROGATE_TRAIN, 4 * steps, s);
    for (int k = 0; k < steps; ++k) {
        const int tglob = ++h->sur_step;
        const float lr_k = (float)(lr * 0.5 * (1.0 + cos(M_PI * k / (double)steps)));
        const float bc1 = (float)(1.0 - pow(0.9, tglob)), bc2 = (float)(1.0 - pow(0.999, tglob));
        FC_CK(fc::launch_mlp_step(p, L, lnT, n, batch, 1, seed, tglob, h->work, h->d_loss + k,
                                  h->d_err, h->d_P, h->d_m1, h->d_m2, lr_k, bc1, bc2, nullptr,
                                  h->d_W1b, h->d_W2b, h->d_W3b, h->d_W2Tb, h->d_W3Tb, s));
    }
    t.end();
    rc = sur_read_err(h, s, "fc_surrogate_train");
    if (rc) return rc;
    if (loss_hist && steps > 0) {
        FC_CK(cudaMemcpyAsync(loss_hist, h->d_loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
        FC_CK(cudaStreamSynchronize(s));
        for (int k = 0; k < steps; ++k) loss_hist[k] /= (float)batch;
    }
    return FC_OK;
}

int fc_surrogate_grad(fc_handle *h, const float *L, const float *lnT, int64_t n, float *grad,
                      float *loss, void *stream)
{
    int rc = sur_check_data(h, "fc_surrogate_grad", L, lnT, true, n);
    if (rc) return rc;
    if (!grad || n % 8 != 0 || n > (1 << 24))
        return fail(FC_EINVAL, "fc_surrogate_grad: need grad and n a multiple of 8 (<= 2^24)");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    rc = sur_work(h, (int)n);
    if (rc) return rc;
    if (h->loss_cap < 1 || !h->d_loss) {
        dfree(h->d_loss);
        h->loss_cap = 0;
        FC_CK(dev_malloc((void **)&h->d_loss, sizeof(float)));
        h->loss_cap = 1;
    }
    FC_CK(cudaMemsetAsync(h->d_loss, 0, sizeof(float), s));
    fc::SurrogateParams p;
    fill_sur_params(h, &p);
    FC_CK(fc::launch_mlp_step(p, L, lnT, n, (int)n, 0, 0, 0, h->work, h->d_loss, h->d_err, h->d_P,
                              h->d_m1, h->d_m2, 0.0f, 1.0f, 1.0f, h->d_grad, h->d_W1b, h->d_W2b,
                              h->d_W3b, h->d_W2Tb, h->d_W3Tb, s));
    FC_CK(cudaMemcpyAsync(grad, h->d_grad, sizeof(float) * fc::kMlpParams, cudaMemcpyDeviceToHost, s));
    if (loss) FC_CK(cudaMemcpyAsync(loss, h->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    FC_CK(cudaStreamSynchronize(s));
    if (loss) *loss /= (float)n;
    return sur_read_err(h, s, "fc_surrogate_grad");
}

int fc_surrogate_get(fc_handle *h, float *state)
{
    if (!h || !state) return fail(FC_EINVAL, "fc_surrogate_get: null argument");
    if (!h->has_sur) return fail(FC_ESTATE, "fc_surrogate_get: no surrogate");
    DeviceGuard dgd(h->device);
    FC_CK(cudaMemcpy(state, h->d_P, sizeof(float) * fc::kMlpPacked, cudaMemcpyDeviceToHost));
    FC_CK(cudaMemcpy(state + fc::kMlpPacked, h->d_m1, sizeof(float) * fc::kMlpParams, cudaMemcpyDeviceToHost));
    FC_CK(cudaMemcpy(state + fc::kMlpPacked + fc::kMlpParams, h->d_m2, sizeof(float) * fc::kMlpParams,
                     cudaMemcpyDeviceToHost));
    state[fc::kMlpPacked + 2 * fc::kMlpParams] = (float)h->sur_step;
    return FC_OK;
}

int fc_surrogate_set(fc_handle *h, const float *state)
{
    if (!h || !state) return fail(FC_EINVAL, "fc_surrogate_set: null argument");
    if (!h->has_spec) return fail(FC_ESTATE, "fc_surrogate_set: set the spectrum first");
    DeviceGuard dgd(h->device);
    int rc = sur_alloc(h);
    if (rc) return rc;
    rc = sur_upload(h, state);
    if (rc) return rc;
    FC_CK(cudaMemcpy(h->d_m1, state + fc::kMlpPacked, sizeof(float) * fc::kMlpParams, cudaMemcpyHostToDevice));
    FC_CK(cudaMemcpy(h->d_m2, state + fc::kMlpPacked + fc::kMlpParams, sizeof(float) * fc::kMlpParams,
                     cudaMemcpyHostToDevice));
    h->sur_step = (int)state[fc::kMlpPacked + 2 * fc::kMlpParams];
    h->has_sur = true;
    h->sur_fitted = true;
    return FC_OK;
}

int fc_surrogate_eval(fc_handle *h, const float *L, int64_t n, float *lnT, int64_t *n_fallback,
                      void *stream)
{
    int rc = sur_check_data(h, "fc_surrogate_eval", L, nullptr, false, n);
    if (rc) return rc;
    if (!lnT) return fail(FC_EINVAL, "fc_surrogate_eval: null output");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    fc::SurrogateParams p;
    fill_sur_params(h, &p);
    if (n_fallback) FC_CK(cudaMemsetAsync(h->d_cnt, 0, sizeof(unsigned int), s));
    Trace t(h, FC_K_SURROGATE_EVAL, 1, s);
    FC_CK(fc::launch_mlp_eval(p, L, n, lnT, h->d_cnt, h->d_err, s));
    t.end();
    if (n_fallback) {
        unsigned int c = 0;
        FC_CK(cudaMemcpyAsync(&c, h->d_cnt, sizeof(c), cudaMemcpyDeviceToHost, s));
        FC_CK(cudaStreamSynchronize(s));
        *n_fallback = c;
        return sur_read_err(h, s, "fc_surrogate_eval");
    }
    return FC_OK;
}

int fc_surrogate_guard(fc_handle *h, const float *L, const float *lnT, int64_t n, double tol,
                       double *threshold, void *stream)
{
    if (!h) return fail(FC_EINVAL, "fc_surrogate_guard: null handle");
    if (!(tol > 0.0)) {
        h->sur_guard = INFINITY;
        if (threshold) *threshold = INFINITY;
        return FC_OK;
    }
    int rc = sur_check_data(h, "fc_surrogate_guard", L, lnT, true, n);
    if (rc) return rc;
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    float *ys = nullptr;
    FC_CK(dev_malloc((void **)&ys, (size_t)n * sizeof(float)));
    fc::SurrogateParams p;
    fill_sur_params(h, &p);
    p.guard = INFINITY;                            // the network alone
    // best = 0x7fffffff (bytes ff ff ff 7f): no ray beyond tol yet
    cudaError_t e = cudaMemsetAsync(h->d_cnt, 0xff, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(reinterpret_cast<char *>(h->d_cnt) + 3, 0x7f, 1, s);
    if (e == cudaSuccess) e = fc::launch_mlp_eval(p, L, n, ys, h->d_cnt + 1, h->d_err, s);
    if (e == cudaSuccess)
        e = fc::launch_guard_scan(p, L, lnT, ys, n, (float)tol, reinterpret_cast<int *>(h->d_cnt), s);
    int best = 0x7fffffff;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&best, h->d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ys);
    FC_CK(e);
    rc = sur_read_err(h, s, "fc_surrogate_guard");
    if (rc) return rc;
    if (best == 0x7fffffff) {
        h->sur_guard = INFINITY;
    } else {
        const int bits = best >= 0 ? best : best ^ 0x7fffffff;
        float v;
        memcpy(&v, &bits, sizeof(v));
        h->sur_guard = v;
    }
    if (threshold) *threshold = h->sur_guard;
    return FC_OK;
}

int fc_surrogate_sigma(const float *z, float *sigma, int64_t n, void *stream)
{
    if (n < 0) return fail(FC_EINVAL, "fc_surrogate_sigma: n = %lld < 0", (long long)n);
    if (n > 0 && (!z || !sigma)) return fail(FC_EINVAL, "fc_surrogate_sigma: NULL pointer");
    FC_CK(fc::launch_sigma_probe(z, sigma, n, (cudaStream_t)stream));
    return FC_OK;
}

int fc_surrogate_project(fc_handle *h, int angle_begin, int angle_count, float *out, int out_where,
                         void *stream)
{
    if (!h || !out) return fail(FC_EINVAL, "fc_surrogate_project: null argument");
    if (out_where != FC_HOST && out_where != FC_DEVICE)
        return fail(FC_EINVAL, "fc_surrogate_project: bad out_where");
    if (!h->has_sur) return fail(FC_ESTATE, "fc_surrogate_project: no surrogate");
    fc::ProjParams p;
    int rc = fill_proj_params(h, angle_begin, angle_count, &p);
    if (rc) return rc;
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)angle_count * h->g.n_v * h->g.n_u;
    if (n == 0) return FC_OK;
    if (n > h->sL_rays || !h->d_sL || !h->d_slnT) {
        dfree(h->d_sL);
        dfree(h->d_slnT);
        h->sL_rays = 0;
        FC_CK(dev_malloc((void **)&h->d_sL, n * h->n_mat * sizeof(float)));
        FC_CK(dev_malloc((void **)&h->d_slnT, n * sizeof(float)));
        h->sL_rays = n;
    }
    {
        Trace t(h, FC_K_LENGTHS, 1, s);
        FC_CK(fc::launch_project(p, nullptr, h->d_sL, s));
        t.end();
    }
    fc::SurrogateParams sp;
    fill_sur_params(h, &sp);
    {
        Trace t(h, FC_K_SURROGATE_EVAL, 1, s);
        FC_CK(fc::launch_mlp_eval(sp, h->d_sL, (long long)n, h->d_slnT, h->d_cnt, h->d_err, s));
        t.end();
    }
    if (out_where == FC_DEVICE) {
        FC_CK(fc::launch_exp(h->d_slnT, out, (long long)n, s));
        return FC_OK;
    }
    FC_CK(fc::launch_exp(h->d_slnT, h->d_slnT, (long long)n, s));
    return copy_out(out, FC_HOST, h->d_slnT, n * sizeof(float), s);
}

int fc_energy_sum_lengths(fc_handle *h, const float *L, int64_t n, float *lnT, void *stream)
{
    if (!h || !L || !lnT || n < 0) return fail(FC_EINVAL, "fc_energy_sum_lengths: bad argument");
    if (!h->has_spec) return fail(FC_ESTATE, "fc_energy_sum_lengths: set the spectrum first");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    fc::SurrogateParams p;
    fill_sur_params(h, &p);
    Trace t(h, FC_K_ENERGY_SUM, 1, s);
    FC_CK(fc::launch_energy_sum_lengths(p, L, n, lnT, s));
    t.end();
    return FC_OK;
}

int fc_cnr_grad(fc_handle *h, const double *logits, const double *D, const double *rho_nominal,
                const float *rho, const float *z, int n_roi, const fc_cnr_roi *rois, double *J,
                double *g_logits, double *g_D, float *g_rho, void *stream)
{
    if (!h || !logits || !D || !rho_nominal || !rho || !J || (n_roi > 0 && !rois))
        return fail(FC_EINVAL, "fc_cnr_grad: null argument");
    if (!h->has_geom || !h->has_phantom || !h->has_spec)
        return fail(FC_ESTATE, "fc_cnr_grad: geometry, phantom and spectrum must be set");
    if (n_roi < 1 || n_roi > fc::kMaxRoi) return fail(FC_EINVAL, "fc_cnr_grad: n_roi outside [1, %d]", fc::kMaxRoi);
    for (int m = 0; m < h->n_mat; ++m)
        if (!(rho_nominal[m] > 0.0)) return fail(FC_EINVAL, "fc_cnr_grad: nominal densities must be > 0");
    DeviceGuard dgd(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    FC_CK(h->order_after_copy(s));   // the volume and HU buffers are rewritten
    int rc = ensure_proj_buffers(h);
    if (rc) return rc;
    rc = ensure_recon_buffers(h, s);
    if (rc) return rc;
    const size_t np = h->proj_elems, nv = h->vol_elems;
    if (!h->d_I) FC_CK(dev_malloc((void **)&h->d_I, np * sizeof(float)));
    if (!h->d_gI) FC_CK(dev_malloc((void **)&h->d_gI, np * sizeof(float)));
    if (!h->d_gT) FC_CK(dev_malloc((void **)&h->d_gT, np * sizeof(float)));
    if (!h->d_gtmp) FC_CK(dev_malloc((void **)&h->d_gtmp, np * sizeof(float)));
    if (!h->d_gf) FC_CK(dev_malloc((void **)&h->d_gf, h->filt_elems * sizeof(float)));
    if (!h->d_gmu) FC_CK(dev_malloc((void **)&h->d_gmu, nv * sizeof(float)));
    if (!h->d_gwd) FC_CK(dev_malloc((void **)&h->d_gwd, (fc::kMaxBins + 1) * sizeof(double)));
    // spectrum: w = softmax(logits), c = w D, wd = c / sum c
    const int ne = h->n_e;
    std::vector<double> w(ne), c(ne);
    double mx = logits[0];
    for (int e = 1; e < ne; ++e) mx = logits[e] > mx ? logits[e] : mx;
    double zs = 0.0;
    for (int e = 0; e < ne; ++e) zs += (w[e] = exp(logits[e] - mx));
    double csum = 0.0;
    for (int e = 0; e < ne; ++e) {
        w[e] /= zs;
        c[e] = w[e] * D[e];
        csum += c[e];
    }
    if (!(csum > 0.0)) return fail(FC_EINVAL, "fc_cnr_grad: sum_E w D must be > 0");
    fc::AdjParams p;
    memset(&p, 0, sizeof(p));
    p.g = h->dg;
    p.trig = h->d_trig;
    p.labels = h->d_labels;
    p.n_e = ne;
    p.inv_csum = (float)(1.0 / csum);
    const double log2e = 1.4426950408889634;
    for (int m = 0; m < fc::kMaxMat; ++m) p.irho0[m] = m < h->n_mat ? (float)(1.0 / rho_nominal[m]) : 0.0f;
    for (int e = 0; e < ne; ++e) {
        p.wd[e] = (float)(c[e] / csum);
        for (int m = 0; m < fc::kMaxMat; ++m) p.mu[e][m] = (float)(h->mu2[(size_t)e * fc::kMaxMat + m] / log2e);
    }
    fc::BlurParams b;
    memset(&b, 0, sizeof(b));
    b.n_u = h->g.n_u;
    b.n_v = h->g.n_v;
    rc = gauss_taps(h->psf, b.gp, &b.rp);
    if (rc) return rc;
    rc = gauss_taps(h->sc, b.gs, &b.rs);
    if (rc) return rc;
    b.n0 = (float)h->n0;
    b.spr = (float)h->spr;
    fc::FdkParams pf;
    memset(&pf, 0, sizeof(pf));
    pf.g = h->dg;
    pf.trig = h->d_trig;
    pf.log_flood = (float)log(h->n0 * (1.0 + h->spr));
    pf.tau = (float)(h->g.du_cm * h->g.sad_cm / h->g.sdd_cm);
    pf.mag = (float)(h->g.sad_cm / h->g.sdd_cm);
    pf.scale = h->g.arc_rad / (2.0 * h->g.n_angles);
    fc::fdk_row_range(h->dg, &pf.v_lo, &pf.v_hi);
    pf.pw = fdk_row_pitch(h->g.n_u);
    pf.ph = pf.v_hi - pf.v_lo + 1 + 3;
    pf.sym_quarter = g_sym_quarter_ok(h->g) ? fdk_sym_turn(h->g, 4) : 0;
    pf.fft_tw = nullptr;
    pf.fft_k = nullptr;
    rc = ensure_fft_tables(h, &pf);
    if (rc) return rc;
    fc::CnrParams cp;
    memset(&cp, 0, sizeof(cp));
    cp.g = h->dg;
    cp.water_r = h->water_r;
    const int zcut = (int)floor(h->g.nz * h->zmargin);
    cp.zcut = (h->g.nz > 2 * zcut) ? zcut : 0;
    cp.n_roi = n_roi;
    for (int r = 0; r < n_roi; ++r) {
        cp.cx[r] = rois[r].cx_cm;
        cp.cy[r] = rois[r].cy_cm;
        cp.rad[r] = rois[r].radius_cm;
    }
    const int na = h->g.n_angles;
    // forward
    FC_CK(fc::launch_project_density(p, rho, h->d_T, s));
    FC_CK(fc::launch_blur_rows(b, h->d_T, h->d_tp, h->d_ts, na, s));
    FC_CK(fc::launch_blur_cols(b, h->d_tp, h->d_ts, h->d_I, na, s));
    FC_CK(fc::launch_noise_gauss(h->d_I, z, h->d_counts, np, s));
    {
        const int bpv = fc::backproject_variant(pf, h->bp_request);
        if (bpv < 0) return fail(FC_EINVAL, "fc_cnr_grad: backprojector variant %d does not apply to this geometry",
                                 h->bp_request);
        pf.filt_quad = fc::backproject_reads_quad(pf, bpv) ? 1 : 0;
        rc = filt_layout(h, pf.filt_quad, s);
        if (rc) return rc;
        FC_CK(fc::launch_fdk_filter(pf, h->d_counts, h->d_filt, s));
        FC_CK(fc::launch_backproject(pf, h->d_filt, h->d_vol, bpv, s));
    }
    if (!h->d_cnr_work) FC_CK(dev_malloc((void **)&h->d_cnr_work, fc::cnr_work_doubles() * sizeof(double)));
    FC_CK(fc::launch_cnr(cp, h->d_vol, h->d_gmu, h->d_gwd + fc::kMaxBins, h->d_cnr_work, s));
    const bool grads = g_logits || g_D || g_rho;
    if (grads) {
        FC_CK(cudaMemsetAsync(h->d_gf, 0, h->filt_elems * sizeof(float), s));
        FC_CK(fc::launch_backproject_adjoint(pf, h->d_gmu, h->d_gf, s));
        FC_CK(cudaMemsetAsync(h->d_gI, 0, np * sizeof(float), s));
        FC_CK(fc::launch_filter_adjoint(pf, h->d_gf, h->d_I, h->d_counts, z, h->d_gI, s));
        // d_tp / d_ts are free once the forward blur has run
        FC_CK(fc::launch_blur_transpose(b, h->d_gI, h->d_tp, h->d_ts, h->d_gT, na, s));
        FC_CK(cudaMemsetAsync(h->d_gwd, 0, fc::kMaxBins * sizeof(double), s));
        float *grho = g_rho ? g_rho : h->d_gtmp;   // scratch when only spectral grads are wanted
        FC_CK(cudaMemsetAsync(grho, 0, nv * sizeof(float), s));
        FC_CK(fc::launch_project_density_adjoint(p, rho, h->d_gT, grho, h->d_gwd, s));
    }
    std::vector<double> host(fc::kMaxBins + 1);
    FC_CK(cudaMemcpyAsync(host.data(), h->d_gwd, (fc::kMaxBins + 1) * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
    FC_CK(cudaStreamSynchronize(s));
    *J = host[fc::kMaxBins];
    if (grads) {
        // c_E = w_E D_E: dJ/dw_E = gc_E D_E, dJ/dD_E = gc_E w_E; softmax Jacobian
        double dot = 0.0;
        std::vector<double> gw(ne);
        for (int e = 0; e < ne; ++e) {
            gw[e] = host[e] * D[e];
            dot += w[e] * gw[e];
        }
        for (int e = 0; e < ne; ++e) {
            if (g_D) g_D[e] = host[e] * w[e];
            if (g_logits) g_logits[e] = w[e] * (gw[e] - dot);
        }
    }
    return FC_OK;
}

int fc_poisson(const float *lam, float *counts, int n_angles, int n_v, int n_u, int angle0,
               uint64_t seed, void *stream)
{
    if (!lam || !counts) return fail(FC_EINVAL, "fc_poisson: null argument");
    if (n_angles < 0 || n_v < 0 || n_u < 0 || angle0 < 0) return fail(FC_EINVAL, "fc_poisson: negative size");
    if (n_angles > 65535 || n_v > 65535) return fail(FC_EINVAL, "fc_poisson: n_angles and n_v must be <= 65535");
    FC_CK(fc::launch_poisson(lam, counts, n_angles, n_v, n_u, angle0, seed, (cudaStream_t)stream));
    return FC_OK;
}

}  // extern "C"

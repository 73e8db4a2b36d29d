// Reverse-mode (adjoint) gradient of an image-quality objective through the
// whole simulate-and-reconstruct path:
//
//   rho (voxel densities) -> A_im = sum_{v in ray i, label m} l_iv rho_v / rho0_m
//   T_i = sum_E (w D)_E exp(-sum_m mu_m(E) A_im) / sum_E (w D)_E    (Sec. II.F)
//   I = N0 (G_psf (x) T + SPR G_sc (x) T)                              (II.E/G)
//   K = I + sqrt(I) z       (Poisson noise replaced by its Gaussian form with
//                            fixed standard normals z, so K is smooth)
//   mu = FDK(ln(I_flood / K))                                          (II.G)
//   J = sum_R CNR_R(HU(mu)),  CNR = |HU_w - HU_R| / sqrt(s_w^2 + s_R^2)  (II.G)
//
// The forward pass reuses the detector-blur and FDK kernels; this file adds
// the density projector, the Gaussian-noise step, the CNR objective and the
// transposes of each linear step:
//   * CNR -> dJ/dmu (FP64, four grid-wide stages with fixed-order folds);
//   * backprojection^T: each ROI voxel scatters its bilinear weights into the
//     filtered-projection gradient (atomics);
//   * Ram-Lak^T = Ram-Lak (symmetric kernel, zero padding: the forward row
//     filter of fc_fdk.cu), then the log / cosine-weight / noise chain rule
//     down to dJ/dI;
//   * clamp-to-edge blur^T: zero-padded correlation plus the clamped mass
//     folded back onto the first and last pixel (the transposed mode of the
//     direct blur kernels, fc_detector.cu);
//   * projector^T: each ray that meets the voxels recomputes its path
//     lengths (first walk), forms dJ/dA_im and the spectral partials (summed
//     over each warp's rays by shuffles), then walks again scattering
//     dJ/drho_v = dJ/dA_{i,m(v)} l_iv / rho0_m(v) (atomics).
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {

__device__ __forceinline__ int clampi_(int v, int lo, int hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// Per-ray set-up shared by both walks: anchor A, direction d, entry/exit.
struct Ray {
    float A[3], d[3], inv[3];
    float t_in, t_out;
    bool hit;
};

__device__ __forceinline__ Ray make_ray(const DevGeom &g, float c, float s, int iu, int iv)
{
    Ray r;
    const float u = ((float)iu - g.cu) * g.du;
    const float v = ((float)iv - g.cv) * g.dv;
    const float uv2 = u * u + v * v;
    const float n2 = g.sdd * g.sdd + uv2;
    const float len = sqrtf(n2);
    const float il = __frcp_rn(len), in2 = __frcp_rn(n2);
    const float gx = -g.sdd * il, gy = u * il, gz = v * il;
    const float sA = g.sad * g.sdd * in2;
    const float agx = g.sad * uv2 * in2, agy = sA * u, agz = sA * v;
    r.A[0] = agx * c - agy * s;
    r.A[1] = agx * s + agy * c;
    r.A[2] = agz;
    r.d[0] = gx * c - gy * s;
    r.d[1] = gx * s + gy * c;
    r.d[2] = gz;
    const float lo[3] = {g.lox, g.loy, g.loz};
    r.t_in = -sA * len;
    r.t_out = (1.0f - sA) * len;
    r.hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.inv[a] = __frcp_rn(r.d[a]);
        if (r.d[a] != 0.0f) {
            const float t0 = (lo[a] - r.A[a]) * r.inv[a], t1 = (-lo[a] - r.A[a]) * r.inv[a];
            r.t_in = fmaxf(r.t_in, fminf(t0, t1));
            r.t_out = fminf(r.t_out, fmaxf(t0, t1));
        } else if (r.A[a] < lo[a] || r.A[a] >= -lo[a]) {
            r.hit = false;
        }
    }
    r.hit = r.hit && r.t_in < r.t_out;
    return r;
}

// Voxel walk along a ray: calls f(voxel index, segment length) for every
// voxel crossed.  Crossings t(i) = fma(i, pitch / d, (lo - A) / d); each
// step advances one index monotonically and stops at the grid edge, so at
// most nx + ny + nz steps occur and every index stays in the grid.
template <class F>
__device__ __forceinline__ void walk(const DevGeom &g, const Ray &r, F f)
{
    // per-axis state in scalars (a runtime axis index would put it in local memory)
    const float px = fmaf(r.t_in, r.d[0], r.A[0]), py = fmaf(r.t_in, r.d[1], r.A[1]);
    const float pz = fmaf(r.t_in, r.d[2], r.A[2]);
    int ix = clampi_((int)floorf((px - g.lox) * g.idx), 0, g.nx - 1);
    int iy = clampi_((int)floorf((py - g.loy) * g.idy), 0, g.ny - 1);
    int iz = clampi_((int)floorf((pz - g.loz) * g.idz), 0, g.nz - 1);
    const int sx = r.d[0] > 0.0f ? 1 : (r.d[0] < 0.0f ? -1 : 0);
    const int sy = r.d[1] > 0.0f ? 1 : (r.d[1] < 0.0f ? -1 : 0);
    const int sz = r.d[2] > 0.0f ? 1 : (r.d[2] < 0.0f ? -1 : 0);
    const int ux = sx > 0, uy = sy > 0, uz = sz > 0;
    const float vx = g.dx * r.inv[0], vy = g.dy * r.inv[1], vz = g.dz * r.inv[2];
    const float bx = (g.lox - r.A[0]) * r.inv[0], by = (g.loy - r.A[1]) * r.inv[1];
    const float bz = (g.loz - r.A[2]) * r.inv[2];
    float tx = sx ? fmaf((float)(ix + ux), vx, bx) : INFINITY;
    float ty = sy ? fmaf((float)(iy + uy), vy, by) : INFINITY;
    float tz = sz ? fmaf((float)(iz + uz), vz, bz) : INFINITY;
    const int nxy = g.nx * g.ny;
    int id = iz * nxy + iy * g.nx + ix;
    float t = r.t_in;
    for (int budget = g.nx + g.ny + g.nz + 3; budget > 0; --budget) {
        const float tm = fminf(tx, fminf(ty, tz));
        const float te = fminf(fmaxf(tm, t), r.t_out);
        f(id, te - t);
        t = te;
        if (tm >= r.t_out) break;
        if (tx == tm) {
            ix += sx;
            if (ix < 0 || ix >= g.nx) break;
            id += sx;
            tx = fmaf((float)(ix + ux), vx, bx);
        } else if (ty == tm) {
            iy += sy;
            if (iy < 0 || iy >= g.ny) break;
            id += sy * g.nx;
            ty = fmaf((float)(iy + uy), vy, by);
        } else {
            iz += sz;
            if (iz < 0 || iz >= g.nz) break;
            id += sz * nxy;
            tz = fmaf((float)(iz + uz), vz, bz);
        }
    }
}

}  // namespace

// Density-weighted path lengths A_m = sum_{v, label m} l_v rho_v / rho0_m of
// one ray (zero when r.hit is false): l_v rho_v is summed over each run of
// one label and the run is scaled by 1 / rho0_m when the label changes.
__device__ __forceinline__ void density_lengths(const AdjParams &p, const float *__restrict__ rho,
                                                const Ray &r, float (&A)[kMaxMat])
{
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) A[m] = 0.0f;
    if (!r.hit) return;
    int cur = -1;
    float run = 0.0f;
    walk(p.g, r, [&](int v, float len) {
        const int m = p.labels[v];
        if (m != cur) {
#pragma unroll
            for (int j = 0; j < kMaxMat; ++j) A[j] += (cur == j) ? run * p.irho0[j] : 0.0f;
            cur = m;
            run = 0.0f;
        }
        run = fmaf(len, rho[v], run);
    });
#pragma unroll
    for (int j = 0; j < kMaxMat; ++j) A[j] += (cur == j) ? run * p.irho0[j] : 0.0f;
}

// Forward density projector: T_i (flood-normalised) for all rays.
__global__ void __launch_bounds__(256)
k_project_density(const __grid_constant__ AdjParams p, const float *__restrict__ rho,
                  float *__restrict__ T)
{
    const DevGeom &g = p.g;
    // warp w of the CTA's 16 x 16 ray tile: columns 2w, 2w + 1, all 16 rows
    // (rays of one column cross the phantom close together and walk alike)
    const int iu = blockIdx.x * 16 + threadIdx.y * 2 + (threadIdx.x & 1);
    const int iv = blockIdx.y * 16 + (threadIdx.x >> 1), k = blockIdx.z;
    if (iu >= g.n_u || iv >= g.n_v) return;
    const float2 cs = p.trig[k];
    const Ray r = make_ray(g, cs.x, cs.y, iu, iv);
    float A[kMaxMat];
    density_lengths(p, rho, r, A);
    float sum = 0.0f;
    for (int e = 0; e < p.n_e; ++e) {
        float a = 0.0f;
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m) a = fmaf(p.mu[e][m], A[m], a);
        sum += p.wd[e] * __expf(-a);
    }
    T[((size_t)k * g.n_v + iv) * g.n_u + iu] = sum;
}

// Adjoint projector.  gT = dJ/dT per ray; accumulates dJ/d(wD)_E (before
// normalisation) into gwd[n_e] (FP64) and dJ/drho into grho.  A warp takes
// 32 rays of one row: rays of one column, as the forward kernel groups them,
// would add into the same voxels at the same steps and serialise the atomics
// (forward + gradient 20.8 ms against 19.2).
__global__ void __launch_bounds__(256)
k_project_density_adjoint(const __grid_constant__ AdjParams p, const float *__restrict__ rho,
                          const float *__restrict__ gT, float *__restrict__ grho,
                          double *__restrict__ gwd)
{
    __shared__ float sgw[8][kMaxBins];   // per-warp sums of dJ/dc_E over its rays
    const DevGeom &g = p.g;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int tid = w * 32 + lane;
    const int iu = blockIdx.x * 32 + lane, iv = blockIdx.y * 8 + w, k = blockIdx.z;
    const bool in = iu < g.n_u && iv < g.n_v;
    float gt = 0.0f;
    Ray r;
    r.hit = false;
    if (in) {
        gt = gT[((size_t)k * g.n_v + iv) * g.n_u + iu];
        const float2 cs = p.trig[k];
        r = make_ray(g, cs.x, cs.y, iu, iv);
    }
    // A ray that misses the voxels has A = 0, T = 1 and e_E - T = 0: it adds
    // nothing to either gradient.
    const bool act = in && r.hit && gt != 0.0f;
    Ray rr = r;
    rr.hit = act;
    float A[kMaxMat];
    density_lengths(p, rho, rr, A);
    // T = sum_E wd_E e_E with wd normalised (sum 1); for the unnormalised
    // weights c_E: dT/dc_E = (e_E - T) / sum c.  Here wd = c / sum c, so the
    // partial w.r.t. c_E is (e_E - T) * p.inv_csum.  Each bin's partial is
    // summed over the warp's 32 rays by a butterfly (fixed order).
    float gA[kMaxMat];
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) gA[m] = 0.0f;
    if (__any_sync(0xffffffffu, act)) {
        float T = 0.0f;
        if (act) {
            for (int e = 0; e < p.n_e; ++e) {
                float a = 0.0f;
#pragma unroll
                for (int m = 0; m < kMaxMat; ++m) a = fmaf(p.mu[e][m], A[m], a);
                T += p.wd[e] * __expf(-a);
            }
        }
        for (int e = 0; e < p.n_e; ++e) {
            float v = 0.0f;
            if (act) {
                float a = 0.0f;
#pragma unroll
                for (int m = 0; m < kMaxMat; ++m) a = fmaf(p.mu[e][m], A[m], a);
                const float ee = __expf(-a);
                v = gt * (ee - T) * p.inv_csum;
                const float c = -gt * p.wd[e] * ee;
#pragma unroll
                for (int m = 0; m < kMaxMat; ++m) gA[m] = fmaf(c, p.mu[e][m], gA[m]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sgw[w][e] = v;
        }
    } else if (lane == 0) {
        for (int e = 0; e < p.n_e; ++e) sgw[w][e] = 0.0f;
    }
    if (act) {
        // dJ/drho_v = gA_m(v) l_v / rho0_m(v): the coefficient changes only
        // with the label.
        int mc = -1;
        float cc = 0.0f;
        walk(g, r, [&](int v, float len) {
            const int m = p.labels[v];
            if (m != mc) {
                mc = m;
                cc = 0.0f;
#pragma unroll
                for (int j2 = 0; j2 < kMaxMat; ++j2) cc = (m == j2) ? gA[j2] * p.irho0[j2] : cc;
            }
            atomicAdd(grho + v, cc * len);
        });
    }
    __syncthreads();
    for (int e = tid; e < p.n_e; e += 256) {
        float sum = 0.0f;
        for (int ww = 0; ww < 8; ++ww) sum += sgw[ww][e];
        if (sum != 0.0f) atomicAdd(gwd + e, (double)sum);
    }
}

// K = I + sqrt(I) z (forward) with z a fixed standard-normal field.
__global__ void k_noise_gauss(const float *__restrict__ I, const float *__restrict__ z,
                              float *__restrict__ K, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float v = I[i];
        K[i] = z ? v + sqrtf(fmaxf(v, 0.0f)) * z[i] : v;
    }
}

// CNR objective and dJ/dmu (FP64).  ROI masks: water = centres within
// water_r of the axis; insert r = centres within rois[r].radius of its centre
// (first match, water first); both on slices [zcut, nz - zcut).
// Four grid-wide stages, each reduced per CTA into partials that every CTA
// of the next stage folds in the same fixed order (reproducible bits):
//   s1  count and sum of mu per region          -> mu_w, mean HU per region
//   s2  sum of (HU - mean HU)^2 per region      -> variances, J, dJ/dHU terms
//   s3  sum over regions of dJ/dHU_u mu_u        -> the mu_w correction
//   s4  dJ/dmu per voxel; CTA 0 writes J
namespace {
constexpr int kCnrBlocks = 304;
constexpr int kCnrThreads = 256;
constexpr int kReg = kMaxRoi + 1;

__device__ int cnr_region(const CnrParams &c, size_t i)
{
    const DevGeom &g = c.g;
    const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((size_t)g.nx * g.ny));
    if (iz < c.zcut || iz >= g.nz - c.zcut) return -1;
    const double x = (ix - 0.5 * (g.nx - 1)) * (double)g.dx, y = (iy - 0.5 * (g.ny - 1)) * (double)g.dy;
    if (x * x + y * y <= c.water_r * c.water_r) return 0;
    for (int r = 0; r < c.n_roi; ++r) {
        const double dx = x - c.cx[r], dy = y - c.cy[r];
        if (dx * dx + dy * dy <= c.rad[r] * c.rad[r]) return r + 1;
    }
    return -1;
}

// fixed-order block sum (tree over kCnrThreads)
__device__ double cnr_block_sum(double v, double *red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = kCnrThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

struct CnrStats {
    double cnt[kReg], mean_mu[kReg], mean_hu[kReg], var[kReg];
    double mu_w;
    double gm0[kReg], gm1[kReg];   // dJ/dHU_v = gm0[r] + gm1[r] (HU_v - mean_hu[r])
    double J;
};

// totals of stage 1 (and 2 when part2 != nullptr), folded by the whole CTA in
// a fixed order (thread t takes partials t, t + kCnrThreads, ...; then the
// block tree), so every CTA obtains the same bits.  All threads call it.
__device__ void cnr_fold(const CnrParams &c, const double *part1, const double *part2, CnrStats &t,
                         double *red)
{
    const int nr = c.n_roi + 1;
    for (int r = 0; r < nr; ++r) {
        double n = 0.0, sm = 0.0;
        for (int b = threadIdx.x; b < kCnrBlocks; b += kCnrThreads) {
            n += part1[(size_t)b * 2 * kReg + r];
            sm += part1[(size_t)b * 2 * kReg + kReg + r];
        }
        n = cnr_block_sum(n, red);
        sm = cnr_block_sum(sm, red);
        if (threadIdx.x == 0) {
            t.cnt[r] = n;
            t.mean_mu[r] = sm / n;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        t.mu_w = t.mean_mu[0];
        for (int r = 0; r < nr; ++r) t.mean_hu[r] = 1000.0 * (t.mean_mu[r] - t.mu_w) / t.mu_w;
    }
    __syncthreads();
    if (!part2) return;
    for (int r = 0; r < nr; ++r) {
        double q = 0.0;
        for (int b = threadIdx.x; b < kCnrBlocks; b += kCnrThreads) q += part2[(size_t)b * kReg + r];
        q = cnr_block_sum(q, red);
        if (threadIdx.x == 0) t.var[r] = q / t.cnt[r];   // population variance
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double J = 0.0, cw_mean = 0.0, cw_dev = 0.0;
        const double nw = t.cnt[0], mw = t.mean_hu[0], vw = t.var[0];
        // dCNR/dHU_v: water v: sgn/(nw sd) - |a|/sd^3 (HU_v - mw)/nw
        //             insert v: -sgn/(nr sd) - |a|/sd^3 (HU_v - mr)/nr
        for (int r = 1; r < nr; ++r) {
            const double nrr = t.cnt[r], mr = t.mean_hu[r], vr = t.var[r];
            const double a = mw - mr, sd = sqrt(vw + vr), sgn = a >= 0.0 ? 1.0 : -1.0;
            J += fabs(a) / sd;
            cw_mean += sgn / (nw * sd);
            cw_dev += -fabs(a) / (sd * sd * sd) / nw;
            t.gm0[r] = -sgn / (nrr * sd);
            t.gm1[r] = -fabs(a) / (sd * sd * sd) / nrr;
        }
        t.gm0[0] = cw_mean;
        t.gm1[0] = cw_dev;
        t.J = J;
    }
    __syncthreads();
}
}  // namespace

__global__ void __launch_bounds__(kCnrThreads)
k_cnr_s1(const __grid_constant__ CnrParams c, const double *__restrict__ mu, double *part1)
{
    __shared__ double red[kCnrThreads];
    const size_t n = (size_t)c.g.nx * c.g.ny * c.g.nz;
    double cnt[kReg], sm[kReg];
#pragma unroll
    for (int r = 0; r < kReg; ++r) cnt[r] = sm[r] = 0.0;
    for (size_t i = (size_t)blockIdx.x * kCnrThreads + threadIdx.x; i < n; i += (size_t)kCnrBlocks * kCnrThreads) {
        const int r = cnr_region(c, i);
#pragma unroll
        for (int rr = 0; rr < kReg; ++rr)
            if (r == rr) { cnt[rr] += 1.0; sm[rr] += mu[i]; }
    }
    for (int r = 0; r < kReg; ++r) {
        const double a = cnr_block_sum(cnt[r], red), b = cnr_block_sum(sm[r], red);
        if (threadIdx.x == 0) {
            part1[(size_t)blockIdx.x * 2 * kReg + r] = a;
            part1[(size_t)blockIdx.x * 2 * kReg + kReg + r] = b;
        }
    }
}

__global__ void __launch_bounds__(kCnrThreads)
k_cnr_s2(const __grid_constant__ CnrParams c, const double *__restrict__ mu, const double *part1,
         double *part2)
{
    __shared__ double red[kCnrThreads];
    __shared__ CnrStats t;
    cnr_fold(c, part1, nullptr, t, red);
    const size_t n = (size_t)c.g.nx * c.g.ny * c.g.nz;
    double q[kReg];
#pragma unroll
    for (int r = 0; r < kReg; ++r) q[r] = 0.0;
    for (size_t i = (size_t)blockIdx.x * kCnrThreads + threadIdx.x; i < n; i += (size_t)kCnrBlocks * kCnrThreads) {
        const int r = cnr_region(c, i);
        if (r < 0) continue;
        const double hu = 1000.0 * (mu[i] - t.mu_w) / t.mu_w;
#pragma unroll
        for (int rr = 0; rr < kReg; ++rr)
            if (r == rr) {
                const double dv = hu - t.mean_hu[rr];
                q[rr] += dv * dv;
            }
    }
    for (int r = 0; r < kReg; ++r) {
        const double a = cnr_block_sum(q[r], red);
        if (threadIdx.x == 0) part2[(size_t)blockIdx.x * kReg + r] = a;
    }
}

__global__ void __launch_bounds__(kCnrThreads)
k_cnr_s3(const __grid_constant__ CnrParams c, const double *__restrict__ mu, const double *part1,
         const double *part2, double *part3)
{
    __shared__ double red[kCnrThreads];
    __shared__ CnrStats t;
    cnr_fold(c, part1, part2, t, red);
    const size_t n = (size_t)c.g.nx * c.g.ny * c.g.nz;
    double gs = 0.0;   // sum_u dJ/dHU_u mu_u
    for (size_t i = (size_t)blockIdx.x * kCnrThreads + threadIdx.x; i < n; i += (size_t)kCnrBlocks * kCnrThreads) {
        const int r = cnr_region(c, i);
        if (r < 0) continue;
        const double hu = 1000.0 * (mu[i] - t.mu_w) / t.mu_w;
        gs += (t.gm0[r] + t.gm1[r] * (hu - t.mean_hu[r])) * mu[i];
    }
    gs = cnr_block_sum(gs, red);
    if (threadIdx.x == 0) part3[blockIdx.x] = gs;
}

// dJ/dmu through HU = 1000 (mu / mu_w - 1), mu_w = mean over the water region
__global__ void __launch_bounds__(kCnrThreads)
k_cnr_s4(const __grid_constant__ CnrParams c, const double *__restrict__ mu, const double *part1,
         const double *part2, const double *part3, float *__restrict__ gmu, double *out)
{
    __shared__ double red[kCnrThreads];
    __shared__ CnrStats t;
    cnr_fold(c, part1, part2, t, red);
    double gs = 0.0;
    for (int b = threadIdx.x; b < kCnrBlocks; b += kCnrThreads) gs += part3[b];
    gs = cnr_block_sum(gs, red);
    const double corr = 1000.0 / (t.mu_w * t.mu_w) * gs / t.cnt[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = t.J;
    const size_t n = (size_t)c.g.nx * c.g.ny * c.g.nz;
    for (size_t i = (size_t)blockIdx.x * kCnrThreads + threadIdx.x; i < n; i += (size_t)kCnrBlocks * kCnrThreads) {
        const int r = cnr_region(c, i);
        double v = 0.0;
        if (r >= 0) {
            const double hu = 1000.0 * (mu[i] - t.mu_w) / t.mu_w;
            const double gh = t.gm0[r] + t.gm1[r] * (hu - t.mean_hu[r]);
            v = 1000.0 / t.mu_w * gh - (r == 0 ? corr : 0.0);
        }
        gmu[i] = (float)v;
    }
}

// Backprojection transpose: gf (padded filtered layout) += B^T gmu.
__global__ void __launch_bounds__(256)
k_backproject_adjoint(const __grid_constant__ FdkParams p, const float *__restrict__ gmu,
                      float *__restrict__ gf)
{
    const DevGeom &g = p.g;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gv = gmu[i];
    if (gv == 0.0f) return;
    const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((size_t)g.nx * g.ny));
    const float x = ((float)ix - 0.5f * (float)(g.nx - 1)) * g.dx;
    const float y = ((float)iy - 0.5f * (float)(g.ny - 1)) * g.dy;
    const float zz = ((float)iz - 0.5f * (float)(g.nz - 1)) * g.dz;
    const float cu1 = g.cu + 1.0f, cv1 = g.cv - (float)p.v_lo + 1.0f;
    const float umax = (float)(p.pw - 2), vmaxp = (float)(p.ph - 2);
    const float sdd_du = g.sdd / g.du, sdd_dv = g.sdd / g.dv;
    const size_t plane = (size_t)p.ph * p.pw;
    const float scale = (float)p.scale;
    for (int k = 0; k < g.n_angles; ++k) {
        const float2 cs = p.trig[k];
        const float U = g.sad - (x * cs.x + y * cs.y);
        const float ru = y * cs.x - x * cs.y;
        const float iU = __frcp_rn(U);
        const float fu = fminf(fmaxf(fmaf(ru * iU, sdd_du, cu1), 0.0f), umax);
        const float fv = fminf(fmaxf(fmaf(zz * iU, sdd_dv, cv1), 0.0f), vmaxp);
        const float w = (g.sad * iU) * (g.sad * iU) * scale * gv;
        const float fu0 = floorf(fu), fv0 = floorf(fv);
        const float au = fu - fu0, av = fv - fv0;
        float *b = gf + (size_t)k * plane + (size_t)fv0 * p.pw + (int)fu0;
        atomicAdd(b, w * (1.0f - au) * (1.0f - av));
        atomicAdd(b + 1, w * au * (1.0f - av));
        atomicAdd(b + p.pw, w * (1.0f - au) * av);
        atomicAdd(b + p.pw + 1, w * au * av);
    }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_project_density(const AdjParams &p, const float *rho, float *T, cudaStream_t s)
{
    dim3 block(32, 8), grid((p.g.n_u + 15) / 16, (p.g.n_v + 15) / 16, p.g.n_angles);
    k_project_density<<<grid, block, 0, s>>>(p, rho, T);
    return cudaGetLastError();
}

cudaError_t launch_project_density_adjoint(const AdjParams &p, const float *rho, const float *gT,
                                           float *grho, double *gwd, cudaStream_t s)
{
    dim3 block(32, 8), grid((p.g.n_u + 31) / 32, (p.g.n_v + 7) / 8, p.g.n_angles);
    k_project_density_adjoint<<<grid, block, 0, s>>>(p, rho, gT, grho, gwd);
    return cudaGetLastError();
}

cudaError_t launch_noise_gauss(const float *I, const float *z, float *K, size_t n, cudaStream_t s)
{
    k_noise_gauss<<<sm_count() * 8, 256, 0, s>>>(I, z, K, n);
    return cudaGetLastError();
}

size_t cnr_work_doubles() { return (size_t)kCnrBlocks * (3 * kReg + 1); }

cudaError_t launch_cnr(const CnrParams &c, const double *mu, float *gmu, double *out, double *work,
                       cudaStream_t s)
{
    double *p1 = work, *p2 = p1 + (size_t)kCnrBlocks * 2 * kReg, *p3 = p2 + (size_t)kCnrBlocks * kReg;
    k_cnr_s1<<<kCnrBlocks, kCnrThreads, 0, s>>>(c, mu, p1);
    k_cnr_s2<<<kCnrBlocks, kCnrThreads, 0, s>>>(c, mu, p1, p2);
    k_cnr_s3<<<kCnrBlocks, kCnrThreads, 0, s>>>(c, mu, p1, p2, p3);
    k_cnr_s4<<<kCnrBlocks, kCnrThreads, 0, s>>>(c, mu, p1, p2, p3, gmu, out);
    return cudaGetLastError();
}

cudaError_t launch_backproject_adjoint(const FdkParams &p, const float *gmu, float *gf, cudaStream_t s)
{
    const size_t n = (size_t)p.g.nx * p.g.ny * p.g.nz;
    k_backproject_adjoint<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, gmu, gf);
    return cudaGetLastError();
}

}  // namespace fc

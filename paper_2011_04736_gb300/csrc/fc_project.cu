// Polyenergetic cone-beam projector (paper Sec. II.F "Raytracing" and the
// energy-weighting equation I_f = sum_E phi(E) eta(E) I(E)).
//
// One thread per detector pixel ray.  The ray is traversed in voxel order
// (Siddon / Amanatides-Woo) on two levels: bricks of 8 x 8 voxels in-plane
// and 16 along the rotation axis whose voxels all carry one label are crossed
// in a single step, mixed bricks voxel by voxel.  (Rays of one detector
// column, which share a warp, differ mostly in z; deep bricks keep their brick
// sequences in step through thin slabs.)
// Every plane crossing, coarse or fine, is t(i) = fma(i, pitch / d, (lo - A) / d)
// for the plane's index i, so both levels agree bit for bit on brick faces.
// The path length inside each material is accumulated run by run: a length
// is added only when the label changes, so binary32 rounding enters once per
// material transition instead of once per voxel.  The per-material lengths stay in
// registers and feed the energy integral
//     T = sum_E (w D)_E exp(-sum_m mu_m(E) L_m)        (w D normalised)
// evaluated with exp2 and a compensated (Kahan) sum over the energy bins.
// A warp covers 32 consecutive rays of one detector column (the band order
// below), so each lane's T store lands in its own detector row: one store
// per ray, a small part of the walk's cost; the rows of T that the band
// does not cover are written by a store-only kernel in float4 rows.
//
// Numerics: the ray is represented by its point A closest to the rotation
// axis and a unit direction, both rotated from the gantry frame, so every
// coordinate the traversal uses is O(volume size) and every component of the
// direction carries a relative error of a few ulp of itself.
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {

__device__ __forceinline__ void add_run(float (&L)[kMaxMat], int m, float len)
{
#pragma unroll
    for (int j = 0; j < kMaxMat; ++j) L[j] += (m == j) ? len : 0.0f;
}

// Crossing parameter of plane i of one axis (INFINITY if the ray is
// parallel to that axis).
__device__ __forceinline__ float plane_t(int i, float vs, float base, int sgn)
{
    return sgn ? fmaf((float)i, vs, base) : INFINITY;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

}  // namespace

// Ray order inside the traced band [r0, r0 + R) of one projection: ray t is
// row r0 + t % R of column t / R, so a warp's 32 consecutive rays run down
// the columns of the band (CTAs of 256 rays).  Rays of one detector column
// cross the phantom above one another, a slice apart or less, so where
// labels vary slowly along z they meet the same bricks and voxel runs and the
// warp's lanes step together; 32 rays along a row fan out in-plane and meet
// mixed bricks at different steps.  The band is not padded, so however thin
// it is no lane holds a ray outside it.  (Every ray's result is the same in
// any order; only the grouping into warps changes.)
constexpr int kBandCta = 256;

__device__ __forceinline__ bool band_ray(int t, int r0, int R, int n_u, int &iu, int &iv)
{
    if (t >= R * n_u) return false;
    iu = t / R;
    iv = r0 + (t - iu * R);
    return true;
}

__device__ __forceinline__ int band_t() { return (int)blockIdx.x * kBandCta + (int)threadIdx.y * 32 + (int)threadIdx.x; }

// Per-material path lengths L of pixel ray (iu, iv) of projection k; returns
// whether the ray meets the voxel box.  TEST_ONLY: return after the box test
// (L not computed).  SMEM_BRICKS: the brick map is read from the CTA's
// shared-memory copy sb instead of global memory.
template <bool TEST_ONLY = false, bool SMEM_BRICKS = false>
__device__ __forceinline__ bool trace_ray(const ProjParams &p, int iu, int iv, int k,
                                          float (&L)[kMaxMat], const uint8_t *sb = nullptr)
{
    const DevGeom &g = p.g;
#pragma unroll
    for (int m = 0; m < kMaxMat; ++m) L[m] = 0.0f;

    // Rows outside [v_hit_lo, v_hit_hi] cannot meet the voxel slab (host
    // bound with margin): their rays keep L = 0 and T = 1.
    bool hit = iv >= p.v_hit_lo && iv <= p.v_hit_hi;
    if (hit) {
        const float2 cs = p.trig[k];
        const float c = cs.x, s = cs.y;
        // pixel in the gantry frame: source (SAD, 0, 0), pixel (SAD - SDD, u, v)
        const float u = ((float)iu - g.cu) * g.du;
        const float v = ((float)iv - g.cv) * g.dv;
        const float uv2 = u * u + v * v;
        const float n2 = g.sdd * g.sdd + uv2;
        const float len = sqrtf(n2);
        const float inv_len = __frcp_rn(len);
        const float inv_n2 = __frcp_rn(n2);
        const float gx = -g.sdd * inv_len, gy = u * inv_len, gz = v * inv_len;
        // closest point to the axis: fraction sA of the way from source to pixel
        const float sA = g.sad * g.sdd * inv_n2;
        const float agx = g.sad * uv2 * inv_n2, agy = sA * u, agz = sA * v;
        const float Ax = agx * c - agy * s, Ay = agx * s + agy * c, Az = agz;
        const float dx = gx * c - gy * s, dy = gx * s + gy * c, dz = gz;
        const float ix_ = __frcp_rn(dx), iy_ = __frcp_rn(dy), iz_ = __frcp_rn(dz);

        // clip to the source-pixel segment and to the voxel box (slab method)
        float t_in = -sA * len, t_out = (1.0f - sA) * len;
        {
            const float A3[3] = {Ax, Ay, Az}, d3[3] = {dx, dy, dz}, i3[3] = {ix_, iy_, iz_};
            const float lo3[3] = {g.lox, g.loy, g.loz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float hi = -lo3[a];
                if (d3[a] != 0.0f) {
                    const float t0 = (lo3[a] - A3[a]) * i3[a];
                    const float t1 = (hi - A3[a]) * i3[a];
                    t_in = fmaxf(t_in, fminf(t0, t1));
                    t_out = fminf(t_out, fmaxf(t0, t1));
                } else if (A3[a] < lo3[a] || A3[a] >= hi) {
                    hit = false;
                }
            }
        }
        hit = hit && t_in < t_out;
        if (TEST_ONLY) return hit;
        if (hit) {
            const float px = fmaf(t_in, dx, Ax), py = fmaf(t_in, dy, Ay), pz = fmaf(t_in, dz, Az);
            const int nx = g.nx, ny = g.ny, nz = g.nz;
            const int ix0 = clampi((int)floorf((px - g.lox) * g.idx), 0, nx - 1);
            const int iy0 = clampi((int)floorf((py - g.loy) * g.idy), 0, ny - 1);
            const int iz0 = clampi((int)floorf((pz - g.loz) * g.idz), 0, nz - 1);
            const int sx = dx > 0.0f ? 1 : (dx < 0.0f ? -1 : 0);
            const int sy = dy > 0.0f ? 1 : (dy < 0.0f ? -1 : 0);
            const int sz = dz > 0.0f ? 1 : (dz < 0.0f ? -1 : 0);
            const int ux = sx > 0, uy = sy > 0, uz = sz > 0;   // next plane = index + u
            // t(i) = fma(i, v*, b*): v* = pitch / d, b* = (lo - A) / d
            const float vx = g.dx * ix_, vy = g.dy * iy_, vz = g.dz * iz_;
            const float bx_ = (g.lox - Ax) * ix_, by_ = (g.loy - Ay) * iy_, bz_ = (g.loz - Az) * iz_;
            const int nbx = (nx + kBrick - 1) / kBrick, nby = (ny + kBrick - 1) / kBrick;
            const int nbz = (nz + kBrickZ - 1) / kBrickZ;
            int bx = ix0 / kBrick, by = iy0 / kBrick, bz = iz0 / kBrickZ;
            int bi = (bz * nby + by) * nbx + bx;       // brick index, kept incrementally
            // coarse crossing: far face of the current brick along the ray
            // (plane index cp*, kept incrementally)
            int cpx = ux ? min((bx + 1) * kBrick, nx) : bx * kBrick;
            int cpy = uy ? min((by + 1) * kBrick, ny) : by * kBrick;
            int cpz = uz ? min((bz + 1) * kBrickZ, nz) : bz * kBrickZ;
            float tcx = plane_t(cpx, vx, bx_, sx);
            float tcy = plane_t(cpy, vy, by_, sy);
            float tcz = plane_t(cpz, vz, bz_, sz);
            // labels z fastest: voxel (x, y, z) at (y nx + x) nz + z, so the
            // rays of one detector column (a warp's lanes, a slice or less
            // apart) read neighbouring bytes
            const int zsx = nz, zsy = nx * nz;
            int cur = __ldg(p.labels_zf + (iy0 * nx + ix0) * nz + iz0);
            float t_run = t_in, t_cur = t_in;
            // Coarse passes: each advances one brick index by one step along
            // the ray, so at most nbx + nby + nbz passes occur before an index
            // leaves the grid.  Fine passes inside a brick: each advances one
            // voxel index inside the brick (a step that would cross the brick
            // face has t >= t_exit and ends the fine walk), at most
            // 2 kBrick + kBrickZ.
            // The budgets only guard against non-finite geometry.
            for (int cb = nbx + nby + nbz + 3; cb > 0; --cb) {
                const float tmin = fminf(tcx, fminf(tcy, tcz));
                const float t_exit = fmaxf(tmin, t_cur);
                const int bl = SMEM_BRICKS ? (int)sb[bi] : (int)__ldg(p.bricks + bi);
                if (bl != kMixed) {
                    if (bl != cur) {
                        add_run(L, cur, t_cur - t_run);
                        t_run = t_cur;
                        cur = bl;
                    }
                } else if (tmin > t_cur) {
                    // Fine walk through the brick over [t_cur, t_exit).  The
                    // brick's faces are crossed at t >= t_exit = tmin (same
                    // plane index, same formula as the coarse crossings), so
                    // only interior planes are stepped and the voxel indices
                    // stay inside the brick.  (A brick with tmin <= t_cur is
                    // crossed over zero length and has nothing to add.)
                    const float qx = fmaf(t_cur, dx, Ax), qy = fmaf(t_cur, dy, Ay);
                    const float qz = fmaf(t_cur, dz, Az);
                    int jx = clampi((int)floorf((qx - g.lox) * g.idx), bx * kBrick,
                                    min((bx + 1) * kBrick, nx) - 1);
                    int jy = clampi((int)floorf((qy - g.loy) * g.idy), by * kBrick,
                                    min((by + 1) * kBrick, ny) - 1);
                    int jz = clampi((int)floorf((qz - g.loz) * g.idz), bz * kBrickZ,
                                    min((bz + 1) * kBrickZ, nz) - 1);
                    // next plane index per axis; an axis that is stepped
                    // has a nonzero direction, so its crossing is a plain fma
                    int fx = jx + ux, fy = jy + uy, fz = jz + uz;
                    float tfx = plane_t(fx, vx, bx_, sx);
                    float tfy = plane_t(fy, vy, by_, sy);
                    float tfz = plane_t(fz, vz, bz_, sz);
                    int id = (jy * nx + jx) * nz + jz;
                    int lab = __ldg(p.labels_zf + id);
                    if (lab != cur) {
                        add_run(L, cur, t_cur - t_run);
                        t_run = t_cur;
                        cur = lab;
                    }
                    for (int fb = 2 * kBrick + kBrickZ + 3; fb > 0; --fb) {
                        const float tn = fminf(tfx, fminf(tfy, tfz));
                        if (tn >= t_exit) break;
                        if (tfx == tn) {
                            fx += sx; id += sx * zsx; tfx = fmaf((float)fx, vx, bx_);
                        } else if (tfy == tn) {
                            fy += sy; id += sy * zsy; tfy = fmaf((float)fy, vy, by_);
                        } else {
                            fz += sz; id += sz; tfz = fmaf((float)fz, vz, bz_);
                        }
                        lab = __ldg(p.labels_zf + id);
                        if (lab != cur) {
                            const float tb = fmaxf(tn, t_run);
                            add_run(L, cur, tb - t_run);
                            t_run = tb;
                            cur = lab;
                        }
                    }
                }
                // step to the next brick along the axis of the nearest face
                t_cur = t_exit;
                bool inside;
                // (a stepped axis has a nonzero direction; leaving the last
                // brick ends the walk, so the clip to n only matters going up)
                if (tcx == tmin) {
                    bx += sx;
                    bi += sx;
                    inside = (unsigned)bx < (unsigned)nbx;
                    cpx = min(cpx + kBrick * sx, nx);
                    tcx = fmaf((float)cpx, vx, bx_);
                } else if (tcy == tmin) {
                    by += sy;
                    bi += sy * nbx;
                    inside = (unsigned)by < (unsigned)nby;
                    cpy = min(cpy + kBrick * sy, ny);
                    tcy = fmaf((float)cpy, vy, by_);
                } else {
                    bz += sz;
                    bi += sz * nbx * nby;
                    inside = (unsigned)bz < (unsigned)nbz;
                    cpz = min(cpz + kBrickZ * sz, nz);
                    tcz = fmaf((float)cpz, vz, bz_);
                }
                if (!inside) break;
            }
            add_run(L, cur, t_cur - t_run);
        }
    }

    return hit;
}

// Energy integral of one ray from its path lengths (compensated sum over the
// bins; T = 1 for a ray that misses the voxels).
__device__ __forceinline__ float energy_T(const ProjParams &p, bool hit, const float (&L)[kMaxMat])
{
    float Tv = 1.0f;
    if (hit) {
        float sum = 0.0f, comp = 0.0f;
        for (int e = 0; e < p.n_e; ++e) {
            float a = 0.0f;
#pragma unroll
            for (int m = 0; m < kMaxMat; ++m) a = fmaf(p.mu2[e][m], L[m], a);
            const float term = p.wd[e] * exp2_hw(-a);
            const float y = term - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        Tv = sum;
    }
    return Tv;
}

// The traced band with its rays compacted: in a thin slab most rays of the
// band pass above or below the voxels (their T is 1), and the rays that do
// meet them would leave most lanes of a warp idle through the walk.  Each
// CTA takes kCompact consecutive band rays of one projection (the band
// order above); phase 1 tests every one against the voxel box with the
// walk's own set-up (the same binary32 operations, so the decision is the
// walk's), stores T = 1 for the misses and appends the others, in order, to
// a queue in shared memory (one aggregated append per warp); phase 2 hands
// the queue out to the warps 32 rays at a time, so every lane walks a ray
// that meets the voxels.  T of a ray does not depend on which thread traces
// it.  The brick map (one byte per 8 x 8 x 16 voxels: 16 KB for 1024^2 x 16
// voxels) is copied into shared memory by every CTA when it fits, so the
// walk's coarse steps read it there; the labels of mixed bricks stay in
// L2 / L1 (the whole label volume of the thin slab is 10 MB, resident in L2).
constexpr int kCompact = 2048;
constexpr int kSmemBricks = 16384;   // largest brick map staged in shared memory

__device__ __forceinline__ bool stage_bricks(const ProjParams &p, uint8_t *sb, int tid)
{
    const DevGeom &g = p.g;
    const int nb = ((g.nx + kBrick - 1) / kBrick) * ((g.ny + kBrick - 1) / kBrick) *
                   ((g.nz + kBrickZ - 1) / kBrickZ);
    if (nb > kSmemBricks) return false;
    const int n16 = nb / 16;   // the map is a cudaMalloc allocation: 16-byte aligned
    for (int i = tid; i < n16; i += 256)
        reinterpret_cast<uint4 *>(sb)[i] = __ldg(reinterpret_cast<const uint4 *>(p.bricks) + i);
    for (int i = n16 * 16 + tid; i < nb; i += 256) sb[i] = __ldg(p.bricks + i);
    return true;
}

__global__ void __launch_bounds__(256)
k_project_compact(const __grid_constant__ ProjParams p, float *__restrict__ T, int r0, int R)
{
    __shared__ int queue[kCompact];
    __shared__ int q_len, q_head;
    __shared__ __align__(16) uint8_t sb[kSmemBricks];
    const DevGeom &g = p.g;
    const int tid = threadIdx.y * 32 + threadIdx.x, lane = threadIdx.x;
    const int kl = blockIdx.z;
    const int k = p.angle0 + kl;
    const int base = (int)blockIdx.x * kCompact;
    if (tid == 0) {
        q_len = 0;
        q_head = 0;
    }
    const bool smem_bricks = stage_bricks(p, sb, tid);
    __syncthreads();
    for (int c = tid; c < kCompact; c += 256) {       // a warp takes 32 consecutive rays
        int iu = 0, iv = 0;
        const bool valid = band_ray(base + c, r0, R, g.n_u, iu, iv);
        float L[kMaxMat];
        const bool hit = valid && trace_ray<true>(p, iu, iv, k, L);
        if (valid && !hit) T[((size_t)k * g.n_v + iv) * g.n_u + iu] = 1.0f;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        int pos = 0;
        if (lane == 0 && m) pos = atomicAdd(&q_len, __popc(m));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (hit) queue[pos + __popc(m & ((1u << lane) - 1u))] = base + c;
    }
    __syncthreads();
    const int n = q_len;
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(&q_head, 32);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= n) break;
        const int i = chunk + lane;
        if (i < n) {
            int iu, iv;
            band_ray(queue[i], r0, R, g.n_u, iu, iv);
            float L[kMaxMat];
            const bool hit = smem_bricks ? trace_ray<false, true>(p, iu, iv, k, L, sb)
                                         : trace_ray<false>(p, iu, iv, k, L);
            T[((size_t)k * g.n_v + iv) * g.n_u + iu] = energy_T(p, hit, L);
        }
    }
}

template <bool EMIT_L>
__global__ void __launch_bounds__(256)
k_project(const __grid_constant__ ProjParams p, float *__restrict__ T, float *__restrict__ Lout, int r0,
          int R)
{
    const DevGeom &g = p.g;
    int iu, iv;
    if (!band_ray(band_t(), r0, R, g.n_u, iu, iv)) return;
    const int kl = blockIdx.z;
    const int k = p.angle0 + kl;
    float L[kMaxMat];
    const bool hit = trace_ray(p, iu, iv, k, L);
    const size_t ray = ((size_t)kl * g.n_v + iv) * g.n_u + iu;
    if (EMIT_L) {
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m)
            if (m < p.n_mat) Lout[ray * p.n_mat + m] = L[m];
        return;
    }
    T[((size_t)k * g.n_v + iv) * g.n_u + iu] = energy_T(p, hit, L);
}

// Value planes of the rows outside the traced band: plane z starts at
// z * stride elements and is filled with v[z].
struct FillPlanes {
    float v[FC_MAX_GROUPS];
    size_t stride;
};

// Rows [a0, a1) and [b0, b1) (a1 <= b0) of projection angle0 + blockIdx.y
// in plane blockIdx.z (VEC: four floats per store) get the value of a ray
// that misses the voxel slab.
template <bool VEC>
__global__ void __launch_bounds__(256)
k_fill_miss_rows(float *__restrict__ T, int n_u, int n_v, int angle0, int a0, int a1, int b0, int b1,
                 const __grid_constant__ FillPlanes f)
{
    const int w = VEC ? 4 : 1;
    const size_t s0 = (size_t)a0 * n_u / w, lo = (size_t)(a1 - a0) * n_u / w;
    const size_t hs = (size_t)b0 * n_u / w, n_fill = lo + (size_t)(b1 - b0) * n_u / w;
    const size_t base = (blockIdx.z * f.stride + (size_t)(angle0 + blockIdx.y) * n_v * n_u) / w;
    const float v = f.v[blockIdx.z];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_fill;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = base + (e < lo ? s0 + e : hs + (e - lo));
        if (VEC)
            reinterpret_cast<float4 *>(T)[i] = make_float4(v, v, v, v);
        else
            T[i] = v;
    }
}

// Rows of [f_lo, f_hi) outside the traced band [r0, r1) (the band lies
// inside [f_lo, f_hi) or is empty).
static void fill_ranges(int r0, int r1, int f_lo, int f_hi, int &a0, int &a1, int &b0, int &b1)
{
    a0 = f_lo;
    a1 = r1 > r0 ? max(f_lo, min(r0, f_hi)) : f_lo;
    b0 = r1 > r0 ? max(a1, min(r1, f_hi)) : f_lo;
    b1 = f_hi;
}

static cudaError_t launch_fill(const ProjParams &p, float *T, int r0, int r1, int f_lo, int f_hi,
                               const FillPlanes &f, int n_planes, cudaStream_t s)
{
    const int n_v = p.g.n_v, n_u = p.g.n_u;
    int a0, a1, b0, b1;
    fill_ranges(r0, r1, f_lo, f_hi, a0, a1, b0, b1);
    const size_t n_fill = (size_t)((a1 - a0) + (b1 - b0)) * n_u;
    if (!n_fill || n_planes <= 0) return cudaSuccess;
    const bool vec = n_u % 4 == 0 && reinterpret_cast<uintptr_t>(T) % 16 == 0 &&
                     (n_planes == 1 || f.stride % 4 == 0);
    const size_t per = vec ? n_fill / 4 : n_fill;
    const size_t want = (per + 256 * 8 - 1) / (256 * 8);
    dim3 grid((unsigned)(want < 1024 ? want : 1024), p.n_angles_launch, n_planes);
    if (vec)
        k_fill_miss_rows<true><<<grid, 256, 0, s>>>(T, n_u, n_v, p.angle0, a0, a1, b0, b1, f);
    else
        k_fill_miss_rows<false><<<grid, 256, 0, s>>>(T, n_u, n_v, p.angle0, a0, a1, b0, b1, f);
    return cudaGetLastError();
}

// Traced band [r0, r1): the rows in [v_hit_lo, v_hit_hi] clipped to the
// detector (r0 = r1 = 0 when no row can meet the slab).
// CTAs of kBandCta rays covering R rows x n_u columns of one projection.
static unsigned band_ctas(int R, int n_u)
{
    return (unsigned)(((long long)R * n_u + kBandCta - 1) / kBandCta);
}

static void project_band(const ProjParams &p, int &r0, int &r1)
{
    const int n_v = p.g.n_v;
    const int lo = max(p.v_hit_lo, 0), hi = min(p.v_hit_hi, n_v - 1);
    r0 = r1 = 0;
    if (lo <= hi) {
        r0 = lo;
        r1 = hi + 1;
    }
}

// Kernels launch_project (T output, fill rows [f_lo, f_hi); f_hi < 0: every
// row) or launch_project_groups starts: the traced band and the fill.
int project_launches(const ProjParams &p, int f_lo, int f_hi)
{
    if (p.n_angles_launch <= 0) return 0;
    int r0, r1;
    project_band(p, r0, r1);
    if (f_hi < 0) {
        f_lo = 0;
        f_hi = p.g.n_v;
    }
    int a0, a1, b0, b1;
    fill_ranges(r0, r1, f_lo, f_hi, a0, a1, b0, b1);
    return (r1 > r0) + ((a1 - a0) + (b1 - b0) > 0);
}

cudaError_t launch_project(const ProjParams &p, float *T, float *L_out, cudaStream_t s, int f_lo,
                           int f_hi)
{
    if (p.n_angles_launch <= 0) return cudaSuccess;
    dim3 block(32, 8);
    if (L_out) {
        dim3 grid(band_ctas(p.g.n_v, p.g.n_u), 1, p.n_angles_launch);
        k_project<true><<<grid, block, 0, s>>>(p, T, L_out, 0, p.g.n_v);
        return cudaGetLastError();
    }
    // Only the rows in [v_hit_lo, v_hit_hi] are traced; the other rows of
    // [f_lo, f_hi) are filled with T = 1 by a store-only kernel (rows outside
    // it are left as they are: a consumer that takes them as 1 without
    // reading them narrows the range).
    int r0, r1;
    project_band(p, r0, r1);
    if (r1 > r0 && p.compact) {
        const long long rays = (long long)(r1 - r0) * p.g.n_u;
        dim3 grid((unsigned)((rays + kCompact - 1) / kCompact), 1, p.n_angles_launch);
        k_project_compact<<<grid, block, 0, s>>>(p, T, r0, r1 - r0);
    } else if (r1 > r0) {
        dim3 grid(band_ctas(r1 - r0, p.g.n_u), 1, p.n_angles_launch);
        k_project<false><<<grid, block, 0, s>>>(p, T, nullptr, r0, r1 - r0);
    }
    FillPlanes f{};
    f.v[0] = 1.0f;
    f.stride = 0;
    if (f_hi < 0) {
        f_lo = 0;
        f_hi = p.g.n_v;
    }
    return launch_fill(p, T, r0, r1, f_lo, f_hi, f, 1, s);
}

// Energy-group primaries (the I_f equation of Sec. II.F split over groups of
// contiguous bins): P_g = sum_{E in g} w D exp(-sum_m mu_m L_m) / sum_E w D,
// a compensated sum per group, written to P + g * grp_stride at the ray's
// absolute position.  Rays that miss the volume give P_g = sum_{E in g} wD.
__global__ void __launch_bounds__(256)
k_project_groups(const __grid_constant__ ProjParams p, float *__restrict__ P, int r0, int R)
{
    const DevGeom &g = p.g;
    int iu, iv;
    if (!band_ray(band_t(), r0, R, g.n_u, iu, iv)) return;
    const int k = p.angle0 + blockIdx.z;
    float L[kMaxMat];
    const bool hit = trace_ray(p, iu, iv, k, L);
    const size_t ray = ((size_t)k * g.n_v + iv) * g.n_u + iu;
    if (!hit) {
        // no attenuation: each group's share of the flood
        for (int gi = 0; gi < p.n_groups; ++gi) P[(size_t)gi * p.grp_stride + ray] = p.grp_flood[gi];
        return;
    }
    int e = 0;
    for (int gi = 0; gi < p.n_groups; ++gi) {
        float sum = 0.0f, comp = 0.0f;
        for (const int e1 = p.grp_end[gi]; e < e1; ++e) {
            float a = 0.0f;
#pragma unroll
            for (int m = 0; m < kMaxMat; ++m) a = fmaf(p.mu2[e][m], L[m], a);
            const float term = p.wd[e] * exp2_hw(-a);
            const float y = term - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        P[(size_t)gi * p.grp_stride + ray] = sum;
    }
}

cudaError_t launch_project_groups(const ProjParams &p, float *P, cudaStream_t s)
{
    if (p.n_angles_launch <= 0) return cudaSuccess;
    dim3 block(32, 8);
    int r0, r1;
    project_band(p, r0, r1);
    if (r1 > r0) {
        dim3 grid(band_ctas(r1 - r0, p.g.n_u), 1, p.n_angles_launch);
        k_project_groups<<<grid, block, 0, s>>>(p, P, r0, r1 - r0);
    }
    FillPlanes f{};
    for (int gi = 0; gi < p.n_groups; ++gi) f.v[gi] = p.grp_flood[gi];
    f.stride = p.grp_stride;
    return launch_fill(p, P, r0, r1, 0, p.g.n_v, f, p.n_groups, s);
}

// Dose estimate, Sec. II.H: for every energy bin E, the sum over the rays of
// the fraction a ray loses in the phantom, 1 - exp(-sum_m mu_m(E) L_m).
// Rays outside the rows [r0, r1) cannot meet the voxel slab and lose nothing,
// so only that band is visited.  Blocks walk tiles of 256 rays of the
// projector's band order in a fixed order; each warp traces its 32 rays,
// stages their path lengths in its own shared slice and then sums
// bins lane, lane + 32, ... over those 32 rays (warp-synchronous: no block
// barrier inside the loop, so a warp with long rays holds up no other).  The
// warps' per-bin sums are folded in a fixed order at the end: the partials
// are reproducible.
static_assert(kMaxMat == 8 && kMaxBins <= 256, "dose kernel: two float4 per ray, 8 bins per lane");

template <int NQ>
__global__ void __launch_bounds__(256)
k_dose_partial(const __grid_constant__ ProjParams p, double *__restrict__ part, int r0, int r1)
{
    __shared__ float4 sL[8][32][2];
    __shared__ double red[8][kMaxBins];
    const DevGeom &g = p.g;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int R = r1 - r0;
    const int tpa = (R * g.n_u + kBandCta - 1) / kBandCta;   // tiles per projection
    const long long n_tiles = (long long)tpa * p.n_angles_launch;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int kl = (int)(t / tpa);
        const int tr = (int)(t % tpa) * kBandCta + w * 32 + lane;
        int iu, iv;
        float L[kMaxMat];
        if (band_ray(tr, r0, R, g.n_u, iu, iv)) {
            trace_ray(p, iu, iv, p.angle0 + kl, L);
        } else {
#pragma unroll
            for (int m = 0; m < kMaxMat; ++m) L[m] = 0.0f;
        }
        sL[w][lane][0] = make_float4(L[0], L[1], L[2], L[3]);
        sL[w][lane][1] = make_float4(L[4], L[5], L[6], L[7]);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = lane + 32 * q;
            if (e < p.n_e) {
                float mu[kMaxMat];
#pragma unroll
                for (int m = 0; m < kMaxMat; ++m) mu[m] = p.mu2[e][m];
                float sum = 0.0f, comp = 0.0f;
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    const float4 a0 = sL[w][r][0], a1 = sL[w][r][1];
                    float a = mu[0] * a0.x;
                    a = fmaf(mu[1], a0.y, a);
                    a = fmaf(mu[2], a0.z, a);
                    a = fmaf(mu[3], a0.w, a);
                    a = fmaf(mu[4], a1.x, a);
                    a = fmaf(mu[5], a1.y, a);
                    a = fmaf(mu[6], a1.z, a);
                    a = fmaf(mu[7], a1.w, a);
                    const float y = (1.0f - exp2f(-a)) - comp;
                    const float s2 = sum + y;
                    comp = (s2 - sum) - y;
                    sum = s2;
                }
                acc[q] += (double)sum;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (lane + 32 * q < p.n_e) red[w][lane + 32 * q] = acc[q];
    __syncthreads();
    const int tid = w * 32 + lane;
    if (tid < p.n_e) {
        double a = 0.0;
        for (int ww = 0; ww < 8; ++ww) a += red[ww][tid];
        part[(size_t)blockIdx.x * p.n_e + tid] = a;
    }
}

// Voxels per label (for the phantom mass): one ballot per label and warp.
__global__ void __launch_bounds__(256)
k_label_count(const uint8_t *__restrict__ lab, size_t n, int n_mat, unsigned long long *count)
{
    __shared__ unsigned int c[kMaxMat];
    if (threadIdx.x < kMaxMat) c[threadIdx.x] = 0;
    __syncthreads();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t n_pad = (n + 31) / 32 * 32;   // every lane of a warp takes each ballot
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x % 32 < n_pad;
         i += stride) {
        const int v = i < n ? lab[i] : -1;
        for (int m = 0; m < n_mat; ++m) {
            const unsigned int b = __ballot_sync(0xffffffffu, v == m);
            if (threadIdx.x % 32 == 0 && b) atomicAdd(&c[m], (unsigned int)__popc(b));
        }
    }
    __syncthreads();
    if (threadIdx.x < n_mat && c[threadIdx.x])
        atomicAdd(&count[threadIdx.x], (unsigned long long)c[threadIdx.x]);
}

// Sum over the partial rows for bin blockIdx.x: thread t takes rows t,
// t + 256, ..., then a fixed tree (reproducible); the sum goes to out[e].
__global__ void __launch_bounds__(256)
k_dose_fold(const __grid_constant__ DoseParams d, const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double s[256];
    const int e = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < d.n_part; b += 256) a += part[(size_t)b * d.n_e + e];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[e] = s[0];
}

// D0(E) = E (mu_en/mu)_w(E) sum_i (1 - exp(-mu_i(E) x_i)) / (N_i M) and
// Dp = sum_E phi(E) D0(E) (Sec. II.H); out = [D0(E_0) .. D0(E_{n-1}), Dp],
// the sums over rays already in out[0 .. n_e).
__global__ void __launch_bounds__(256)
k_dose_final(const __grid_constant__ DoseParams d, const unsigned long long *__restrict__ count,
             double *__restrict__ out)
{
    __shared__ double s[kMaxBins];
    const int e = threadIdx.x;
    double mass = 0.0;
    for (int m = 0; m < d.n_mat; ++m) mass += (double)count[m] * d.rho[m];
    mass *= d.voxel_cm3;
    if (e < d.n_e) {
        const double d0 = kGyGramPerKev * d.e_kev[e] * d.muen[e] * out[e] / (d.n_rays * mass);
        out[e] = d0;
        s[e] = d.phi[e] * d0;
    }
    __syncthreads();
    if (e == 0) {
        double dp = 0.0;
        for (int i = 0; i < d.n_e; ++i) dp += s[i];
        out[d.n_e] = dp;
    }
}

template <int NQ>
static int dose_grid(long long tiles)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dose_partial<NQ>, 256, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1, sms = sms > 0 ? sms : 1;
    long long n = (long long)sms * per_sm;
    n = n < kDoseBlocks ? n : kDoseBlocks;
    return (int)(tiles < n ? tiles : n);
}

int dose_blocks(const ProjParams &p)
{
    int r0, r1;
    project_band(p, r0, r1);
    long long tiles = (long long)band_ctas(r1 - r0, p.g.n_u) * p.n_angles_launch;
    tiles = tiles > 0 ? tiles : 1;   // one block writes zero partials
    if (p.n_e <= 32) return dose_grid<1>(tiles);
    if (p.n_e <= 64) return dose_grid<2>(tiles);
    if (p.n_e <= 128) return dose_grid<4>(tiles);
    return dose_grid<8>(tiles);
}

cudaError_t launch_dose(const ProjParams &p, const DoseParams &d, double *part,
                        unsigned long long *count, double *out, cudaStream_t s)
{
    const size_t nvox = (size_t)p.g.nx * p.g.ny * p.g.nz;
    cudaError_t e = cudaMemsetAsync(count, 0, kMaxMat * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_label_count<<<sm_count() * 4, 256, 0, s>>>(p.labels, nvox, d.n_mat, count);
    const dim3 blk(32, 8);
    int r0, r1;
    project_band(p, r0, r1);
    if (d.n_e <= 32)
        k_dose_partial<1><<<d.n_part, blk, 0, s>>>(p, part, r0, r1);
    else if (d.n_e <= 64)
        k_dose_partial<2><<<d.n_part, blk, 0, s>>>(p, part, r0, r1);
    else if (d.n_e <= 128)
        k_dose_partial<4><<<d.n_part, blk, 0, s>>>(p, part, r0, r1);
    else
        k_dose_partial<8><<<d.n_part, blk, 0, s>>>(p, part, r0, r1);
    k_dose_fold<<<d.n_e, 256, 0, s>>>(d, part, out);
    k_dose_final<<<1, 256, 0, s>>>(d, count, out);
    return cudaGetLastError();
}

// One warp per 8x8x16 brick (lane l takes voxels l, l + 32, ... of the
// brick, clipped to the grid): its single label, or kMixed; flags any label
// >= n_mat.
__global__ void k_brick_map(const uint8_t *__restrict__ lab, uint8_t *__restrict__ bricks, int nx,
                            int ny, int nz, int n_mat, unsigned int *bad)
{
    const int nbx = (nx + kBrick - 1) / kBrick, nby = (ny + kBrick - 1) / kBrick;
    const int nbz = (nz + kBrickZ - 1) / kBrickZ;
    const int nb = nbx * nby * nbz;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += warps) {
        const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
        const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrickZ;
        const int first = lab[((size_t)z0 * ny + y0) * nx + x0];
        bool uniform = true, badlab = false;
        for (int v = lane; v < kBrick * kBrick * kBrickZ; v += 32) {
            const int x = x0 + v % kBrick, y = y0 + (v / kBrick) % kBrick, z = z0 + v / (kBrick * kBrick);
            if (x < nx && y < ny && z < nz) {
                const int l = lab[((size_t)z * ny + y) * nx + x];
                uniform = uniform && l == first;
                badlab = badlab || l >= n_mat;
            }
        }
        uniform = __all_sync(0xffffffffu, uniform);
        badlab = __any_sync(0xffffffffu, badlab);
        if (lane == 0) {
            if (badlab) atomicOr(bad, 1u);
            bricks[b] = uniform ? (uint8_t)first : (uint8_t)kMixed;
        }
    }
}

// Labels [nz][ny][nx] -> [ny][nx][nz] (z fastest), one output byte per thread.
__global__ void __launch_bounds__(256) k_labels_zfast(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                                      int nx, int ny, int nz)
{
    const long long n = (long long)nx * ny * nz;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n;
         o += (long long)gridDim.x * blockDim.x) {
        const long long col = o / nz;            // y nx + x
        const int z = (int)(o - col * nz);
        dst[o] = src[(long long)z * nx * ny + col];
    }
}

cudaError_t launch_labels_zfast(const uint8_t *labels, uint8_t *labels_zf, int nx, int ny, int nz,
                                cudaStream_t s)
{
    k_labels_zfast<<<sm_count() * 8, 256, 0, s>>>(labels, labels_zf, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_brick_map(const uint8_t *labels, uint8_t *bricks, int nx, int ny, int nz,
                             int n_mat, unsigned int *bad, cudaStream_t s)
{
    const int nb = ((nx + kBrick - 1) / kBrick) * ((ny + kBrick - 1) / kBrick) *
                   ((nz + kBrickZ - 1) / kBrickZ);
    const int blocks = (nb + 3) / 4 < sm_count() * 16 ? (nb + 3) / 4 : sm_count() * 16;   // 4 warps per block
    k_brick_map<<<blocks, 128, 0, s>>>(labels, bricks, nx, ny, nz, n_mat, bad);
    return cudaGetLastError();
}

}  // namespace fc

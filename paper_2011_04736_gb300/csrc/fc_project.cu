// Polyenergetic cone-beam projector (paper Sec. II.F "Raytracing" and the
// energy-weighting equation I_f = sum_E phi(E) eta(E) I(E)).
//
// One thread per detector pixel ray.  The ray is traversed voxel by voxel
// (incremental Siddon / Amanatides-Woo order) and the path length inside
// each material is accumulated run by run: a length is added only when the
// material label changes, so binary32 rounding enters once per material
// transition instead of once per voxel.  The per-material lengths stay in
// registers and feed the energy integral
//     T = sum_E (w D)_E exp(-sum_m mu_m(E) L_m)        (w D normalised)
// evaluated with exp2 and a compensated (Kahan) sum over the energy bins.
// A warp covers 32 consecutive pixels of one detector row, so the T stores
// are coalesced 128-byte rows.
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

struct AxisWalk {
    float t0;    // first crossing
    float dt;    // spacing of crossings
    int step;    // index increment in the padded volume
};

__device__ __forceinline__ AxisWalk setup_axis(float A, float d, float inv_d, float lo, float vox,
                                               int i, int stride, float t_in)
{
    AxisWalk w;
    if (d > 0.0f) {
        w.t0 = (lo + (float)(i + 1) * vox - A) * inv_d;
        w.dt = vox * inv_d;
        w.step = stride;
    } else if (d < 0.0f) {
        w.t0 = (lo + (float)i * vox - A) * inv_d;
        w.dt = -vox * inv_d;
        w.step = -stride;
    } else {
        w.t0 = INFINITY;
        w.dt = 0.0f;
        w.step = 0;
    }
    w.t0 = fmaxf(w.t0, t_in);
    return w;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

}  // namespace

template <bool EMIT_L>
__global__ void __launch_bounds__(256)
k_project(const __grid_constant__ ProjParams p, float *__restrict__ T, float *__restrict__ Lout)
{
    const DevGeom &g = p.g;
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * blockDim.y + threadIdx.y;
    const int kl = blockIdx.z;
    if (iu >= g.n_u || iv >= g.n_v) return;
    const int k = p.angle0 + kl;

    float L[kMaxMat];
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
        if (hit) {
            const float px = fmaf(t_in, dx, Ax), py = fmaf(t_in, dy, Ay), pz = fmaf(t_in, dz, Az);
            const int ix = clampi((int)floorf((px - g.lox) * g.idx), 0, g.nx - 1);
            const int iy = clampi((int)floorf((py - g.loy) * g.idy), 0, g.ny - 1);
            const int iz = clampi((int)floorf((pz - g.loz) * g.idz), 0, g.nz - 1);
            const int pnx = g.nx + 2, pnxy = (g.nx + 2) * (g.ny + 2);
            AxisWalk wx = setup_axis(Ax, dx, ix_, g.lox, g.dx, ix, 1, t_in);
            AxisWalk wy = setup_axis(Ay, dy, iy_, g.loy, g.dy, iy, pnx, t_in);
            AxisWalk wz = setup_axis(Az, dz, iz_, g.loz, g.dz, iz, pnxy, t_in);
            float tx = wx.t0, ty = wy.t0, tz = wz.t0;
            float cx = 0.0f, cy = 0.0f, cz = 0.0f;
            int idx = (iz + 1) * pnxy + (iy + 1) * pnx + (ix + 1);
            int cur = __ldg(p.labels + idx);
            float t_run = t_in;
            // The padded volume has a one-voxel border labelled kBorder, so
            // the walk ends when it steps into the border.  Each pass moves
            // at least one index one voxel along the ray, so the border is
            // reached within nx + ny + nz + 3 passes; the pass budget only
            // guards against non-finite geometry.
            bool open = true;
            for (int budget = g.nx + g.ny + g.nz + 3; budget > 0; --budget) {
                const float tn = fminf(tx, fminf(ty, tz));
                if (tx == tn) { idx += wx.step; cx += 1.0f; tx = fmaf(cx, wx.dt, wx.t0); }
                if (ty == tn) { idx += wy.step; cy += 1.0f; ty = fmaf(cy, wy.dt, wy.t0); }
                if (tz == tn) { idx += wz.step; cz += 1.0f; tz = fmaf(cz, wz.dt, wz.t0); }
                const int lab = __ldg(p.labels + idx);
                if (lab != cur) {
                    add_run(L, cur, tn - t_run);
                    if (lab == kBorder) { open = false; break; }
                    t_run = tn;
                    cur = lab;
                }
            }
            if (open) add_run(L, cur, t_out - t_run);
        }
    }

    const size_t ray = ((size_t)kl * g.n_v + iv) * g.n_u + iu;
    if (EMIT_L) {
#pragma unroll
        for (int m = 0; m < kMaxMat; ++m)
            if (m < p.n_mat) Lout[ray * p.n_mat + m] = L[m];
        return;
    }
    float Tv = 1.0f;
    if (hit) {
        float sum = 0.0f, comp = 0.0f;
        for (int e = 0; e < p.n_e; ++e) {
            float a = 0.0f;
#pragma unroll
            for (int m = 0; m < kMaxMat; ++m) a = fmaf(p.mu2[e][m], L[m], a);
            const float term = p.wd[e] * exp2f(-a);
            const float y = term - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        Tv = sum;
    }
    T[((size_t)k * g.n_v + iv) * g.n_u + iu] = Tv;
}

cudaError_t launch_project(const ProjParams &p, float *T, float *L_out, cudaStream_t s)
{
    if (p.n_angles_launch <= 0) return cudaSuccess;
    dim3 block(32, 8);
    dim3 grid((p.g.n_u + 31) / 32, (p.g.n_v + 7) / 8, p.n_angles_launch);
    if (L_out)
        k_project<true><<<grid, block, 0, s>>>(p, T, L_out);
    else
        k_project<false><<<grid, block, 0, s>>>(p, T, L_out);
    return cudaGetLastError();
}

// Copy labels [nz][ny][nx] into the padded [nz + 2][ny + 2][nx + 2] layout
// with a kBorder frame, flagging any label >= n_mat.
__global__ void k_pad_labels(const uint8_t *__restrict__ lab, uint8_t *__restrict__ pad, int nx,
                             int ny, int nz, int n_mat, unsigned int *bad)
{
    const size_t px = nx + 2, py = ny + 2, n = px * py * (size_t)(nz + 2);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % px) - 1;
        const int y = (int)((i / px) % py) - 1;
        const int z = (int)(i / (px * py)) - 1;
        uint8_t v = kBorder;
        if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz) {
            v = lab[((size_t)z * ny + y) * nx + x];
            if (v >= n_mat) atomicOr(bad, 1u);
        }
        pad[i] = v;
    }
}

cudaError_t launch_pad_labels(const uint8_t *labels, uint8_t *padded, int nx, int ny, int nz,
                              int n_mat, unsigned int *bad, cudaStream_t s)
{
    k_pad_labels<<<152 * 4, 256, 0, s>>>(labels, padded, nx, ny, nz, n_mat, bad);
    return cudaGetLastError();
}

}  // namespace fc

/*
 * FP64 CPU oracle for the fastCAT CBCT hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests, the package smoke check and the benchmark's CPU-baseline leg
 * use this code.  It shares nothing with the CUDA library: every quantity
 * is recomputed here from its definition, in double precision, with plain
 * loops in the order the definitions give.  OpenMP only splits independent
 * output elements across threads; it does not change any arithmetic.
 *
 * Sections of the paper (O'Connell & Bazalova-Carter, fastCAT) followed:
 *   - Sec. II.F "Raytracing": a projection is the sum of attenuation along
 *     each source-to-pixel ray; one forward projection per energy.  Here the
 *     per-material path lengths L_m of each ray are computed exactly by
 *     Siddon's parametric method (all plane crossings, merged, voxel of each
 *     segment from its midpoint), and reused for every energy.
 *   - Sec. II.F, Eq. for I_f: the detected signal is the sum over energies of
 *     fluence x detector efficiency x intensity; intensity relative to the
 *     flood field is exp(-sum_m mu_m(E) L_m).
 *   - Sec. II.G: optical spread (and scatter) are convolutions of the
 *     intensity profile; FDK reconstruction [Feldkamp 1984] and HU
 *     normalisation on the water region.
 * Function headers name the step they implement.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double sad, sdd;
    int32_t n_u, n_v;
    double du, dv;
    int32_t n_angles;
    double theta0, arc;
    int32_t nx, ny, nz;
    double dx, dy, dz;
} orc_geom;

/* ------------------------------------------------------------------ */
/* Geometry: source and pixel centre of ray (k, iv, iu), volume frame.  */
/* ------------------------------------------------------------------ */
static void ray_endpoints(const orc_geom *g, int k, int iv, int iu,
                          double S[3], double P[3])
{
    double th = g->theta0 + g->arc * (double)k / (double)g->n_angles;
    double c = cos(th), s = sin(th);
    double u = ((double)iu - (g->n_u - 1) / 2.0) * g->du;
    double v = ((double)iv - (g->n_v - 1) / 2.0) * g->dv;
    double back = g->sdd - g->sad;
    S[0] = g->sad * c;  S[1] = g->sad * s;  S[2] = 0.0;
    /* detector centre -(SDD-SAD)(c, s, 0); u axis (-s, c, 0); v axis z */
    P[0] = -back * c - u * s;
    P[1] = -back * s + u * c;
    P[2] = v;
}

/* ------------------------------------------------------------------ */
/* Siddon (1985): exact radiological path per material.               */
/* X(a) = S + a (P - S), a in [0, 1].                                   */
/* ------------------------------------------------------------------ */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Path length (cm) of the segment S->P inside each material label.
 * L[0..n_mat-1] is overwritten.  Returns the total intersected length. */
double orc_siddon(const orc_geom *g, const uint8_t *lab, int n_mat,
                  const double S[3], const double P[3], double *L)
{
    const int N[3] = {g->nx, g->ny, g->nz};
    const double d[3] = {g->dx, g->dy, g->dz};
    double lo[3], D[3];
    double amin = 0.0, amax = 1.0;
    for (int m = 0; m < n_mat; ++m) L[m] = 0.0;
    for (int a = 0; a < 3; ++a) {
        lo[a] = -0.5 * N[a] * d[a];
        D[a] = P[a] - S[a];
        if (D[a] != 0.0) {
            double a0 = (lo[a] - S[a]) / D[a];
            double a1 = (lo[a] + N[a] * d[a] - S[a]) / D[a];
            double lo_a = a0 < a1 ? a0 : a1, hi_a = a0 < a1 ? a1 : a0;
            if (lo_a > amin) amin = lo_a;
            if (hi_a < amax) amax = hi_a;
        } else if (S[a] < lo[a] || S[a] >= lo[a] + N[a] * d[a]) {
            return 0.0; /* parallel to this slab and outside it */
        }
    }
    if (amin >= amax) return 0.0;
    const double len = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    /* every plane crossing strictly inside (amin, amax), plus the ends */
    int cap = N[0] + N[1] + N[2] + 8;
    double *al = (double *)malloc(sizeof(double) * (size_t)cap);
    int n = 0;
    al[n++] = amin;
    al[n++] = amax;
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.0) continue;
        for (int i = 0; i <= N[a]; ++i) {
            double av = (lo[a] + i * d[a] - S[a]) / D[a];
            if (av > amin && av < amax) al[n++] = av;
        }
    }
    qsort(al, (size_t)n, sizeof(double), cmp_double);
    double total = 0.0;
    for (int j = 0; j + 1 < n; ++j) {
        double a0 = al[j], a1 = al[j + 1];
        if (a1 <= a0) continue; /* coincident crossings: zero-length segment */
        double am = 0.5 * (a0 + a1);
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            double x = S[a] + am * D[a];
            int i = (int)floor((x - lo[a]) / d[a]);
            if (i < 0) i = 0;
            if (i > N[a] - 1) i = N[a] - 1;
            idx[a] = i;
        }
        int m = lab[((size_t)idx[2] * N[1] + idx[1]) * N[0] + idx[0]];
        double seg = (a1 - a0) * len;
        if (m < n_mat) L[m] += seg;
        total += seg;
    }
    free(al);
    return total;
}

/* Voxels crossed by the segment S->P and their path lengths (Siddon, as in
 * orc_siddon).  Writes up to cap (index, length) pairs; returns the count. */
static int siddon_voxels(const orc_geom *g, const double S[3], const double P[3], int cap,
                         int64_t *vidx, double *vlen, double *al)
{
    const int N[3] = {g->nx, g->ny, g->nz};
    const double d[3] = {g->dx, g->dy, g->dz};
    double lo[3], D[3];
    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 3; ++a) {
        lo[a] = -0.5 * N[a] * d[a];
        D[a] = P[a] - S[a];
        if (D[a] != 0.0) {
            double a0 = (lo[a] - S[a]) / D[a];
            double a1 = (lo[a] + N[a] * d[a] - S[a]) / D[a];
            double lo_a = a0 < a1 ? a0 : a1, hi_a = a0 < a1 ? a1 : a0;
            if (lo_a > amin) amin = lo_a;
            if (hi_a < amax) amax = hi_a;
        } else if (S[a] < lo[a] || S[a] >= lo[a] + N[a] * d[a]) {
            return 0;
        }
    }
    if (amin >= amax) return 0;
    const double len = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    int n = 0;
    al[n++] = amin;
    al[n++] = amax;
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.0) continue;
        for (int i = 0; i <= N[a]; ++i) {
            double av = (lo[a] + i * d[a] - S[a]) / D[a];
            if (av > amin && av < amax) al[n++] = av;
        }
    }
    qsort(al, (size_t)n, sizeof(double), cmp_double);
    int out = 0;
    for (int j = 0; j + 1 < n && out < cap; ++j) {
        double a0 = al[j], a1 = al[j + 1];
        if (a1 <= a0) continue;
        double am = 0.5 * (a0 + a1);
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            double x = S[a] + am * D[a];
            int i = (int)floor((x - lo[a]) / d[a]);
            if (i < 0) i = 0;
            if (i > N[a] - 1) i = N[a] - 1;
            idx[a] = i;
        }
        vidx[out] = ((int64_t)idx[2] * N[1] + idx[1]) * N[0] + idx[0];
        vlen[out] = (a1 - a0) * len;
        ++out;
    }
    return out;
}

/* Sparse ray x voxel path-length matrix of all pixel rays of angles
 * [a0, a0 + na), row r = ((k - a0) n_v + iv) n_u + iu, in CSR form: row r
 * holds entries rowptr[r] .. rowptr[r + 1].  Each row has room for
 * nx + ny + nz + 2 entries (cap of a ray); the arrays must hold
 * nrays * cap entries.  Returns the total number of entries. */
int64_t orc_path_matrix(const orc_geom *g, int a0, int na, int64_t *rowptr, int64_t *col,
                        double *val)
{
    const long nrays = (long)na * g->n_v * g->n_u;
    const int cap = g->nx + g->ny + g->nz + 2;
    int *cnt = (int *)malloc(sizeof(int) * (size_t)nrays);
#pragma omp parallel
    {
        double *al = (double *)malloc(sizeof(double) * (size_t)(cap + 8));
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; ++r) {
            int iu = (int)(r % g->n_u);
            int iv = (int)((r / g->n_u) % g->n_v);
            int k = a0 + (int)(r / ((long)g->n_u * g->n_v));
            double S[3], P[3];
            ray_endpoints(g, k, iv, iu, S, P);
            cnt[r] = siddon_voxels(g, S, P, cap, col + r * cap, val + r * cap, al);
        }
        free(al);
    }
    /* compact the fixed-stride rows into CSR */
    int64_t pos = 0;
    for (long r = 0; r < nrays; ++r) {
        rowptr[r] = pos;
        for (int j = 0; j < cnt[r]; ++j) {
            col[pos] = col[r * cap + j];
            val[pos] = val[r * cap + j];
            ++pos;
        }
    }
    rowptr[nrays] = pos;
    free(cnt);
    return pos;
}

/* Path lengths of pixel ray (k, iv, iu). */
double orc_ray_lengths(const orc_geom *g, const uint8_t *lab, int n_mat,
                       int k, int iv, int iu, double *L)
{
    double S[3], P[3];
    ray_endpoints(g, k, iv, iu, S, P);
    return orc_siddon(g, lab, n_mat, S, P, L);
}

/* Energy integral (Sec. II.F): T = sum_E w D exp(-sum_m mu L) / sum_E w D.
 * mu is [n_e][n_mat]. */
double orc_energy_sum(int n_e, int n_mat, const double *w, const double *D,
                      const double *mu, const double *L)
{
    double num = 0.0, den = 0.0;
    for (int e = 0; e < n_e; ++e) {
        double s = 0.0;
        for (int m = 0; m < n_mat; ++m) s += mu[(size_t)e * n_mat + m] * L[m];
        num += w[e] * D[e] * exp(-s);
        den += w[e] * D[e];
    }
    return num / den;
}

/* Primary transmission T[k][iv][iu] for angles [a0, a0 + na). */
void orc_project_T(const orc_geom *g, const uint8_t *lab, int n_mat,
                   int n_e, const double *w, const double *D, const double *mu,
                   int a0, int na, double *T)
{
    const long nrays = (long)na * g->n_v * g->n_u;
#pragma omp parallel
    {
        double *L = (double *)malloc(sizeof(double) * (size_t)n_mat);
#pragma omp for schedule(dynamic, 256)
        for (long r = 0; r < nrays; ++r) {
            int iu = (int)(r % g->n_u);
            int iv = (int)((r / g->n_u) % g->n_v);
            int k = a0 + (int)(r / ((long)g->n_u * g->n_v));
            orc_ray_lengths(g, lab, n_mat, k, iv, iu, L);
            T[r] = orc_energy_sum(n_e, n_mat, w, D, mu, L);
        }
        free(L);
    }
}

/* Sampled rays: rays[3*i + 0..2] = (k, iv, iu). Writes L[i][n_mat], T[i]. */
void orc_rays(const orc_geom *g, const uint8_t *lab, int n_mat,
              int n_e, const double *w, const double *D, const double *mu,
              long n, const int32_t *rays, double *Lout, double *T)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) {
        double *L = Lout + (size_t)i * n_mat;
        orc_ray_lengths(g, lab, n_mat, rays[3 * i], rays[3 * i + 1], rays[3 * i + 2], L);
        T[i] = orc_energy_sum(n_e, n_mat, w, D, mu, L);
    }
}

/* ------------------------------------------------------------------ */
/* Detector optical spread + scatter (Sec. II.E, II.G).               */
/* Sampled Gaussian g[j] ~ exp(-j^2 / 2 sigma^2), |j| <= ceil(4 sigma),  */
/* normalised to sum 1; separable, clamp-to-edge.                     */
/* ------------------------------------------------------------------ */
static int gauss_taps(double sigma, double **taps)
{
    int R = (int)ceil(4.0 * sigma);
    if (sigma <= 0.0) R = 0;
    double *g = (double *)malloc(sizeof(double) * (size_t)(2 * R + 1));
    double s = 0.0;
    for (int j = -R; j <= R; ++j) {
        g[j + R] = (R == 0) ? 1.0 : exp(-(double)j * j / (2.0 * sigma * sigma));
        s += g[j + R];
    }
    for (int j = 0; j < 2 * R + 1; ++j) g[j] /= s;
    *taps = g;
    return R;
}

/* out = G_sigma (x) in over each [nv][nu] image (u pass, then v pass). */
void orc_gauss_blur(const double *in, int nimg, int nv, int nu, double sigma,
                    double *out)
{
    double *g;
    int R = gauss_taps(sigma, &g);
    size_t plane = (size_t)nv * nu;
#pragma omp parallel
    {
        double *tmp = (double *)malloc(sizeof(double) * plane);
#pragma omp for
        for (int im = 0; im < nimg; ++im) {
            const double *src = in + im * plane;
            double *dst = out + im * plane;
            for (int v = 0; v < nv; ++v)
                for (int u = 0; u < nu; ++u) {
                    double acc = 0.0;
                    for (int j = -R; j <= R; ++j) {
                        int uu = u + j;
                        if (uu < 0) uu = 0;
                        if (uu > nu - 1) uu = nu - 1;
                        acc += g[j + R] * src[(size_t)v * nu + uu];
                    }
                    tmp[(size_t)v * nu + u] = acc;
                }
            for (int v = 0; v < nv; ++v)
                for (int u = 0; u < nu; ++u) {
                    double acc = 0.0;
                    for (int j = -R; j <= R; ++j) {
                        int vv = v + j;
                        if (vv < 0) vv = 0;
                        if (vv > nv - 1) vv = nv - 1;
                        acc += g[j + R] * tmp[(size_t)vv * nu + u];
                    }
                    dst[(size_t)v * nu + u] = acc;
                }
        }
        free(tmp);
    }
    free(g);
}

/* Detected intensity I = N0 (G_psf (x) T + SPR * G_scatter (x) T). */
void orc_intensity(const double *T, int nimg, int nv, int nu, double sig_psf,
                   double sig_sc, double spr, double n0, double *I)
{
    size_t n = (size_t)nimg * nv * nu;
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    orc_gauss_blur(T, nimg, nv, nu, sig_psf, a);
    orc_gauss_blur(T, nimg, nv, nu, sig_sc, b);
    for (size_t i = 0; i < n; ++i) I[i] = n0 * (a[i] + spr * b[i]);
    free(a);
    free(b);
}

/* ------------------------------------------------------------------ */
/* FDK [Feldkamp, Davis, Kress 1984] as cited in Sec. II.G.            */
/* ------------------------------------------------------------------ */

/* Log + cosine weight: q = ln(I_flood / max(K, 1)) * SAD / sqrt(SAD^2 +
 * u_i^2 + v_i^2), with (u_i, v_i) the pixel rescaled to the isocentre. */
void orc_fdk_weight(const orc_geom *g, const double *counts, int na,
                    double i_flood, double *q)
{
    const double mag = g->sad / g->sdd;
#pragma omp parallel for
    for (int k = 0; k < na; ++k)
        for (int iv = 0; iv < g->n_v; ++iv)
            for (int iu = 0; iu < g->n_u; ++iu) {
                size_t i = ((size_t)k * g->n_v + iv) * g->n_u + iu;
                double ui = ((double)iu - (g->n_u - 1) / 2.0) * g->du * mag;
                double vi = ((double)iv - (g->n_v - 1) / 2.0) * g->dv * mag;
                double K = counts[i] > 1.0 ? counts[i] : 1.0;
                double p = log(i_flood / K);
                q[i] = p * g->sad / sqrt(g->sad * g->sad + ui * ui + vi * vi);
            }
}

/* Ram-Lak row filter, sampling interval tau (cm at the isocentre):
 * out[i] = tau * sum_j h[i - j] q[j], h[0] = 1 / (4 tau^2),
 * h[n odd] = -1 / (pi^2 n^2 tau^2), h[n even, n != 0] = 0; zero padding. */
void orc_ramp_filter(const double *q, int nrows, int nu, double tau, double *out)
{
#pragma omp parallel for
    for (int r = 0; r < nrows; ++r)
        for (int i = 0; i < nu; ++i) {
            double acc = 0.0;
            for (int j = 0; j < nu; ++j) {
                int n = i - j;
                double h;
                if (n == 0) h = 1.0 / (4.0 * tau * tau);
                else if (n % 2 != 0) h = -1.0 / (M_PI * M_PI * (double)n * n * tau * tau);
                else h = 0.0;
                acc += h * q[(size_t)r * nu + j];
            }
            out[(size_t)r * nu + i] = tau * acc;
        }
}

/* Bilinear sample of image [nv][nu] at fractional (fu, fv); zero outside. */
static double bilinear(const double *img, int nv, int nu, double fu, double fv)
{
    int u0 = (int)floor(fu), v0 = (int)floor(fv);
    double au = fu - u0, av = fv - v0;
    double acc = 0.0;
    for (int dv = 0; dv <= 1; ++dv)
        for (int du = 0; du <= 1; ++du) {
            int u = u0 + du, v = v0 + dv;
            if (u < 0 || u >= nu || v < 0 || v >= nv) continue;
            double wgt = (du ? au : 1.0 - au) * (dv ? av : 1.0 - av);
            acc += wgt * img[(size_t)v * nu + u];
        }
    return acc;
}

/* Voxel-driven FDK backprojection of filtered rows f[k][iv][iu]:
 * mu(x) = 1/2 * (arc / N) * sum_k (SAD / U)^2 * f_k(u(x), v(x)),
 * U = SAD - x.(cos, sin, 0); detector coordinates u = SDD (x.e_u) / U,
 * v = SDD z / U. */
void orc_backproject(const orc_geom *g, const double *f, double *vol)
{
    const size_t plane = (size_t)g->n_v * g->n_u;
    const double scale = 0.5 * g->arc / g->n_angles;
#pragma omp parallel for collapse(2)
    for (int iz = 0; iz < g->nz; ++iz)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                double x = ((double)ix - (g->nx - 1) / 2.0) * g->dx;
                double y = ((double)iy - (g->ny - 1) / 2.0) * g->dy;
                double z = ((double)iz - (g->nz - 1) / 2.0) * g->dz;
                double acc = 0.0;
                for (int k = 0; k < g->n_angles; ++k) {
                    double th = g->theta0 + g->arc * (double)k / g->n_angles;
                    double c = cos(th), s = sin(th);
                    double U = g->sad - (x * c + y * s);
                    double ru = -x * s + y * c;
                    double u = g->sdd * ru / U, v = g->sdd * z / U;
                    double fu = u / g->du + (g->n_u - 1) / 2.0;
                    double fv = v / g->dv + (g->n_v - 1) / 2.0;
                    double wgt = (g->sad / U) * (g->sad / U);
                    acc += wgt * bilinear(f + k * plane, g->n_v, g->n_u, fu, fv);
                }
                vol[((size_t)iz * g->ny + iy) * g->nx + ix] = scale * acc;
            }
}

/* Full FDK of counts[k][iv][iu] (all n_angles) to vol[z][y][x] (1/cm). */
void orc_fdk(const orc_geom *g, const double *counts, double i_flood, double *vol)
{
    size_t n = (size_t)g->n_angles * g->n_v * g->n_u;
    double *q = (double *)malloc(sizeof(double) * n);
    double *f = (double *)malloc(sizeof(double) * n);
    orc_fdk_weight(g, counts, g->n_angles, i_flood, q);
    orc_ramp_filter(q, g->n_angles * g->n_v, g->n_u, g->du * g->sad / g->sdd, f);
    orc_backproject(g, f, vol);
    free(q);
    free(f);
}

/* Number of OpenMP threads the parallel loops above use. */
int orc_omp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

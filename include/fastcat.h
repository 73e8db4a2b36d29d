/*
 * fastcat.h -- C ABI of the GB300 (sm_103a) fastCAT CBCT hot path.
 *
 * The operations follow O'Connell & Bazalova-Carter, "FastCAT: Fast Cone
 * Beam CT (CBCT) Simulation" (arXiv 2011.04736):
 *   Sec. II.F  Raytracing: line integrals of attenuation along every
 *              source-to-pixel ray, one projection per energy, combined by
 *              the energy-weighting equation I_f = sum_E phi(E) eta(E) I(E).
 *   Sec. II.E/G  detector optical spread and scatter added to the intensity
 *              profiles; Poisson noise from the particle counts (Sec. II.H,
 *              fluence equation H = N / (A / A_p)); conversion back to
 *              projections with the flood field; FDK reconstruction
 *              [Feldkamp 1984]; HU normalised on the water region.
 *
 * Conventions (all lengths in cm, angles in rad):
 *   angle k:   theta_k = theta0 + arc * k / n_angles
 *   source:    SAD * (cos theta, sin theta, 0)
 *   detector:  centre -(SDD - SAD) * (cos, sin, 0), u axis (-sin, cos, 0),
 *              v axis (0, 0, 1); pixel (iu, iv) centre at
 *              ((iu - (n_u - 1) / 2) du, (iv - (n_v - 1) / 2) dv)
 *   volume:    centred at the origin, voxel (ix, iy, iz) centre at
 *              ((ix - (nx - 1) / 2) dx, ...), voxel intervals half-open
 *   layouts:   projections float [angle][v][u] (u fastest);
 *              volumes [z][y][x] (x fastest); labels uint8 [z][y][x]
 *
 * Every call returns FC_OK (0) or a negative FC_E* code; fc_last_error()
 * then returns a message for the calling thread.  Memory passed in is owned
 * by the caller and only read (inputs) or written (outputs) during the call;
 * the library copies what it keeps.  A handle must not be used by two
 * threads at once.  All device work runs on the caller's stream (a
 * cudaStream_t passed as void*, NULL = the legacy default stream); calls
 * that write host memory synchronise that stream before returning.
 */
#ifndef FASTCAT_H
#define FASTCAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FC_OK        0
#define FC_EINVAL   -1   /* bad argument, shape or state transition */
#define FC_ENOMEM   -2   /* device allocation failed */
#define FC_ECUDA    -3   /* a CUDA runtime call or kernel launch failed */
#define FC_ESTATE   -4   /* a required set_* call has not been made */
#define FC_ETIMEOUT -5   /* a bounded device-side wait gave up */

/* where a pointer lives */
#define FC_HOST   0
#define FC_DEVICE 1
/* Host destination in page-locked memory, filled asynchronously (accepted
 * by fc_reconstruct's outputs; see fc_wait_outputs). */
#define FC_HOST_ASYNC 2

/* what fc_project returns */
#define FC_OUT_NONE      0  /* keep results on the device only */
#define FC_OUT_PRIMARY   1  /* T: flood-normalised primary signal */
#define FC_OUT_INTENSITY 2  /* I = N0 (G_psf * T + SPR G_sc * T), noise-free */
#define FC_OUT_COUNTS    3  /* Poisson(I) if noise is on, else I */

/* limits */
#define FC_MAX_MATERIALS 8
#define FC_MAX_BINS      256
#define FC_MAX_SIGMA_PX  64.0

typedef struct fc_handle fc_handle;

typedef struct fc_geometry {
    double sad_cm;          /* source to rotation axis */
    double sdd_cm;          /* source to detector, > sad_cm */
    int32_t n_u, n_v;       /* detector pixels (u across, v along z) */
    double du_cm, dv_cm;    /* pixel pitch */
    int32_t n_angles;       /* projections */
    double theta0_rad;      /* first angle */
    double arc_rad;         /* angular range covered by n_angles (2 pi for FDK) */
    int32_t nx, ny, nz;     /* voxel grid */
    double dx_cm, dy_cm, dz_cm;
} fc_geometry;

typedef struct fc_spectrum_detector {
    int32_t n_e;            /* energy bins, 1 .. FC_MAX_BINS */
    int32_t n_mat;          /* materials (columns of mu), 1 .. FC_MAX_MATERIALS */
    const double *w;        /* [n_e] fluence weights phi(E) (host) */
    const double *d;        /* [n_e] detector response eta(E) (host) */
    const double *mu;       /* [n_e][n_mat] linear attenuation, 1/cm (host) */
    double psf_sigma_px;    /* detector optical spread, Gaussian sigma in pixels */
    double scatter_sigma_px;/* scatter kernel, Gaussian sigma in pixels */
    double spr;             /* scatter-to-primary ratio */
    double n0;              /* flood photons per pixel (H) */
    uint64_t seed;          /* Poisson noise seed */
    int32_t noise;          /* 1: FC_OUT_COUNTS draws Poisson noise */
} fc_spectrum_detector;

/* Create a handle bound to CUDA device `device`.  *out receives it.
 * (Library set-up: the paper has no counterpart.)
 * Errors: FC_EINVAL (null out, bad device), FC_ECUDA. */
int fc_create(fc_handle **out, int device);

/* Release the handle and every device buffer it owns.  NULL is accepted.
 * (Library set-up: the paper has no counterpart.) */
int fc_destroy(fc_handle *h);

/* Message describing the last failure on this thread ("" if none).
 * (Error reporting: the paper has no counterpart.) */
const char *fc_last_error(void);

/* Scan geometry (Sec. II.F raytracing set-up; Sec. II.G FDK).  Copies *g.
 * Reallocates projection and volume buffers when sizes change.
 * Errors: FC_EINVAL (non-positive sizes or pitches, sdd <= sad, volume not
 * strictly between source and detector), FC_ENOMEM. */
int fc_set_geometry(fc_handle *h, const fc_geometry *g);

/* Labelled phantom (Sec. II.D: integer array 0 .. n-1 plus a material map).
 * labels: uint8 [nz][ny][nx] in host (where = FC_HOST) or device memory;
 * copied into the handle.  Every label must be < n_mat; violations are
 * reported as FC_EINVAL (host labels: checked on the host before the copy,
 * which stays queued on `stream` without waiting, so the host buffer must
 * stay unchanged until the stream reaches it, and page-locked memory makes
 * the copy asynchronous; device labels: checked on the device, the call
 * waits for the check).
 * Errors: FC_ESTATE (no geometry), FC_EINVAL, FC_ECUDA. */
int fc_set_phantom(fc_handle *h, const uint8_t *labels, int n_mat, int where,
                   void *stream);

/* Spectrum, attenuation table, detector response, blur, scatter and noise
 * settings (Sec. II.A-B, II.E, II.F energy weighting, II.H).  Arrays are
 * read from host memory and copied.  w and d must be >= 0 with
 * sum_E w d > 0; mu >= 0; sigmas in [0, FC_MAX_SIGMA_PX]; spr >= 0; n0 > 0.
 * Errors: FC_EINVAL. */
int fc_set_spectrum_detector(fc_handle *h, const fc_spectrum_detector *s);

/* Simulate projections angle_begin .. angle_begin + angle_count - 1:
 *   T = sum_E w D exp(-sum_m mu_m(E) L_m) / sum_E w D  (projector with the
 *       energy integral fused; L_m = path length in material m, Siddon:
 *       Sec. II.F raytracing and the I_f equation),
 *   I = N0 (G_psf (x) T + SPR G_scatter (x) T)  (separable, clamp-to-edge:
 *       Sec. II.B/G optical spread, Sec. II.E scatter),
 *   K = Poisson(I) (Philox4x32-10 counters (iu, iv, k, j), if noise is on:
 *       Sec. II.G-H).
 * Results stay in the handle for fc_reconstruct; `out_kind` selects which
 * one (if any) is also copied to `out` ([angle_count][n_v][n_u] float, in
 * host or device memory per `out_where`).
 * Errors: FC_ESTATE, FC_EINVAL (range, out_kind), FC_ECUDA. */
int fc_project(fc_handle *h, int angle_begin, int angle_count, int out_kind,
               float *out, int out_where, void *stream);

/* Order of noise and optical spread in fc_project.
 *   FC_NOISE_AFTER_BLUR (default): I = N0 (G_psf (x) T + SPR G_sc (x) T),
 *     K = Poisson(I): noise on the detected signal.
 *   FC_NOISE_BEFORE_PSF (the order of Sec. II.G: Poisson scaling of the
 *     counts incident on the detector, then the OSF convolution):
 *     lambda = N0 (T + SPR G_sc (x) T), K = G_psf (x) Poisson(lambda).
 *     FC_OUT_INTENSITY then returns lambda; FC_OUT_COUNTS returns K (with
 *     noise off, G_psf (x) lambda).
 * The flood stays N0 (1 + SPR) in both orders (the kernels sum to one).
 * Errors: FC_EINVAL. */
#define FC_NOISE_AFTER_BLUR 0
#define FC_NOISE_BEFORE_PSF 1
int fc_set_noise_order(fc_handle *h, int order);

/* Energy-group detector model (Sec. II.E scatter fit, Sec. II.F I_f
 * equation, Sec. II.G optical spread "at each energy and summed"), with the
 * spectrum's bins lumped into contiguous groups g = [bin_end[g-1], bin_end[g]):
 *   P_g = sum_{E in g} w D exp(-sum_m mu_m(E) L_m) / sum_E w D  (sum_g P_g = T)
 *   I   = N0 sum_g G_g (x) (P_g + A_g y_g(x)),
 *   y_g(x) = (a_g / sqrt(x^2 + a_g^2))^b_g, x = off-axis distance of the
 *   detector column, cm; G_g a sampled Gaussian (clamp-to-edge) of sigma_g px;
 *   K   = Poisson(I) when noise is on.
 * It replaces the single-kernel model of fc_set_spectrum_detector (psf,
 * scatter sigma and spr) for FC_OUT_INTENSITY, FC_OUT_COUNTS and FC_OUT_NONE;
 * FC_OUT_PRIMARY still returns T.  The flood used by fc_reconstruct is then
 * N0 (no phantom, no scatter).  Noise before the optical spread is not
 * defined for this model (fc_project returns FC_EINVAL with that order).
 *   n_groups     0 turns the model off; else 1 .. FC_MAX_GROUPS;
 *   bin_end      [n_groups] strictly increasing, last = n_e of the spectrum;
 *   psf_sigma_px [n_groups] in [0, FC_MAX_GROUP_SIGMA_PX];
 *   scatter_amp  [n_groups] A_g >= 0, relative to the flood;
 *   scatter_a_cm [n_groups] a_g > 0;  scatter_b [n_groups] b_g >= 0.
 * Arrays are host memory, copied.  Call after fc_set_spectrum_detector
 * (which clears the groups).  Errors: FC_ESTATE (no spectrum), FC_EINVAL. */
/* Richardson-Lucy deconvolution of the handle's counts for projections
 * angle_begin .. angle_begin + angle_count - 1 (the discussion of the paper,
 * Sec. IV: projections deconvolved with the detector PSF before
 * reconstruction), in place, as the EM update for Poisson data
 *   u_{k+1} = u_k H^T(d / max(H u_k, 1e-12)) / H^T 1,   u_0 = d (the counts),
 * H the clamp-to-edge separable sampled Gaussian of psf_sigma_px
 * (0 .. FC_MAX_GROUP_SIGMA_PX) and H^T its exact adjoint; n_iter >= 0 steps.
 * The result replaces the counts that fc_reconstruct(counts = NULL) uses and
 * is also copied to `out` ([angle_count][n_v][n_u] float, host or device per
 * `out_where`) when out is not NULL.
 * Errors: FC_ESTATE (no counts), FC_EINVAL, FC_ECUDA. */
int fc_deconvolve_rl(fc_handle *h, int angle_begin, int angle_count, double psf_sigma_px,
                     int n_iter, float *out, int out_where, void *stream);

/* Detector MTF by the slanted-slit method (Sec. II.C): the detector PSF of
 * the current model (the single optical-spread kernel, or each energy
 * group's kernel weighted by the group's share of the flood, sum_E w D) is
 * applied, clamp-to-edge, to a 192 x 192-pixel image of an ideal slit
 * slit_width_mm wide tilted by slit_angle_deg (|angle| < 45) on the u-pitch
 * grid; pixel values are the area fractions inside the slit.  The line spread
 * function is presampled from rows 48 .. 143 on bins du / oversample wide
 * over +-16 pixels (mean per bin); the MTF is its normalised Fourier
 * magnitude at f = k / (32 du), k = 0 .. 16 oversample, written with the
 * frequencies (1/mm) to host arrays of n_cap >= 16 oversample + 1 entries;
 * *n_out receives the count.  Binary64, synchronous (default stream).
 * Optical-spread sigmas above FC_MAX_GROUP_SIGMA_PX are refused.
 * Errors: FC_ESTATE, FC_EINVAL, FC_ENOMEM, FC_ECUDA. */
int fc_detector_mtf(fc_handle *h, double slit_width_mm, double slit_angle_deg, int oversample,
                    double *freq_per_mm, double *mtf, int n_cap, int *n_out);

#define FC_MAX_GROUPS 8
#define FC_MAX_GROUP_SIGMA_PX 4.0
typedef struct fc_energy_groups {
    int32_t n_groups;
    const int32_t *bin_end;
    const double *psf_sigma_px;
    const double *scatter_amp;
    const double *scatter_a_cm;
    const double *scatter_b;
} fc_energy_groups;
int fc_set_energy_groups(fc_handle *h, const fc_energy_groups *g);

/* FDK reconstruction (Sec. II.G): p = ln(I_flood / max(K, 1)),
 * I_flood = N0 (1 + SPR); cosine weight SAD / sqrt(SAD^2 + u^2 + v^2) at the
 * isocentre; Ram-Lak row filter; voxel-driven bilinear backprojection with
 * weight (SAD / U)^2 and factor arc / (2 n_angles), accumulated in FP64.
 * counts: [n_angles][n_v][n_u] float in host or device memory, or NULL to
 * use the handle's last FC_OUT_COUNTS result.  vol_mu (double [nz][ny][nx],
 * 1/cm) and vol_hu (float, HU normalised on the water region) may each be
 * NULL; `out_where` (FC_HOST, FC_DEVICE or FC_HOST_ASYNC, see
 * fc_wait_outputs) applies to both.
 * Errors: FC_ESTATE, FC_EINVAL, FC_ECUDA. */
int fc_reconstruct(fc_handle *h, const float *counts, int counts_where,
                   double *vol_mu, float *vol_hu, int out_where, void *stream);

/* Wait for the results of earlier fc_reconstruct calls made with out_where =
 * FC_HOST_ASYNC (library plumbing: the paper has no counterpart).  With
 * FC_HOST_ASYNC, vol_mu / vol_hu must be page-locked host memory (e.g.
 * cudaHostAlloc; pageable memory is refused with FC_EINVAL): the call queues
 * the device-to-host copies on a stream of the handle's own, ordered after
 * the results are complete on `stream`, and returns without waiting, so the
 * copies overlap the caller's next calls on `stream` (the next fc_project,
 * the next filter).  The host buffers hold the results once
 * fc_wait_outputs returns; until then they must not be read or freed.  A
 * later call that rewrites the volume (fc_reconstruct before its
 * backprojection, fc_cnr_grad) makes its stream wait on the device for the
 * queued copies; fc_set_geometry and fc_destroy wait on the host.  Returns
 * FC_OK at once when nothing is queued.
 * Errors: FC_EINVAL (null handle), FC_ECUDA, FC_ETIMEOUT (as fc_project's
 * host outputs report it). */
int fc_wait_outputs(fc_handle *h);

/* FDK backprojector variant (instrumentation and testing: the paper has no
 * counterpart; every variant computes the same backprojection of
 * fc_reconstruct, Sec. II.G, the sums differing only in rounding).
 *   FC_BP_AUTO          (default) the fastest applicable for the geometry:
 *                       FC_BP_SLAB_SYM, else FC_BP_SLAB, else
 *                       FC_BP_CHUNKED_SYM, else FC_BP_CHUNKED_DENSE for
 *                       grids of two or more waves, else FC_BP_CHUNKED;
 *   FC_BP_CHUNKED       one thread per (x, y) column and chunk of z slices,
 *                       four bilinear taps per voxel update;
 *   FC_BP_CHUNKED_DENSE the same body capped at 32 registers (8 CTAs per SM);
 *   FC_BP_SLAB          one thread per column and every slice; each slice
 *                       reuses the previous slice's detector row.  Applies
 *                       when nz <= 16 and the z pitch projects to at most 0.98
 *                       detector rows at every voxel (dz SDD / (SAD - r_max)
 *                       <= 0.98 dv, r_max the half-diagonal of the volume).
 *   FC_BP_SLAB_SYM      the thin-slab walk for the four columns that a
 *                       quarter turn about the axis maps onto one another,
 *                       one column set-up serving projections k, k + N/4,
 *                       k + N/2 and k + 3N/4.  Applies where FC_BP_SLAB does
 *                       and the scan is a full circle (arc_rad = 2 pi within
 *                       1e-12 relative) of n_angles divisible by 4 over a
 *                       grid with nx = ny even and dx_cm = dy_cm.  The
 *                       volume is written with binary64 atomic adds (two per
 *                       voxel onto zero: deterministic).
 *   FC_BP_CHUNKED_SYM   the same quarter-turn sharing for any slab thickness
 *                       (every slice loads its two detector rows): applies
 *                       where the quarter-turn symmetry holds (as for
 *                       FC_BP_SLAB_SYM, without the thin-slab condition).
 * fc_reconstruct and fc_cnr_grad fail with FC_EINVAL when the requested
 * variant does not apply (for every variant: when the stored filtered rows,
 * n_angles x (reachable rows + 3) x (n_u + 3, rounded up to 4), reach 2^31
 * elements).  fc_backprojector_in_use writes the variant the
 * current request resolves to for the handle's geometry.
 * Errors: FC_EINVAL (unknown variant, null pointers, not applicable),
 * FC_ESTATE (no geometry). */
#define FC_BP_AUTO          0
#define FC_BP_CHUNKED       1
#define FC_BP_CHUNKED_DENSE 2
#define FC_BP_SLAB          3
#define FC_BP_SLAB_SYM      4
#define FC_BP_CHUNKED_SYM   5
int fc_set_backprojector(fc_handle *h, int variant);
int fc_backprojector_in_use(fc_handle *h, int *variant);

/* Water region used for HU (Sec. II.G): voxels whose centre lies within
 * radius_cm of the rotation axis, excluding floor(z_margin * nz) slices at
 * each end.  Default 1.0 cm and 0.1.  Errors: FC_EINVAL. */
int fc_set_water_roi(fc_handle *h, double radius_cm, double z_margin);

/* Poisson noise alone (Sec. II.H): counts[k][iv][iu] ~ Poisson(lam[..])
 * with the same counter-based stream as fc_project (projection index
 * angle0 + k).  lam and counts are device pointers of
 * n_angles * n_v * n_u floats; they may alias.  Errors: FC_EINVAL, FC_ECUDA. */
int fc_poisson(const float *lam, float *counts, int n_angles, int n_v, int n_u,
               int angle0, uint64_t seed, void *stream);

/* Per-material path lengths of the rays of projections angle_begin ..
 * angle_begin + angle_count - 1 (the traversal of fc_project without the
 * energy integral; Sec. II.F raytracing), written to the device buffer L
 * ([angle_count][n_v][n_u][n_mat] float, cm).  Errors: FC_ESTATE, FC_EINVAL,
 * FC_ECUDA. */
int fc_project_lengths(fc_handle *h, int angle_begin, int angle_count, float *L,
                       void *stream);

/* Dose estimate per particle (Sec. II.H, the D_0(E) and D_p equations):
 *   D0(E) = E (mu_en/mu)_w(E) sum_i (1 - exp(-sum_m mu_m(E) L_im)) / (N_i M),
 *   Dp    = sum_E phi(E) D0(E),   phi = w / sum w (the fluence spectrum),
 * over the N_i = angle_count * n_v * n_u rays of projections angle_begin ..
 * angle_begin + angle_count - 1 (each ray's attenuation is the projector's
 * multi-material sum, L from the same traversal), with the phantom mass
 * M = dx dy dz sum_v rho(label_v).  Units: keV, grams, Gy per particle
 * (1 keV / g = 1.602176634e-13 Gy).  The paper's empirical linear fit to
 * Monte Carlo doses is not part of this estimate.
 *   e_kev        [n_e] host: bin energies, > 0;
 *   muen_over_mu [n_e] host: energy-absorption over attenuation coefficient
 *                of water, in [0, 1];
 *   rho          [n_mat] host: material mass densities, g/cm^3, > 0;
 *   d0 [n_e], dp [1]: results, host or device memory per `out_where` (with
 *                FC_DEVICE the copies are queued on `stream`).
 * Partial sums run in a fixed order: repeated calls give identical bits.
 * Errors: FC_ESTATE (geometry, phantom or spectrum missing), FC_EINVAL
 * (range, angle_count < 1, values), FC_ECUDA. */
int fc_dose_estimate(fc_handle *h, int angle_begin, int angle_count, const double *e_kev,
                     const double *muen_over_mu, const double *rho, double *d0, double *dp,
                     int out_where, void *stream);

/* Flood height for a requested mean phantom dose per projection (Sec. II.H,
 * the H equation): N_gamma = dose_gy / dp_gy particles over a beam of
 * A / A_p = n_u n_v detector pixels, so *n0 = dose_gy / (dp_gy n_u n_v).
 * Host arithmetic only.  Errors: FC_EINVAL, FC_ESTATE (no geometry). */
int fc_fluence_for_dose(const fc_handle *h, double dose_gy, double dp_gy, double *n0);

/* Kernel-time tracing (instrumentation: the paper has no counterpart).
 * While enabled, every kernel the handle launches is bracketed by CUDA
 * events recorded on the launching stream.  Kernel ids: */
#define FC_K_PROJECT     0  /* projector + energy integral (traced rows + T = 1 fill) */
#define FC_K_BLUR_ROWS   1  /* detector blur, band matrices + row pass */
#define FC_K_BLUR_COLS   2  /* detector blur, column pass */
#define FC_K_FDK_FILTER  3  /* log, cosine weight, Ram-Lak filter */
#define FC_K_BACKPROJECT 4  /* FDK backprojection */
#define FC_K_HU          5  /* water-region mean and HU (two kernels) */
#define FC_K_LENGTHS     6  /* path-length emission (fc_project_lengths) */
#define FC_K_NOISE       7  /* Poisson noise */
#define FC_K_SURROGATE_EVAL  8  /* surrogate inference (fc_surrogate_eval) */
#define FC_K_SURROGATE_TRAIN 9  /* surrogate training steps (4 kernels per step) */
#define FC_K_ENERGY_SUM     10  /* exact energy sum from path lengths */
#define FC_K_DOSE           11  /* dose estimate (four kernels) */
#define FC_K_GROUP_BLUR     12  /* energy-group model: scatter profile + per-group blur (2 kernels) */
#define FC_K_DECONV         13  /* Richardson-Lucy deconvolution (1 + n_iter kernels) */
#define FC_K_BLUR_BAND      14  /* detector blur of a primary that is 1 outside a narrow band of rows */
#define FC_K_COUNT          15

/* Enable (1) or disable (0) tracing; enabling discards pending records.
 * Errors: FC_EINVAL. */
int fc_profile_enable(fc_handle *h, int enable);

/* Wait for every traced launch, then write, per kernel id, the summed device
 * time in milliseconds to ms[FC_K_COUNT] and the number of kernel launches
 * to launches[FC_K_COUNT] (either may be NULL), and reset the totals.
 * Errors: FC_EINVAL, FC_ECUDA. */
int fc_profile_read(fc_handle *h, double *ms, int64_t *launches);

/* ---- Learned surrogate of the energy integral ----
 * The projector's energy loop evaluates, per ray, the I_f equation of
 * Sec. II.F: T = sum_E (w D)_E exp(-sum_m mu_m(E) L_m) / sum_E (w D)_E.  The
 * surrogate approximates ln T from the per-material path lengths L with
 *   ln T ~ ln sum_k a_k exp(-sum_m mu_km L_m) + MLP(L * scale),
 *   the baseline being the same integral with the spectrum lumped into four
 *   groups of equal weight (a_k group weight, mu_km weight-averaged mu_m(E);
 *   one group would give the first-order term -mubar . L), and
 *   MLP 8 -> 128 -> 128 -> 128 -> 1, SiLU (sigma via tanh), bf16 weights,
 *   activations as bf16 hi + lo pairs, tensor cores with f32 accumulation.
 * Path lengths are float [n][n_mat] and ln T float [n], in device memory.
 * The handle's spectrum (fc_set_spectrum_detector) must be set first.
 *
 * Parameter state (fc_surrogate_get/set), FC_SURROGATE_STATE floats:
 *   [0, 34305): W1[128][8], b1[128], W2[128][128], b2, W3[128][128], b3,
 *               w4[128], b4 (fp32 master copies; W[out][in]);
 *   then scale[8] (inputs are L * scale), a[4], mu[4][8] (baseline) and
 *   box[8] (rays with any L_m > box_m are evaluated exactly); then Adam
 *   first and second moments (34305 each) and the Adam step count. */
#define FC_SURROGATE_PARAMS 34305
#define FC_SURROGATE_STATE  (34305 + 52 + 2 * 34305 + 1)

/* Initialise the surrogate with seeded random weights (uniform, scaled by
 * fan-in), the baseline groups from the current spectrum, unit scale and an
 * unbounded box.
 * Errors: FC_ESTATE (no spectrum), FC_ENOMEM, FC_ECUDA. */
int fc_surrogate_init(fc_handle *h, uint64_t seed);

/* Train with Adam (beta 0.9 / 0.999, eps 1e-8) on the mean squared error of
 * ln T for `steps` steps of `batch` samples drawn with replacement from the
 * n pairs (L, lnT) by a seeded hash; learning rate lr with cosine decay over
 * the call.  The first call after fc_surrogate_init fixes scale = 1 / max L
 * and box = max L per material from this data.  loss_hist (host, may be
 * NULL) receives the per-step batch MSE.  batch must be a positive multiple
 * of 128.  Errors: FC_ESTATE, FC_EINVAL, FC_ETIMEOUT (a bounded tensor-core
 * wait expired), FC_ENOMEM, FC_ECUDA. */
int fc_surrogate_train(fc_handle *h, const float *L, const float *lnT, int64_t n, int steps,
                       int batch, float lr, uint64_t seed, float *loss_hist, void *stream);

/* Gradient of the mean squared error over exactly the first n samples with
 * respect to the FC_SURROGATE_PARAMS parameters, written to grad (host), and
 * the loss to *loss (host, may be NULL); no update.  n must be a multiple of
 * 8.  Errors as fc_surrogate_train. */
int fc_surrogate_grad(fc_handle *h, const float *L, const float *lnT, int64_t n, float *grad,
                      float *loss, void *stream);

/* Copy the full state (FC_SURROGATE_STATE floats, host) out of / into the
 * handle (checkpoint and resume).  Errors: FC_EINVAL, FC_ESTATE, FC_ECUDA. */
int fc_surrogate_get(fc_handle *h, float *state);
int fc_surrogate_set(fc_handle *h, const float *state);

/* ln T of n rays from their path lengths by the surrogate, falling back to
 * the exact energy sum for rays outside the training box (and, with a guard
 * set, for rays attenuated beyond its threshold); *n_fallback (host,
 * may be NULL; non-NULL synchronises the stream) receives how many fell
 * back.  Errors: FC_ESTATE, FC_EINVAL, FC_ETIMEOUT, FC_ECUDA. */
int fc_surrogate_eval(fc_handle *h, const float *L, int64_t n, float *lnT, int64_t *n_fallback,
                      void *stream);

/* Per-ray guard of the surrogate, judged by the exact energy sum: from n
 * rays with path lengths L and exact ln T (device, e.g. the training data),
 * evaluate the network alone, take the smallest baseline attenuation
 * -ln sum_k a_k exp(-sum_m mu_km L_m) among the rays whose |ln T error|
 * exceeds tol, and from then on have fc_surrogate_eval (and
 * fc_surrogate_project) evaluate every ray attenuated at least that much
 * with the exact sum (counted in *n_fallback).  *threshold (host, may be
 * NULL) receives it; +inf when no ray exceeded tol.  tol <= 0 removes the
 * guard.  The guard belongs to the handle, not to the
 * fc_surrogate_get/set state: set it again after fc_surrogate_set.
 * Instrumentation of the learned surrogate (the paper has no counterpart).
 * Errors: FC_ESTATE, FC_EINVAL, FC_ETIMEOUT, FC_ENOMEM, FC_ECUDA. */
int fc_surrogate_guard(fc_handle *h, const float *L, const float *lnT, int64_t n, double tol,
                       double *threshold, void *stream);

/* The logistic function sigma(z) = 1 / (1 + exp(-z)) of the surrogate's SiLU
 * activations, evaluated on the GPU exactly as its kernels evaluate it
 * (binary32, (1 + tanh(z / 2)) / 2 with the hardware tanh approximation), for
 * n values z (device) into sigma (device; may alias z).  Lets a test measure
 * the activations' error against the exact function (no handle; runs on
 * the current device).  Errors: FC_EINVAL (n < 0, NULL pointer with n > 0),
 * FC_ECUDA. */
int fc_surrogate_sigma(const float *z, float *sigma, int64_t n, void *stream);

/* Projection with the surrogate in place of the energy loop: the
 * projector's path lengths for projections angle_begin .. + angle_count - 1
 * are fed to the surrogate and T = exp(ln T) of every ray is written to out
 * ([angle_count][n_v][n_u] float, host or device per out_where).  Uses a
 * handle-owned scratch buffer of angle_count * n_v * n_u * (n_mat + 1)
 * floats.  Errors: FC_ESTATE, FC_EINVAL, FC_ENOMEM, FC_ECUDA. */
int fc_surrogate_project(fc_handle *h, int angle_begin, int angle_count, float *out,
                         int out_where, void *stream);

/* ln T of n rays from their path lengths by the exact energy sum (the I_f
 * equation of Sec. II.F; the projector's epilogue as a separate pass).  Errors: FC_ESTATE, FC_EINVAL,
 * FC_ECUDA. */
int fc_energy_sum_lengths(fc_handle *h, const float *L, int64_t n, float *lnT, void *stream);

/* ---- Gradient of an image-quality objective (adjoint) ----
 * J = sum_r CNR_r over the insert ROIs, CNR_r = |HU_w - HU_r| /
 * sqrt(s_w^2 + s_r^2) (Sec. II.G, CNR equation; HU normalised on the water
 * region of fc_set_water_roi), for the FDK image of the simulated scan with
 *   spectrum w = softmax(logits) and detector response D (Sec. II.F, I_f
 *   equation; the handle's attenuation table mu_m(E) at nominal densities),
 *   voxel densities rho: each voxel of label m attenuates as
 *   mu_m(E) rho_v / rho_nominal[m],
 *   detector blur and scatter of the handle (Sec. II.E, II.G),
 *   Poisson noise in its Gaussian form K = I + sqrt(I) z with a fixed
 *   standard-normal field z [n_angles][n_v][n_u] (device; NULL: K = I),
 *   FDK as in fc_reconstruct.
 * ROI r: voxel centres within radius_cm of (cx_cm, cy_cm), on the slices of
 * the water region.  Writes J (host) and, where non-NULL, dJ/dlogits and
 * dJ/dD (host, [n_e]) and dJ/drho (device, [nz][ny][nx] float), computed by
 * the adjoint of every step (projector recomputing each ray's path lengths).
 * rho is float [nz][ny][nx] in device memory; rho_nominal is [n_mat] host.
 * Uses the handle's projection and volume buffers (overwriting them).
 * Errors: FC_ESTATE, FC_EINVAL, FC_ENOMEM, FC_ECUDA. */
typedef struct fc_cnr_roi {
    double cx_cm, cy_cm, radius_cm;
} fc_cnr_roi;

int fc_cnr_grad(fc_handle *h, const double *logits, const double *D, const double *rho_nominal,
                const float *rho, const float *z, int n_roi, const fc_cnr_roi *rois, double *J,
                double *g_logits, double *g_D, float *g_rho, void *stream);

/* Fault injection for failure-handling tests (instrumentation: the paper
 * has no counterpart).  Process-wide and one-shot; nothing faults the GPU:
 *   FC_FAULT_NONE          clear every pending injection;
 *   FC_FAULT_ALLOC         the device allocation after the next `arg` ones
 *                          (arg >= 0) fails as out of memory: the call that
 *                          makes it returns FC_ENOMEM, the handle stays
 *                          usable and a later call allocates again;
 *   FC_FAULT_BLUR_TIMEOUT  the next tensor-core detector blur gives up its
 *                          first bounded accumulator wait at once and takes
 *                          its abort path (its MMAs and copies drained, tensor
 *                          memory freed, the error word set); the call that
 *                          reads the error word (a host output) returns
 *                          FC_ETIMEOUT and later calls run normally.
 * Errors: FC_EINVAL (unknown kind, negative count). */
#define FC_FAULT_NONE         0
#define FC_FAULT_ALLOC        1
#define FC_FAULT_BLUR_TIMEOUT 2
int fc_inject_fault(int kind, int64_t arg);

/* Allocation-free detector blur.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they
 * run -- their device memory is owned by another allocator (for example a
 * pool that reserved the whole GPU at start-up) or fixed by a budget that
 * forbids allocation after initialisation.  It computes the operator of
 * fc_project's FC_OUT_INTENSITY, I = n0 (G_psf (x) T + spr G_scatter (x) T),
 * with fc_project's direct f32 blur passes (the ones fc_project falls back
 * to for radii beyond its tensor-core passes), so it agrees with
 * FC_OUT_INTENSITY within 1e-4 relative, not bit for bit, and is slower.
 * T and I are n_img x n_v x n_u floats in device memory
 * provided by the caller, without a handle, and calls no cudaMalloc,
 * cudaFree or other allocating routine.  The two row-pass intermediates live
 * in a file-scope device array of FC_STATIC_SCRATCH_FLOATS floats (32 MiB)
 * that every GPU loading the library holds until the process exits; calls
 * with 2 * n_img * n_v * n_u > FC_STATIC_SCRATCH_FLOATS fail with FC_EINVAL.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the array: calls whose kernels overlap on the
 * GPU race on it, so order them (one stream, or events).  The looked-up
 * address is kept for the life of the process: a device reset while the
 * library is loaded is not supported.  Runs on the current device and
 * `stream`.  Errors: FC_EINVAL (null pointers, sizes, sigmas, spr < 0,
 * n0 <= 0, a detector too wide for the row pass or too tall for the column
 * pass's shared-memory staging), FC_ECUDA. */
#define FC_STATIC_SCRATCH_FLOATS (8u << 20)
int fc_detector_blur_static(const float *T, float *I, int n_img, int n_v, int n_u,
                            double psf_sigma_px, double scatter_sigma_px, double spr, double n0,
                            void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTCAT_H */

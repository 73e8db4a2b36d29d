"""Seeded synthetic inputs for the fastCAT CBCT hot path.

This module generates what the simulator *consumes*: scan geometries, labelled
voxel phantoms, per-material linear attenuation tables mu_m(E), source spectra
w(E) and detector energy responses D(E).  In the paper these come from outside
the simulation pipeline -- a 336-material attenuation database (Sec. II.D,
"Imaging Phantoms"), EGSnrc / xpecgen spectra (Sec. II.A, Table 1) and Topas
detector efficiencies (Sec. II.B, Table 2) -- and are loaded as tables.  The
data are not available here, so analytic stand-ins produce tables of the same
shape:

* mu_m(E) = rho_m * (a_m * E^-3 + b_m * KN(E)), with E in keV, b_m the
  Thomson mass coefficient N_A * sigma_T * (Z/A)_m and KN(E) the Klein-Nishina
  total cross-section divided by the Thomson one (a photo-electric E^-3 term
  plus incoherent scattering, no K-edges).
* kV spectrum: Kramers' law w ~ (E_max - E) / E times exp(-mu_Al(E) * 0.2 cm).
* MV spectrum: thick-target bremsstrahlung shape w ~ (E_max - E) / E.
* kV detector: D(E) = 1 - exp(-0.06 cm * mu_CsI(E)).
* MV detector: D(E) = (1 - exp(-1.0 cm * mu_GOS(E))) * E (energy deposition).

Nothing here evaluates the method itself (ray tracing, energy integral, blur,
noise, reconstruction): both the CUDA library and the FP64 oracle receive these
arrays as inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# physical constants (CODATA) used to build the attenuation stand-in tables
# ---------------------------------------------------------------------------
AVOGADRO = 6.02214076e23          # 1/mol
SIGMA_THOMSON_CM2 = 6.6524587321e-25  # cm^2 per electron
ELECTRON_REST_KEV = 510.99895     # m_e c^2 in keV
THOMSON_MASS = AVOGADRO * SIGMA_THOMSON_CM2  # cm^2/g per unit Z/A (~0.4006)

# name: (density g/cm^3, Z/A, photo-electric scale a in keV^3 cm^2/g)
# Approximate scales chosen for this project (not NIST data); every consumer
# receives the resulting table, so no result depends on their exact values.
MATERIALS = {
    "air":        (0.001205, 0.4992, 3.7e3),
    "water":      (1.0,      0.5551, 3.8e3),
    "bone":       (1.9,      0.5148, 2.4e4),
    "lung":       (0.3,      0.5497, 3.9e3),
    "adipose":    (0.95,     0.5558, 2.3e3),
    "brain":      (1.04,     0.5524, 3.9e3),
    "b100":       (1.45,     0.5274, 1.2e4),
    "soft_tissue": (1.03,    0.5500, 3.9e3),
    "fat":        (0.95,     0.5558, 2.3e3),
    "cartilage":  (1.10,     0.5502, 4.5e3),
    "blood":      (1.06,     0.5499, 4.0e3),
    "teeth":      (2.75,     0.5100, 3.0e4),
    "aluminium":  (2.699,    0.4818, 2.5e4),
    "csi":        (4.51,     0.4156, 1.2e6),
    "gos":        (7.34,     0.4218, 1.5e6),
}

# label -> material name, in label order (the phantom stores the index)
CATPHAN_LABELS = ("air", "water", "bone", "lung", "adipose", "brain", "b100")
HEAD_LABELS = ("air", "soft_tissue", "brain", "bone", "fat", "cartilage",
               "blood", "teeth")

# Catphan-like inserts: (label, diameter cm); centres on a ring of radius
# 2.5 cm at 0, 60, ..., 300 degrees (the paper shows the layout only in a
# figure, so the placement is this project's reading).
CATPHAN_INSERTS = ((3, 0.5), (2, 0.5), (4, 0.4), (5, 0.3), (6, 0.2), (2, 0.1))
CATPHAN_RADIUS_CM = 8.0
CATPHAN_RING_CM = 2.5


def klein_nishina_ratio(e_kev):
    """sigma_KN(E) / sigma_Thomson for photon energy ``e_kev`` (array)."""
    k = np.asarray(e_kev, dtype=np.float64) / ELECTRON_REST_KEV
    out = np.empty_like(k)
    small = k < 1e-3
    ks = k[small]
    out[small] = 1.0 - 2.0 * ks + 5.2 * ks * ks
    kb = k[~small]
    l2k = np.log1p(2.0 * kb)
    term1 = (1.0 + kb) / kb**2 * (2.0 * (1.0 + kb) / (1.0 + 2.0 * kb) - l2k / kb)
    term2 = l2k / (2.0 * kb)
    term3 = (1.0 + 3.0 * kb) / (1.0 + 2.0 * kb) ** 2
    out[~small] = 0.75 * (term1 + term2 - term3)
    return out


def mu_linear(name, e_kev):
    """Linear attenuation coefficient (1/cm) of material ``name`` at ``e_kev``."""
    rho, zoa, a = MATERIALS[name]
    e = np.asarray(e_kev, dtype=np.float64)
    return rho * (a * e**-3 + THOMSON_MASS * zoa * klein_nishina_ratio(e))


def energy_bins(e_lo, e_hi, n_e):
    """Centres of ``n_e`` equal-width bins spanning [e_lo, e_hi] keV."""
    w = (e_hi - e_lo) / n_e
    return e_lo + (np.arange(n_e) + 0.5) * w


def mu_table(labels, e_kev):
    """mu[E][m] (1/cm), float64, C-contiguous, for label names ``labels``."""
    return np.ascontiguousarray(
        np.stack([mu_linear(n, e_kev) for n in labels], axis=1))


def spectrum_kv(e_kev, e_max=120.0, al_cm=0.2):
    """Kramers photon-number spectrum after Al filtration, normalised to 1."""
    e = np.asarray(e_kev, dtype=np.float64)
    w = np.clip(e_max - e, 0.0, None) / e * np.exp(-mu_linear("aluminium", e) * al_cm)
    return w / w.sum()


def spectrum_mv(e_kev, e_max=2500.0):
    """Thick-target bremsstrahlung shape (E_max - E) / E, normalised to 1."""
    e = np.asarray(e_kev, dtype=np.float64)
    w = np.clip(e_max - e, 0.0, None) / e
    return w / w.sum()


def detector_kv(e_kev, thick_cm=0.06):
    """CsI absorption efficiency 1 - exp(-t * mu_CsI(E))."""
    return 1.0 - np.exp(-thick_cm * mu_linear("csi", e_kev))


def detector_mv(e_kev, thick_cm=1.0):
    """GOS energy-deposition response (1 - exp(-t * mu_GOS(E))) * E."""
    e = np.asarray(e_kev, dtype=np.float64)
    return (1.0 - np.exp(-thick_cm * mu_linear("gos", e))) * e


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Geometry:
    """Circular cone-beam scan of a centred voxel grid (all lengths in cm).

    Angles theta_k = theta0 + arc * k / n_angles.  Source at
    SAD * (cos, sin, 0); flat detector centre at -(SDD - SAD) * (cos, sin, 0);
    detector u axis (-sin, cos, 0), v axis (0, 0, 1); pixel (iu, iv) centre at
    ((iu - (n_u - 1) / 2) * du, (iv - (n_v - 1) / 2) * dv).  Voxel (i, j, k)
    centre at ((i - (nx - 1) / 2) dx, (j - (ny - 1) / 2) dy, (k - (nz - 1) / 2) dz).
    """
    sad: float
    sdd: float
    n_u: int
    n_v: int
    du: float
    dv: float
    n_angles: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    theta0: float = 0.0
    arc: float = 2.0 * math.pi

    def angles(self):
        return self.theta0 + self.arc * np.arange(self.n_angles) / self.n_angles

    @property
    def n_rays(self):
        return self.n_angles * self.n_v * self.n_u

    @property
    def n_voxels(self):
        return self.nx * self.ny * self.nz


@dataclasses.dataclass(frozen=True)
class Workload:
    """One scan: geometry + phantom recipe + spectrum + detector + noise."""
    name: str
    geom: Geometry
    phantom: str            # "catphan" | "head" | "uniform"
    labels: tuple
    e_lo: float
    e_hi: float
    n_e: int
    beam: str               # "kv" | "mv"
    e_max: float
    psf_sigma_px: float
    scatter_sigma_px: float
    spr: float
    n0: float
    seed: int
    noise: bool

    def energies(self):
        return energy_bins(self.e_lo, self.e_hi, self.n_e)

    def spectrum(self):
        e = self.energies()
        if self.beam == "kv":
            return spectrum_kv(e, self.e_max), detector_kv(e)
        return spectrum_mv(e, self.e_max), detector_mv(e)

    def mu(self):
        return mu_table(self.labels, self.energies())

    def densities(self):
        """Mass density of each label's material, g/cm^3."""
        return np.array([MATERIALS[m][0] for m in self.labels], dtype=np.float64)

    def muen_water(self):
        """(mu_en / mu) of water at the bin energies."""
        return muen_over_mu("water", self.energies())

    def make_phantom(self):
        g = self.geom
        if self.phantom == "catphan":
            return catphan_phantom(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)
        if self.phantom == "head":
            return head_phantom(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, seed=self.seed)
        if self.phantom == "uniform":
            return np.ones((g.nz, g.ny, g.nx), dtype=np.uint8)
        raise ValueError(self.phantom)


def _centres(n, d):
    return (np.arange(n) - (n - 1) / 2.0) * d


def catphan_phantom(nx, ny, nz, dx, dy, dz):
    """Catphan-515-like module: 16 cm water cylinder along z, six rod inserts.

    Labels follow CATPHAN_LABELS; voxels are labelled by their centre.
    Returns uint8 [nz][ny][nx].
    """
    x = _centres(nx, dx)[None, :]
    y = _centres(ny, dy)[:, None]
    sl = np.zeros((ny, nx), dtype=np.uint8)
    sl[x * x + y * y <= CATPHAN_RADIUS_CM**2] = 1
    for i, (lab, diam) in enumerate(CATPHAN_INSERTS):
        a = math.radians(60.0 * i)
        cx, cy = CATPHAN_RING_CM * math.cos(a), CATPHAN_RING_CM * math.sin(a)
        r = diam / 2.0
        sl[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = lab
    return np.ascontiguousarray(np.broadcast_to(sl, (nz, ny, nx)))


def catphan_inserts():
    """(label, centre_x, centre_y, radius) of each insert in cm."""
    out = []
    for i, (lab, diam) in enumerate(CATPHAN_INSERTS):
        a = math.radians(60.0 * i)
        out.append((lab, CATPHAN_RING_CM * math.cos(a),
                    CATPHAN_RING_CM * math.sin(a), diam / 2.0))
    return out


def head_phantom(nx, ny, nz, dx, dy, dz, seed=3, n_blobs=40):
    """Head-like phantom: soft-tissue ellipsoid (8.0, 7.0, 7.5) cm semi-axes
    with ``n_blobs`` random rotated ellipsoids painted in order.
    Labels follow HEAD_LABELS. Returns uint8 [nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    x = _centres(nx, dx)[None, None, :]
    y = _centres(ny, dy)[None, :, None]
    z = _centres(nz, dz)[:, None, None]
    semi = np.array([8.0, 7.0, 7.5])
    vol = np.zeros((nz, ny, nx), dtype=np.uint8)
    vol[(x / semi[0]) ** 2 + (y / semi[1]) ** 2 + (z / semi[2]) ** 2 <= 1.0] = 1
    choices = np.array([2, 3, 0, 4, 5, 6, 7], dtype=np.uint8)
    for _ in range(n_blobs):
        while True:  # centre uniform in the 0.7-scaled outer ellipsoid
            p = rng.uniform(-1.0, 1.0, 3)
            if p @ p <= 1.0:
                break
        c = p * semi * 0.7
        ax = rng.uniform(0.3, 2.0, 3)
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        q = q * np.sign(np.diag(r))[None, :]
        lab = choices[rng.integers(0, len(choices))]
        ext = ax.max()
        sx = slice(max(0, int((c[0] - ext) / dx + (nx - 1) / 2.0) - 1),
                   min(nx, int((c[0] + ext) / dx + (nx - 1) / 2.0) + 2))
        sy = slice(max(0, int((c[1] - ext) / dy + (ny - 1) / 2.0) - 1),
                   min(ny, int((c[1] + ext) / dy + (ny - 1) / 2.0) + 2))
        sz = slice(max(0, int((c[2] - ext) / dz + (nz - 1) / 2.0) - 1),
                   min(nz, int((c[2] + ext) / dz + (nz - 1) / 2.0) + 2))
        xs, ys, zs = x[:, :, sx] - c[0], y[:, sy, :] - c[1], z[sz, :, :] - c[2]
        # coordinates in the blob frame: rows of q^T applied to (x, y, z)
        u0 = q[0, 0] * xs + q[1, 0] * ys + q[2, 0] * zs
        u1 = q[0, 1] * xs + q[1, 1] * ys + q[2, 1] * zs
        u2 = q[0, 2] * xs + q[1, 2] * ys + q[2, 2] * zs
        inside = (u0 / ax[0]) ** 2 + (u1 / ax[1]) ** 2 + (u2 / ax[2]) ** 2 <= 1.0
        vol[sz, sy, sx][inside] = lab
    return vol


SAD_CM = 100.0
SDD_CM = 150.0

WORKLOADS = {
    # plain method, small kV case
    "small_kv": Workload(
        "small_kv",
        Geometry(SAD_CM, SDD_CM, 128, 128, 0.08, 0.08, 90, 64, 64, 64, 0.25, 0.25, 0.25),
        "catphan", CATPHAN_LABELS, 20.0, 120.0, 20, "kv", 120.0,
        0.6, 20.0, 0.2, 1e5, 0, True),
    # Catphan-like kV case (the measured workload)
    "catphan_kv": Workload(
        "catphan_kv",
        Geometry(SAD_CM, SDD_CM, 512, 384, 0.04, 0.04, 360, 256, 256, 10, 0.0625, 0.0625, 0.0625),
        "catphan", CATPHAN_LABELS, 20.0, 120.0, 30, "kv", 120.0,
        0.8, 20.0, 0.2, 1e5, 1, True),
    # paper-scale MV case (1024^2 x 10, 720 angles), noise-free
    "paper_mv": Workload(
        "paper_mv",
        Geometry(SAD_CM, SDD_CM, 1024, 768, 0.0392, 0.0392, 720, 1024, 1024, 10,
                 0.015625, 0.015625, 0.015625),
        "catphan", CATPHAN_LABELS, 100.0, 2500.0, 60, "mv", 2500.0,
        1.2, 20.0, 0.2, 1e5, 2, False),
    # head-like phantom for the learned surrogate
    "head_surrogate": Workload(
        "head_surrogate",
        Geometry(SAD_CM, SDD_CM, 512, 512, 0.05, 0.05, 360, 256, 256, 256, 0.0625, 0.0625, 0.0625),
        "head", HEAD_LABELS, 20.0, 140.0, 120, "kv", 140.0,
        0.8, 20.0, 0.2, 1e5, 3, False),
    # the paper's timing scan: 180 projections of a 6 MV beam in 18 energy
    # bins, reconstructed to 1024^2 x 10 and to 512^2 x 10 (noise drawn
    # before the optical spread, as the paper orders it)
    "timing_mv_1024": Workload(
        "timing_mv_1024",
        Geometry(SAD_CM, SDD_CM, 1024, 768, 0.0392, 0.0392, 180, 1024, 1024, 10,
                 0.015625, 0.015625, 0.015625),
        "catphan", CATPHAN_LABELS, 100.0, 6000.0, 18, "mv", 6000.0,
        1.2, 20.0, 0.2, 1e5, 5, True),
    "timing_mv_512": Workload(
        "timing_mv_512",
        Geometry(SAD_CM, SDD_CM, 1024, 768, 0.0392, 0.0392, 180, 512, 512, 10,
                 0.03125, 0.03125, 0.03125),
        "catphan", CATPHAN_LABELS, 100.0, 6000.0, 18, "mv", 6000.0,
        1.2, 20.0, 0.2, 1e5, 5, True),
    # adjoint design case
    "adjoint_kv": Workload(
        "adjoint_kv",
        Geometry(SAD_CM, SDD_CM, 512, 384, 0.04, 0.04, 180, 128, 128, 32, 0.125, 0.125, 0.125),
        "catphan", CATPHAN_LABELS, 20.0, 120.0, 30, "kv", 120.0,
        0.8, 20.0, 0.2, 1e5, 4, False),
}


def scaled(w: Workload, **geom_changes) -> Workload:
    """Copy of ``w`` with geometry fields replaced (for small test cases)."""
    return dataclasses.replace(w, geom=dataclasses.replace(w.geom, **geom_changes))


def water_roi_mask(g: Geometry, radius_cm=1.0, z_margin=0.1):
    """Central water disc used to normalise HU: voxel centres within
    ``radius_cm`` of the axis, excluding the outer ``z_margin`` of slices."""
    x = _centres(g.nx, g.dx)[None, None, :]
    y = _centres(g.ny, g.dy)[None, :, None]
    m = np.broadcast_to(x * x + y * y <= radius_cm**2, (g.nz, g.ny, g.nx)).copy()
    cut = int(math.floor(g.nz * z_margin))
    if cut > 0 and g.nz > 2 * cut:
        m[:cut] = False
        m[g.nz - cut:] = False
    return m


def adjoint_inputs(w: Workload, seed=4):
    """Inputs of the CNR-gradient case: spectrum logits (seeded normals),
    detector response D, nominal densities per label, voxel densities (the
    nominal ones), a fixed standard-normal noise field z [angle][v][u] and
    the bone and lung insert ROIs (centre, radius = 0.7 insert radius, at
    least reaching the nearest voxel centre)."""
    rng = np.random.default_rng(seed)
    g = w.geom
    logits = rng.normal(0.0, 0.5, w.n_e)
    _, D = w.spectrum()
    rho0 = np.array([MATERIALS[n][0] for n in w.labels])
    lab = w.make_phantom()
    rho = rho0[lab].astype(np.float32)
    z = rng.standard_normal((g.n_angles, g.n_v, g.n_u)).astype(np.float32)
    x = _centres(g.nx, g.dx)
    y = _centres(g.ny, g.dy)
    rois = []
    for lab_id, cx, cy, r in catphan_inserts():
        if lab_id not in (2, 3) or r < 0.2:
            continue   # the 5 mm bone and lung rods
        dmin = np.min(np.hypot(x[None, :] - cx, y[:, None] - cy))
        rois.append((cx, cy, max(0.7 * r, dmin + 1e-6)))
    return dict(logits=logits, D=D, rho0=rho0, rho=rho, z=z, rois=rois, labels=lab)


def klein_nishina_scatter_ratio(e_kev):
    """sigma_s / sigma_Thomson: the part of the Klein-Nishina cross-section
    carried off by the scattered photon's energy (Evans' closed form)."""
    k = np.asarray(e_kev, dtype=np.float64) / ELECTRON_REST_KEV
    l2k = np.log1p(2.0 * k)
    t = (l2k / k**3 + 2.0 * (1.0 + k) * (2.0 * k * k - 2.0 * k - 1.0) / (k * k * (1.0 + 2.0 * k) ** 2)
         + 8.0 * k * k / (3.0 * (1.0 + 2.0 * k) ** 3))
    return 0.375 * t


def muen_over_mu(name, e_kev):
    """Energy-absorption to attenuation ratio of material ``name``: the
    photo-electric part deposits all its energy, incoherent scattering the
    Klein-Nishina energy-transfer fraction (no fluorescence or radiative
    losses)."""
    rho, zoa, a = MATERIALS[name]
    e = np.asarray(e_kev, dtype=np.float64)
    tau = a * e**-3
    kn = klein_nishina_ratio(e)
    sig = THOMSON_MASS * zoa * kn
    ftr = 1.0 - klein_nishina_scatter_ratio(e) / kn
    return (tau + sig * ftr) / (tau + sig)


def energy_groups(w: Workload, n_groups=4):
    """Energy-group detector model inputs (stand-ins for the paper's per-energy
    Topas fits, which are not available): contiguous groups of about equal bin
    count; optical-spread sigma growing from 0.75x to 1.5x the workload's PSF
    sigma across the groups; scatter fit parameters a from 14 to 9 cm and b
    from 1.2 to 2.0; amplitudes spr * (the group's share of the flood), so the
    profiles peak at the workload's scatter-to-primary ratio."""
    n = w.n_e
    bin_end = np.array([int(round(n * (i + 1) / n_groups)) for i in range(n_groups)], np.int32)
    wts, d = w.spectrum()
    wd = wts * d
    start = np.concatenate([[0], bin_end[:-1]])
    share = np.array([wd[a:b].sum() for a, b in zip(start, bin_end)]) / wd.sum()
    t = np.linspace(0.0, 1.0, n_groups)
    return {"bin_end": bin_end,
            "psf_sigma_px": w.psf_sigma_px * (0.75 + 0.75 * t),
            "scatter_amp": w.spr * share,
            "scatter_a_cm": 14.0 - 5.0 * t,
            "scatter_b": 1.2 + 0.8 * t}

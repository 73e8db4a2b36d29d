"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerances: primary signal and intensity relative
error <= 1e-4 per pixel, reconstruction |d mu| <= 5e-4 mu_water (0.5 HU),
Poisson counts bit-identical for identical rates."""
import math

import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_T = 1e-4
HU_TOL = 0.5


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


def _scanner(fc, wl, lab=None, noise=None):
    return fc.Scanner(wl, labels=wl.make_phantom() if lab is None else lab, noise=noise)


def _project(fc, sc, kind, a0=0, na=None):
    g = sc.g
    na = g.n_angles - a0 if na is None else na
    out = torch.empty((na, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
    fc.fc_project(sc.h, a0, na, kind, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ragged_random():
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=45, n_angles=7, nx=24, ny=20, nz=16,
                  dx=0.25, dy=0.25, dz=0.25, du=0.12, dv=0.12)
    rng = np.random.default_rng(21)
    g = wl.geom
    lab = rng.integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    return wl, lab


def test_path_lengths_ragged_random_labels(fc, orc, precision):
    wl, lab = _ragged_random()
    g = wl.geom
    sc = _scanner(fc, wl, lab)
    try:
        L = torch.empty((g.n_angles, g.n_v, g.n_u, 7), dtype=torch.float32, device="cuda")
        fc.fc_project_lengths(sc.h, 0, g.n_angles, L)
        torch.cuda.synchronize()
        L = L.cpu().numpy().reshape(-1, 7)
    finally:
        sc.close()
    k, v, u = np.meshgrid(np.arange(g.n_angles), np.arange(g.n_v), np.arange(g.n_u), indexing="ij")
    rays = np.stack([k.ravel(), v.ravel(), u.ravel()], 1)
    w, d = wl.spectrum()
    Lr, _ = orc.rays(g, lab, w, d, wl.mu(), rays)
    err = np.abs(L - Lr)
    precision("L (path lengths)", "ragged 24x20x16 random labels, every ray", err.max(), 2e-4, "cm")
    precision("sum of L (chord)", "ragged 24x20x16 random labels, every ray",
              np.abs(L.sum(1) - Lr.sum(1)).max(), 1e-4, "cm")
    # binary32 traversal: errors per material transition, a few ulp of the
    # in-volume coordinates (<= ~1e-6 cm) each; the chord ends on a z face
    # are crossed at grazing angles (|d_z| <= 0.05 for these cone angles), so
    # a ~5e-7 cm displacement of the binary32 ray moves them by up to ~20x.
    assert err.max() < 2e-4, err.max()
    assert np.abs(L.sum(1) - Lr.sum(1)).max() < 1e-4


def test_primary_ragged_random_labels(fc, orc):
    wl, lab = _ragged_random()
    g = wl.geom
    sc = _scanner(fc, wl, lab)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
    finally:
        sc.close()
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    rel = np.abs(T - Tr) / Tr
    assert rel.max() <= REL_T, rel.max()


def test_eight_materials_ragged_random_labels(fc, orc):
    """All eight material slots (labels 0..7, the head-like phantom's
    table): per-material path lengths and T of every ray against the
    oracle on a ragged grid."""
    wl = W.scaled(W.WORKLOADS["head_surrogate"], n_u=70, n_v=45, n_angles=7, nx=24, ny=20, nz=16,
                  dx=0.25, dy=0.25, dz=0.25, du=0.12, dv=0.12)
    g = wl.geom
    assert len(wl.labels) == 8
    lab = np.random.default_rng(25).integers(0, 8, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    assert (np.bincount(lab.ravel(), minlength=8) > 0).all()
    sc = _scanner(fc, wl, lab, noise=False)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
        L = torch.empty((g.n_angles, g.n_v, g.n_u, 8), dtype=torch.float32, device="cuda")
        fc.fc_project_lengths(sc.h, 0, g.n_angles, L)
        torch.cuda.synchronize()
        L = L.cpu().numpy().reshape(-1, 8)
    finally:
        sc.close()
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    assert np.max(np.abs(T - Tr) / Tr) <= REL_T
    k, v, u = np.meshgrid(np.arange(g.n_angles), np.arange(g.n_v), np.arange(g.n_u), indexing="ij")
    Lr, _ = orc.rays(g, lab, w, d, wl.mu(), np.stack([k.ravel(), v.ravel(), u.ravel()], 1))
    assert (Lr[:, 7] > 0).sum() > 100                  # slot 7 is exercised
    assert np.abs(L - Lr).max() < 2e-4


def test_head_phantom_reduced_every_ray(fc, orc):
    """The head-like phantom (8 materials, 40 random ellipsoids) at 64^3
    voxels of 0.25 cm, 24 projections of 128 x 128, 120 bins: every ray."""
    wl = W.scaled(W.WORKLOADS["head_surrogate"], n_u=128, n_v=128, n_angles=24, nx=64, ny=64,
                  nz=64, dx=0.25, dy=0.25, dz=0.25, du=0.2, dv=0.2)
    g = wl.geom
    lab = wl.make_phantom()
    sc = _scanner(fc, wl, lab, noise=False)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
    finally:
        sc.close()
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    assert np.max(np.abs(T - Tr) / Tr) <= REL_T


def test_head_phantom_full_size_sampled(fc, orc, precision):
    """Full head-like scan (256^3 voxels of 0.0625 cm, 360 projections of
    512 x 512, 120 bins): T at 4000 sampled rays of five projections."""
    wl = W.WORKLOADS["head_surrogate"]
    g = wl.geom
    lab = wl.make_phantom()
    ks = [0, 77, 180, 251, 359]
    sc = _scanner(fc, wl, lab, noise=False)
    try:
        T = np.stack([_project(fc, sc, fc.FC_OUT_PRIMARY, k, 1)[0] for k in ks])
    finally:
        sc.close()
    rng = np.random.default_rng(26)
    n = 4000
    kk = rng.integers(0, len(ks), n)
    rows = rng.integers(0, g.n_v, n)
    cols = rng.integers(0, g.n_u, n)
    w, d = wl.spectrum()
    Lr, Tr = orc.rays(g, lab, w, d, wl.mu(), np.stack([np.array(ks)[kk], rows, cols], 1))
    assert (Lr[:, 7] > 0).sum() > 10                   # teeth crossed by some sampled rays
    precision("T (primary)", "head 256^3, 360x512x512, 120 bins, %d rays" % n,
              np.max(np.abs(T[kk, rows, cols] - Tr) / Tr), REL_T)
    assert np.max(np.abs(T[kk, rows, cols] - Tr) / Tr) <= REL_T


def test_primary_thin_slab_band_edges(fc, orc):
    """A 3-slice slab seen by a 45-row detector: only a band of rows can meet
    the voxels, so the projector traces 8-row blocks around it and a store
    kernel writes the other rows.  Every ray is checked against the oracle,
    and rays that miss the voxels must give exactly T = 1."""
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=45, n_angles=9, nx=24, ny=20, nz=3,
                  dx=0.25, dy=0.25, dz=0.1, du=0.12, dv=0.05)
    g = wl.geom
    rng = np.random.default_rng(22)
    lab = rng.integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    sc = _scanner(fc, wl, lab)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
    finally:
        sc.close()
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    rel = np.abs(T - Tr) / Tr
    assert rel.max() <= REL_T, rel.max()
    miss = Tr == 1.0
    rows_hit = np.where((~miss).any(axis=(0, 2)))[0]
    assert 0 < len(rows_hit) < g.n_v // 2          # a band, not the whole detector
    assert np.all(T[miss] == 1.0)


def test_intensity_thin_band_every_pixel(fc, orc):
    """A 3-slice slab on a 240-row detector with a 5 px scatter kernel: the
    projector traces a band of rows, the row pass computes the 64-line tiles
    holding it, the column pass the 128-row tiles within the larger blur
    radius of it, and a store kernel writes the rest.  Every pixel of I (and
    of the rate of the Sec. II.G noise order) against the oracle."""
    import dataclasses
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=240, n_angles=6, nx=24, ny=20, nz=3,
                  dx=0.25, dy=0.25, dz=0.1, du=0.12, dv=0.05)
    wl = dataclasses.replace(wl, scatter_sigma_px=5.0, psf_sigma_px=0.8)
    g = wl.geom
    lab = np.random.default_rng(24).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    sc = _scanner(fc, wl, lab, noise=False)
    try:
        I = _project(fc, sc, fc.FC_OUT_INTENSITY)
        fc.fc_set_noise_order(sc.h, fc.FC_NOISE_BEFORE_PSF)
        lam = _project(fc, sc, fc.FC_OUT_INTENSITY)
    finally:
        sc.close()
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    hit_rows = np.where((Tr < 1.0).any(axis=(0, 2)))[0]
    assert 0 < len(hit_rows) < 20          # a narrow band: most rows are filled
    Ir = orc.intensity(Tr, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    assert np.max(np.abs(I - Ir) / Ir) <= REL_T
    lam_r, _ = orc.counts_noise_before_psf(Tr, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    assert np.max(np.abs(lam - lam_r) / lam_r) <= REL_T


def test_tiny_geometry_and_empty_angle_range(fc, orc):
    """A volume smaller than one 8-voxel brick on every axis (5 x 3 x 2, random
    labels) seen by a 3 x 4 detector: every ray's T and the reconstruction
    (a 3-column ramp filter) against the oracle; an empty angle range
    leaves the output untouched."""
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=3, n_v=4, n_angles=5, nx=5, ny=3, nz=2,
                  dx=0.5, dy=0.5, dz=0.5, du=0.3, dv=0.3)
    g = wl.geom
    lab = np.random.default_rng(23).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    sc = _scanner(fc, wl, lab)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
        out = torch.full((1, g.n_v, g.n_u), -7.0, dtype=torch.float32, device="cuda")
        fc.fc_project(sc.h, 2, 0, fc.FC_OUT_PRIMARY, out)
        torch.cuda.synchronize()
        assert bool(torch.all(out == -7.0))
    finally:
        sc.close()
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    assert (Tr < 1.0).all()                       # every ray crosses the voxels
    rel = np.abs(T - Tr) / Tr
    assert rel.max() <= REL_T, rel.max()
    counts = orc.intensity(Tr, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0).astype(np.float32)
    vol, _ = _recon_gpu(fc, wl, counts, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    assert np.max(np.abs(vol - vref)) <= 5e-4 * np.max(np.abs(vref)), np.max(np.abs(vol - vref))


@pytest.fixture(scope="module")
def small_kv_ref(orc):
    wl = W.WORKLOADS["small_kv"]
    g = wl.geom
    lab = wl.make_phantom()
    w, d = wl.spectrum()
    T = orc.project_T(g, lab, w, d, wl.mu())
    I = orc.intensity(T, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    return wl, lab, T, I


def test_primary_small_kv(fc, small_kv_ref):
    wl, lab, Tr, _ = small_kv_ref
    sc = _scanner(fc, wl, lab)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
    finally:
        sc.close()
    rel = np.abs(T - Tr) / Tr
    assert rel.max() <= REL_T, rel.max()


def test_intensity_small_kv(fc, small_kv_ref):
    wl, lab, _, Ir = small_kv_ref
    sc = _scanner(fc, wl, lab)
    try:
        I = _project(fc, sc, fc.FC_OUT_INTENSITY)
    finally:
        sc.close()
    rel = np.abs(I - Ir) / Ir
    assert rel.max() <= REL_T, rel.max()


def test_poisson_bit_identical(fc, orc, small_kv_ref, precision):
    wl, _, _, Ir = small_kv_ref
    rng = np.random.default_rng(5)
    lam = (Ir[:20] * rng.uniform(0.0, 1.0, Ir[:20].shape) ** 6).astype(np.float32)
    lam[0, 0, :8] = [0.0, -1.0, 1e-3, 0.5, 9.999, 10.0, 10.001, 2e7]
    ref = orc.poisson(lam, seed=wl.seed, k0=3)
    d_lam = torch.from_numpy(lam).cuda()
    d_out = torch.empty_like(d_lam)
    n, nv, nu = lam.shape
    fc.fc_poisson(d_lam, d_out, n, nv, nu, 3, wl.seed)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    precision("Poisson counts", "%d draws, identical rates" % got.size,
              np.count_nonzero(got.view(np.uint32) != ref.view(np.uint32)), 0, "mismatched draws")
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), \
        np.count_nonzero(got != ref)
    assert (lam < 10).sum() > 100  # both sampler branches exercised


def test_counts_fused_equals_standalone_and_repeats(fc, small_kv_ref):
    wl, lab, _, _ = small_kv_ref
    sc = _scanner(fc, wl, lab, noise=True)
    try:
        I = _project(fc, sc, fc.FC_OUT_INTENSITY)
        K1 = _project(fc, sc, fc.FC_OUT_COUNTS)
        K2 = np.concatenate([_project(fc, sc, fc.FC_OUT_COUNTS, 0, 37),
                             _project(fc, sc, fc.FC_OUT_COUNTS, 37, None)])
    finally:
        sc.close()
    d_I = torch.from_numpy(I).cuda()
    d_K = torch.empty_like(d_I)
    fc.fc_poisson(d_I, d_K, *I.shape, 0, wl.seed)
    torch.cuda.synchronize()
    assert np.array_equal(K1.view(np.uint32), K2.view(np.uint32))
    assert np.array_equal(K1.view(np.uint32), d_K.cpu().numpy().view(np.uint32))
    z = (K1 - I) / np.sqrt(I)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def _recon_gpu(fc, wl, counts, lab=None):
    g = wl.geom
    sc = _scanner(fc, wl, lab)
    try:
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        hu = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device="cuda")
        fc.fc_reconstruct(sc.h, np.ascontiguousarray(counts, np.float32), vol_mu=vol, vol_hu=hu)
        torch.cuda.synchronize()
        return vol.cpu().numpy(), hu.cpu().numpy()
    finally:
        sc.close()


def test_reconstruct_small_kv(fc, orc, small_kv_ref):
    wl, lab, _, Ir = small_kv_ref
    g = wl.geom
    counts = Ir.astype(np.float32)
    vol, hu = _recon_gpu(fc, wl, counts, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    mask = W.water_roi_mask(g)
    huref, mu_w = orc.hu(vref, mask)
    assert np.max(np.abs(vol - vref)) <= 5e-4 * mu_w, np.max(np.abs(vol - vref)) / mu_w
    assert np.max(np.abs(hu - huref)) <= HU_TOL, np.max(np.abs(hu - huref))


def test_reconstruct_ragged_volume(fc, orc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=45, n_angles=30, nx=37, ny=29, nz=11,
                  dx=0.3, dy=0.3, dz=0.3, du=0.2, dv=0.2)
    g = wl.geom
    lab = wl.make_phantom()
    w, d = wl.spectrum()
    T = orc.project_T(g, lab, w, d, wl.mu())
    counts = orc.intensity(T, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0).astype(np.float32)
    vol, _ = _recon_gpu(fc, wl, counts, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    mu_w = float(np.mean(vref[W.water_roi_mask(g)]))
    assert np.max(np.abs(vol - vref)) <= 5e-4 * mu_w


@pytest.mark.parametrize("n_u", [1, 2, 5, 33, 97, 600])
def test_reconstruct_detector_widths(fc, orc, n_u):
    """Edge cases of the ramp filter's row layout and per-warp offset range:
    a one-pixel row, even and odd widths, rows of one and of two warps.
    Reconstruction of random counts against the oracle's FDK."""
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=n_u, n_v=6, n_angles=9, nx=8, ny=7, nz=3,
                  dx=0.05, dy=0.05, dz=0.05, du=0.08, dv=0.08)
    g = wl.geom
    counts = (np.random.default_rng(n_u).uniform(0.3, 1.0, (g.n_angles, g.n_v, g.n_u)) *
              wl.n0).astype(np.float32)
    sc = _scanner(fc, wl, None)
    try:
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        fc.fc_reconstruct(sc.h, counts, vol_mu=vol)
        torch.cuda.synchronize()
        got = vol.cpu().numpy()
    finally:
        sc.close()
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    assert np.max(np.abs(vref)) > 0.0
    assert np.max(np.abs(got - vref)) <= 5e-4 * np.max(np.abs(vref)), np.max(np.abs(got - vref))


def test_beer_lambert_single_bin_uniform(fc):
    """One energy bin, D = 1, uniform water box: T = exp(-mu * chord)."""
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=33, n_v=9, n_angles=5, nx=16, ny=16, nz=16,
                  dx=0.5, dy=0.5, dz=0.5, du=0.4, dv=0.4)
    g = wl.geom
    h = fc.fc_create(0)
    try:
        fc.fc_set_geometry(h, g)
        fc.fc_set_phantom(h, np.ones((16, 16, 16), np.uint8), 2)
        fc.fc_set_spectrum_detector(h, [1.0], [1.0], np.array([[0.0, 0.2]]), 0.0, 0.0, 0.0, 1.0, 0, 0)
        T = torch.empty((g.n_angles, g.n_v, g.n_u), device="cuda")
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_PRIMARY, T)
        torch.cuda.synchronize()
        T = T.cpu().numpy()
        # blur with sigma 0 and SPR 0 is the identity times N0 = 1, up to the
        # tensor-core blur's bf16 hi + lo split of the samples (2^-17 relative)
        I = torch.empty_like(torch.from_numpy(T)).cuda()
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_INTENSITY, I)
        torch.cuda.synchronize()
        np.testing.assert_allclose(I.cpu().numpy(), T, rtol=2.0**-16, atol=0)
    finally:
        fc.fc_destroy(h)
    for k in range(g.n_angles):
        th = 2 * math.pi * k / g.n_angles
        for iv in range(g.n_v):
            for iu in range(g.n_u):
                u = (iu - (g.n_u - 1) / 2) * g.du
                v = (iv - (g.n_v - 1) / 2) * g.dv
                S = np.array([g.sad * math.cos(th), g.sad * math.sin(th), 0.0])
                P = np.array([-(g.sdd - g.sad) * math.cos(th) - u * math.sin(th),
                              -(g.sdd - g.sad) * math.sin(th) + u * math.cos(th), v])
                D = P - S
                t0, t1 = 0.0, 1.0
                for a in range(3):
                    lo, hi = sorted(((-4.0 - S[a]) / D[a], (4.0 - S[a]) / D[a])) if D[a] else (-1e9, 1e9)
                    t0, t1 = max(t0, lo), min(t1, hi)
                chord = max(0.0, t1 - t0) * np.linalg.norm(D)
                assert T[k, iv, iu] == pytest.approx(math.exp(-0.2 * chord), rel=1e-5)


def test_errors_are_reported(fc):
    wl = W.WORKLOADS["small_kv"]
    g = wl.geom
    h = fc.fc_create(0)
    try:
        with pytest.raises(fc.FastcatError) as ei:
            fc.fc_project(h, 0, 1, fc.FC_OUT_NONE)
        assert ei.value.code == fc.FC_ESTATE
        fc.fc_set_geometry(h, g)
        bad = np.zeros((g.nz, g.ny, g.nx), np.uint8)
        bad[3, 4, 5] = 9
        with pytest.raises(fc.FastcatError) as ei:
            fc.fc_set_phantom(h, bad, 7)
        assert ei.value.code == fc.FC_EINVAL and "n_mat" in fc.fc_last_error()
        fc.fc_set_phantom(h, np.ones((g.nz, g.ny, g.nx), np.uint8), 7)
        w, d = wl.spectrum()
        fc.fc_set_spectrum_detector(h, w, d, wl.mu(), 0.6, 20.0, 0.2, 1e5, 0, 0)
        with pytest.raises(fc.FastcatError):
            fc.fc_project(h, 80, 20, fc.FC_OUT_NONE)
        with pytest.raises(fc.FastcatError):
            fc.fc_set_spectrum_detector(h, w, d, wl.mu(), 70.0, 20.0, 0.2, 1e5, 0, 0)
        fc.fc_project(h, 5, 0, fc.FC_OUT_NONE)  # empty range is a no-op
    finally:
        fc.fc_destroy(h)


# ------------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def catphan_full(fc):
    wl = W.WORKLOADS["catphan_kv"]
    lab = wl.make_phantom()
    sc = _scanner(fc, wl, lab, noise=False)
    try:
        T = _project(fc, sc, fc.FC_OUT_PRIMARY)
        I = _project(fc, sc, fc.FC_OUT_INTENSITY)
    finally:
        sc.close()
    return wl, lab, T, I


def test_full_catphan_primary_sampled(orc, catphan_full, precision):
    wl, lab, T, _ = catphan_full
    g = wl.geom
    rng = np.random.default_rng(1)
    n = 4000
    rays = np.stack([rng.integers(0, g.n_angles, n), rng.integers(170, 214, n),
                     rng.integers(0, g.n_u, n)], 1)
    # plus one full row through the insert ring at a few angles
    extra = [(k, 192, u) for k in (0, 45, 91, 180, 359) for u in range(g.n_u)]
    rays = np.concatenate([rays, np.array(extra)])
    w, d = wl.spectrum()
    _, Tr = orc.rays(g, lab, w, d, wl.mu(), rays)
    got = T[rays[:, 0], rays[:, 1], rays[:, 2]]
    precision("T (primary)", "catphan_kv 256^2x10, 360x512x384, %d rays" % len(rays),
              np.max(np.abs(got - Tr) / Tr), REL_T)
    assert np.max(np.abs(got - Tr) / Tr) <= REL_T


def test_full_catphan_intensity_sampled(orc, catphan_full, precision):
    """I at sampled pixels: the oracle blurs its own T over the projections
    that contain the samples."""
    wl, lab, _, I = catphan_full
    g = wl.geom
    w, d = wl.spectrum()
    ks = [0, 123, 301]
    Tr = np.concatenate([orc.project_T(g, lab, w, d, wl.mu(), a0=k, na=1) for k in ks])
    Ir = orc.intensity(Tr, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    got = I[ks]
    precision("I (blur + scatter)", "catphan_kv, 3 full projections", np.max(np.abs(got - Ir) / Ir), REL_T)
    assert np.max(np.abs(got - Ir) / Ir) <= REL_T


def test_full_catphan_reconstruct(fc, orc, catphan_full, precision):
    """Full-size FDK of oracle-made noise-free counts, every voxel."""
    wl, lab, _, _ = catphan_full
    g = wl.geom
    w, d = wl.spectrum()
    Tr = orc.project_T(g, lab, w, d, wl.mu())
    Ir = orc.intensity(Tr, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    counts = Ir.astype(np.float32)
    vol, hu = _recon_gpu(fc, wl, counts, lab)
    # oracle FDK on the detector rows the volume projects onto (others are
    # never sampled); generous margin
    zmax = (g.nz - 1) / 2 * g.dz
    rmax = math.hypot(g.nx * g.dx / 2, g.ny * g.dy / 2)
    vmax = zmax * g.sdd / (g.sad - rmax) / g.dv
    lo = max(0, int(math.floor((g.n_v - 1) / 2 - vmax)) - 4)
    hi = min(g.n_v - 1, int(math.ceil((g.n_v - 1) / 2 + vmax)) + 4)
    q = orc.fdk_weight(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    f = np.zeros_like(q)
    f[:, lo:hi + 1] = orc.ramp_filter(np.ascontiguousarray(q[:, lo:hi + 1]), g.du * g.sad / g.sdd)
    vref = orc.backproject(g, f)
    mask = W.water_roi_mask(g)
    huref, mu_w = orc.hu(vref, mask)
    precision("mu (FDK)", "catphan_kv, every voxel", np.max(np.abs(vol - vref)) / mu_w, 5e-4, "of mu_water")
    precision("HU", "catphan_kv, every voxel", np.max(np.abs(hu - huref)), HU_TOL, "HU")
    assert np.max(np.abs(vol - vref)) <= 5e-4 * mu_w
    assert np.max(np.abs(hu - huref)) <= HU_TOL


def test_full_paper_mv_sampled(fc, orc, precision):
    """Paper-scale MV case (1024^2 x 10 voxels of 0.015625 cm, 1024 x 768
    detector, 60 MV bins): primary signal at sampled rays of six projections
    and the intensity of one whole projection against the oracle."""
    wl = W.WORKLOADS["paper_mv"]
    g = wl.geom
    lab = wl.make_phantom()
    sc = _scanner(fc, wl, lab, noise=False)
    ks = [0, 97, 211, 360, 531, 719]
    try:
        T = np.stack([_project(fc, sc, fc.FC_OUT_PRIMARY, k, 1)[0] for k in ks])
        I = _project(fc, sc, fc.FC_OUT_INTENSITY, 531, 1)
        L = torch.empty((1, g.n_v, g.n_u, 7), dtype=torch.float32, device="cuda")
        fc.fc_project_lengths(sc.h, 211, 1, L)
        torch.cuda.synchronize()
        L = L.cpu().numpy()[0]
    finally:
        sc.close()
    rng = np.random.default_rng(2)
    n = 3000
    kk = rng.integers(0, len(ks), n)
    rows = rng.integers(g.n_v // 2 - 16, g.n_v // 2 + 16, n)
    cols = rng.integers(0, g.n_u, n)
    rays = np.stack([np.array(ks)[kk], rows, cols], 1)
    w, d = wl.spectrum()
    Lr, Tr = orc.rays(g, lab, w, d, wl.mu(), rays)
    precision("T (primary)", "paper_mv 1024^2x10, 720x1024x768, %d rays" % n,
              np.max(np.abs(T[kk, rows, cols] - Tr) / Tr), REL_T)
    assert np.max(np.abs(T[kk, rows, cols] - Tr) / Tr) <= REL_T
    sel = np.array(ks)[kk] == 211
    eL = np.max(np.abs(L[rows[sel], cols[sel]] - Lr[sel]))
    precision("L (path lengths)", "paper_mv, projection 211, %d rays" % sel.sum(), eL, 2e-4, "cm")
    assert eL < 2e-4
    Tp = orc.project_T(g, lab, w, d, wl.mu(), a0=531, na=1)
    Ir = orc.intensity(Tp, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    precision("I (blur + scatter)", "paper_mv, projection 531 (every pixel)", np.max(np.abs(I - Ir) / Ir), REL_T)
    assert np.max(np.abs(I - Ir) / Ir) <= REL_T

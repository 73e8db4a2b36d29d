"""GPU parity of the FDK backprojector variants (fc_set_backprojector)
against the FP64 oracle: the chunked kernel, its 32-register variant, the
thin-slab kernel and its quarter-turn form (one column set-up shared by the
four columns a quarter turn maps onto one another), each forced on small
ragged cases and on the full paper-scale grid (1024^2 x 10 voxels, 720
projections).  Tolerance |d mu| <= 5e-4 mu_water (0.5 HU)."""
import math

import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MU_TOL = 5e-4


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


def _thin_slab(nx=37, ny=29, nz=10, n_angles=24):
    """A slab whose z pitch projects to about half a detector row (the slab
    kernel applies), ragged in x and y."""
    return W.scaled(W.WORKLOADS["small_kv"], n_u=96, n_v=40, n_angles=n_angles, nx=nx, ny=ny,
                    nz=nz, dx=0.09, dy=0.09, dz=0.03, du=0.06, dv=0.09)


def _recon(fc, wl, counts, variant, lab=None):
    g = wl.geom
    sc = fc.Scanner(wl, labels=wl.make_phantom() if lab is None else lab, noise=False)
    try:
        fc.fc_set_backprojector(sc.h, variant)
        used = fc.fc_backprojector_in_use(sc.h)
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        c = counts if isinstance(counts, torch.Tensor) else np.ascontiguousarray(counts, np.float32)
        fc.fc_reconstruct(sc.h, c, vol_mu=vol)
        torch.cuda.synchronize()
        return vol.cpu().numpy(), used
    finally:
        sc.close()


def _oracle_counts(orc, wl, lab=None):
    g = wl.geom
    lab = wl.make_phantom() if lab is None else lab
    w, d = wl.spectrum()
    T = orc.project_T(g, lab, w, d, wl.mu())
    return orc.intensity(T, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0).astype(np.float32)


@pytest.mark.parametrize("nz", [10, 1, 16, 7])
def test_variants_thin_slab(fc, orc, nz):
    wl = _thin_slab(nz=nz)
    g = wl.geom
    assert fc_step(g) <= 0.98
    lab = np.random.default_rng(40 + nz).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    counts = _oracle_counts(orc, wl, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    scale = float(np.max(np.abs(vref)))
    vols = {}
    for req in (fc.FC_BP_AUTO, fc.FC_BP_SLAB, fc.FC_BP_CHUNKED, fc.FC_BP_CHUNKED_DENSE):
        vol, used = _recon(fc, wl, counts, req)
        if req == fc.FC_BP_AUTO:
            assert used == fc.FC_BP_SLAB
        else:
            assert used == req
        err = np.max(np.abs(vol - vref))
        assert err <= MU_TOL * scale, (req, err / scale)
        vols[req] = vol
    # the slab kernel repeats the chunked kernel's per-slice arithmetic (the
    # v coordinate of a slice formed from another origin)
    d = np.max(np.abs(vols[fc.FC_BP_SLAB] - vols[fc.FC_BP_CHUNKED]))
    assert d <= 1e-5 * scale, d / scale


def quad_layout(g):
    """Whether the thin-slab quarter-turn kernel reads the filtered rows
    interleaved by quarter turn: the in-plane voxel pitch projects to at
    most one detector column at the axis."""
    return g.dx * g.sdd <= g.du * g.sad


@pytest.mark.parametrize("nz,n_u,dxy", [(10, 96, 0.09), (1, 96, 0.09), (16, 96, 0.09), (7, 96, 0.09),
                                        (10, 40, 0.09), (10, 96, 0.03), (1, 96, 0.03), (16, 96, 0.03),
                                        (7, 96, 0.03), (10, 24, 0.03)])
def test_quarter_turn_thin_slab(fc, orc, nz, n_u, dxy):
    """The quarter-turn kernel on a square grid with an even side (38: a
    19 x 19 quadrant of base columns, ragged against the 32 x 8 CTA tile)
    and 24 projections over 360 degrees; n_u = 40 (24 at the finer pitch)
    leaves the volume's shadow wider than the detector (the clamped
    coordinates).  The 0.09 cm voxel pitch projects to 2.25 detector
    columns (filtered rows in projection order), the 0.03 cm pitch to 0.75
    (filtered rows interleaved by quarter turn).  Compared with the oracle
    and with the thin-slab kernel."""
    wl = _thin_slab(nx=38, ny=38, nz=nz)
    wl = W.scaled(wl, n_u=n_u, dx=dxy, dy=dxy)
    g = wl.geom
    assert fc_step(g) <= 0.98 and g.n_angles % 4 == 0 and abs(g.arc - 2 * math.pi) < 1e-15
    assert quad_layout(g) == (dxy < 0.05)
    lab = np.random.default_rng(60 + nz).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    counts = _oracle_counts(orc, wl, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    scale = float(np.max(np.abs(vref)))
    vols = {}
    for req in (fc.FC_BP_AUTO, fc.FC_BP_SLAB_SYM, fc.FC_BP_SLAB):
        vol, used = _recon(fc, wl, counts, req)
        assert used == (fc.FC_BP_SLAB_SYM if req == fc.FC_BP_AUTO else req)
        err = np.max(np.abs(vol - vref))
        assert err <= MU_TOL * scale, (req, err / scale)
        vols[req] = vol
    # the same sums in another order and from rotated trigonometry
    d = np.max(np.abs(vols[fc.FC_BP_SLAB_SYM] - vols[fc.FC_BP_SLAB]))
    assert d <= 1e-5 * scale, d / scale
    # deterministic: the two halves of the projections add onto zero
    vol2, _ = _recon(fc, wl, counts, fc.FC_BP_SLAB_SYM)
    assert np.array_equal(vol2, vols[fc.FC_BP_SLAB_SYM])


@pytest.mark.parametrize("n_u", [128, 240])
def test_quarter_turn_chunked(fc, orc, n_u):
    """The quarter-turn kernel on a thick slab (the z pitch projects to about
    five detector rows: every slice loads its two rows), 38 x 38 x 12 voxels
    over 24 projections; n_u = 128 leaves the volume's shadow wider than the
    detector (clamped coordinates).  Compared with the oracle and with the
    chunked kernel, repeated bit for bit."""
    wl = W.scaled(W.WORKLOADS["small_kv"], n_angles=24, nx=38, ny=38, nz=12, n_u=n_u)
    g = wl.geom
    assert fc_step(g) > 1.0
    lab = np.random.default_rng(70 + n_u).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    counts = _oracle_counts(orc, wl, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    scale = float(np.max(np.abs(vref)))
    vols = {}
    for req in (fc.FC_BP_AUTO, fc.FC_BP_CHUNKED_SYM, fc.FC_BP_CHUNKED):
        vol, used = _recon(fc, wl, counts, req)
        assert used == (fc.FC_BP_CHUNKED_SYM if req == fc.FC_BP_AUTO else req)
        err = np.max(np.abs(vol - vref))
        assert err <= MU_TOL * scale, (req, err / scale)
        vols[req] = vol
    d = np.max(np.abs(vols[fc.FC_BP_CHUNKED_SYM] - vols[fc.FC_BP_CHUNKED]))
    assert d <= 1e-5 * scale, d / scale
    vol2, _ = _recon(fc, wl, counts, fc.FC_BP_CHUNKED_SYM)
    assert np.array_equal(vol2, vols[fc.FC_BP_CHUNKED_SYM])


@pytest.mark.parametrize("thick", [False, True])
def test_variant_switch_on_one_handle(fc, orc, thick):
    """The quarter-turn kernels read the filtered rows interleaved by quarter
    turn, the others in projection order, and the zero padding of one layout
    holds data in the other: one handle switched between a quarter-turn
    kernel and a plain one (and back) gives, every time, the volume of a
    fresh handle bit for bit, with a detector narrower than the volume's
    shadow (the clamped taps read the padding)."""
    if thick:
        wl = W.scaled(W.WORKLOADS["small_kv"], n_angles=24, nx=38, ny=38, nz=12, n_u=128)
        sym, plain = fc.FC_BP_CHUNKED_SYM, fc.FC_BP_CHUNKED
    else:
        wl = W.scaled(_thin_slab(nx=38, ny=38, nz=10), n_u=24, dx=0.03, dy=0.03)
        sym, plain = fc.FC_BP_SLAB_SYM, fc.FC_BP_SLAB
    g = wl.geom
    assert quad_layout(g) != thick
    lab = np.random.default_rng(90 + thick).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    counts = _oracle_counts(orc, wl, lab)
    fresh = {v: _recon(fc, wl, counts, v, lab)[0] for v in (sym, plain)}
    sc = fc.Scanner(wl, labels=lab, noise=False)
    try:
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        for v in (sym, plain, sym, plain):
            fc.fc_set_backprojector(sc.h, v)
            assert fc.fc_backprojector_in_use(sc.h) == v
            fc.fc_reconstruct(sc.h, counts, vol_mu=vol)
            torch.cuda.synchronize()
            assert np.array_equal(vol.cpu().numpy(), fresh[v]), v
    finally:
        sc.close()


@pytest.mark.parametrize("dxy", [0.09, 0.03])
def test_quarter_turn_thin_slab_unequal_runs(fc, orc, dxy):
    """A 256 x 256 x 11 thin slab: 11 slices do not split into equal runs of
    at most 5, so the quarter-turn kernel takes runs of unequal length (the
    form with the run-length test in its slice loop); with filtered rows in
    projection order (0.09 cm voxels) and interleaved by quarter turn (0.03
    cm, the volume's shadow wider than the detector)."""
    wl = W.scaled(_thin_slab(nx=256, ny=256, nz=11, n_angles=24), dx=dxy, dy=dxy)
    g = wl.geom
    assert fc_step(g) <= 0.98 and quad_layout(g) == (dxy < 0.05)
    lab = np.random.default_rng(81).integers(0, 7, size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    counts = _oracle_counts(orc, wl, lab)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    scale = float(np.max(np.abs(vref)))
    vol, used = _recon(fc, wl, counts, fc.FC_BP_AUTO)
    assert used == fc.FC_BP_SLAB_SYM
    assert np.max(np.abs(vol - vref)) <= MU_TOL * scale
    vs, _ = _recon(fc, wl, counts, fc.FC_BP_SLAB)
    assert np.max(np.abs(vol - vs)) <= 1e-5 * scale


@pytest.mark.parametrize("change", ["angles", "arc", "rect", "odd", "pitch"])
def test_quarter_turn_refused_without_symmetry(fc, change):
    """Without the quarter-turn symmetry (projections not a multiple of 4,
    a partial arc, a rectangular or odd grid, unequal x and y pitch) the
    kernel is refused and the default falls back to the thin-slab kernel."""
    kw = {"angles": dict(n_angles=22), "arc": dict(arc=1.5 * math.pi),
          "rect": dict(nx=38, ny=36), "odd": dict(nx=37, ny=37), "pitch": dict(nx=38, ny=38, dy=0.085)}[change]
    base = dict(nx=38, ny=38)
    base.update({k: v for k, v in kw.items() if k in ("nx", "ny")})
    wl = _thin_slab(**base)
    rest = {k: v for k, v in kw.items() if k not in ("nx", "ny")}
    if rest:
        wl = W.scaled(wl, **rest)
    assert fc_step(wl.geom) <= 0.98
    sc = fc.Scanner(wl, noise=False)
    try:
        assert fc.fc_backprojector_in_use(sc.h) == fc.FC_BP_SLAB
        for req in (fc.FC_BP_SLAB_SYM, fc.FC_BP_CHUNKED_SYM):
            fc.fc_set_backprojector(sc.h, req)
            with pytest.raises(fc.FastcatError) as ei:
                fc.fc_backprojector_in_use(sc.h)
            assert ei.value.code == fc.FC_EINVAL
    finally:
        sc.close()


def fc_step(g):
    """Largest projected z pitch in detector rows (host restatement of the
    condition the slab kernel needs)."""
    rmax = math.hypot(0.5 * g.nx * g.dx, 0.5 * g.ny * g.dy)
    return g.dz * g.sdd / (g.sad - rmax) / g.dv


def test_chunked_dense_small_kv(fc, orc):
    """The 32-register chunked kernel (the default for grids of two or more
    waves) forced on the 64^3 small kV case."""
    wl = W.WORKLOADS["small_kv"]
    g = wl.geom
    counts = _oracle_counts(orc, wl)
    vref = orc.fdk(g, counts.astype(np.float64), orc.i_flood(wl.n0, wl.spr))
    mu_w = float(np.mean(vref[W.water_roi_mask(g)]))
    for req in (fc.FC_BP_CHUNKED_DENSE, fc.FC_BP_CHUNKED):
        vol, used = _recon(fc, wl, counts, req)
        assert used == req
        assert np.max(np.abs(vol - vref)) <= MU_TOL * mu_w, (req, np.max(np.abs(vol - vref)) / mu_w)


def test_slab_refused_where_it_does_not_apply(fc):
    wl = W.WORKLOADS["small_kv"]          # z pitch ~5 detector rows
    assert fc_step(wl.geom) > 1.0
    sc = fc.Scanner(wl, noise=False)
    try:
        assert fc.fc_backprojector_in_use(sc.h) in (fc.FC_BP_CHUNKED, fc.FC_BP_CHUNKED_DENSE)
        fc.fc_set_backprojector(sc.h, fc.FC_BP_SLAB)
        with pytest.raises(fc.FastcatError) as ei:
            fc.fc_backprojector_in_use(sc.h)
        assert ei.value.code == fc.FC_EINVAL
        fc.fc_project(sc.h, 0, wl.geom.n_angles, fc.FC_OUT_NONE)
        with pytest.raises(fc.FastcatError) as ei:
            fc.fc_reconstruct(sc.h)
        assert ei.value.code == fc.FC_EINVAL
        with pytest.raises(fc.FastcatError):
            fc.fc_set_backprojector(sc.h, 7)
        fc.fc_set_backprojector(sc.h, fc.FC_BP_AUTO)
        fc.fc_reconstruct(sc.h)
    finally:
        sc.close()


def _synthetic_band_counts(g, rows, flood, seed=7):
    """Counts on detector rows `rows` of every projection: the flood times
    exp(-p), p a water cylinder's chord (mu 0.05 / cm, radius 8 cm at the
    isocentre) plus seeded smooth random modes in u, v and the angle."""
    rng = np.random.default_rng(seed)
    u = (np.arange(g.n_u) - (g.n_u - 1) / 2) * g.du * g.sad / g.sdd
    v = (rows - (g.n_v - 1) / 2) * g.dv * g.sad / g.sdd
    th = g.theta0 + g.arc * np.arange(g.n_angles) / g.n_angles
    chord = 2.0 * np.sqrt(np.clip(64.0 - u * u, 0.0, None))
    p = np.broadcast_to(0.05 * chord, (g.n_angles, len(rows), g.n_u)).copy()
    for _ in range(6):
        a, fu, fv, ft, ph = rng.uniform(0.005, 0.02), rng.uniform(0.1, 2.0), rng.uniform(1.0, 20.0), \
            rng.integers(1, 4), rng.uniform(0, 2 * np.pi)
        p += a * (np.sin(fu * u[None, None, :] + fv * v[None, :, None] + ft * th[:, None, None] + ph)
                  * (chord > 0)[None, None, :])
    return (flood * np.exp(-p)).astype(np.float32)


def test_full_paper_mv_reconstruct_variants(fc, orc, precision):
    """Full paper-scale grid (1024^2 x 10 voxels of 0.015625 cm, 720
    projections of 1024 x 768): synthetic counts on the rows the volume
    projects onto, flood elsewhere.  The oracle reconstructs from a
    32-row detector centred like the full one (the same pixel centres; no
    voxel projects outside it); every voxel of the quarter-turn kernel (the
    default here), the thin-slab kernel and the 32-register chunked kernel
    is compared."""
    wl = W.WORKLOADS["paper_mv"]
    g = wl.geom
    flood = wl.n0 * (1.0 + wl.spr)
    assert fc_step(g) <= 0.98
    crop = 32
    r0 = g.n_v // 2 - crop // 2
    rows = np.arange(r0, r0 + crop)
    band = _synthetic_band_counts(g, rows, flood)
    gc = W.Geometry(g.sad, g.sdd, g.n_u, crop, g.du, g.dv, g.n_angles, g.nx, g.ny, g.nz,
                    g.dx, g.dy, g.dz, g.theta0, g.arc)
    assert 2 * r0 == g.n_v - crop           # crop row r has full-detector row r0 + r's centre
    q = orc.fdk_weight(gc, band.astype(np.float64), flood)
    f = orc.ramp_filter(q, g.du * g.sad / g.sdd)
    vref = orc.backproject(gc, f)
    mu_w = float(np.mean(vref[W.water_roi_mask(g)]))
    counts = torch.full((g.n_angles, g.n_v, g.n_u), flood, dtype=torch.float32, device="cuda")
    counts[:, r0:r0 + crop] = torch.from_numpy(band).cuda()
    for req in (fc.FC_BP_AUTO, fc.FC_BP_SLAB, fc.FC_BP_CHUNKED_DENSE):
        vol, used = _recon(fc, wl, counts, req, lab=np.zeros((g.nz, g.ny, g.nx), np.uint8))
        assert used == (fc.FC_BP_SLAB_SYM if req == fc.FC_BP_AUTO else req)
        err = np.max(np.abs(vol - vref))
        precision("mu (FDK)", "paper_mv every voxel, %s" % fc.FC_BP_NAMES[used], err / mu_w, MU_TOL,
                  "of mu_water")
        assert err <= MU_TOL * mu_w, (req, err / mu_w)

"""GPU parity of the dose estimate (Sec. II.H, D0(E) and Dp) through the C ABI
against the FP64 oracle on the same seeded inputs.

Tolerance: D0 and Dp relative error <= 1e-4.  Per ray the binary32 path
lengths differ from the FP64 ones by at most ~1e-4 cm (grazing voxel faces),
i.e. an absorbed fraction off by <= mu_max * 1e-4 ~ 2e-4 on the worst rays;
the sums run over >= 16k rays of which those are a small minority, and the
per-bin Kahan sums add ~1e-7."""
import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


def _oracle_dose(wl, lab, a0, na):
    from oracle import dose as OD
    w, _ = wl.spectrum()
    return OD.dose_estimate(wl.geom, lab, wl.mu(), wl.energies(), wl.muen_water(), w,
                            wl.densities(), a0=a0, na=na)


def _case(fc, wl, lab, a0, na):
    sc = fc.Scanner(wl, labels=lab)
    try:
        d0, dp = sc.dose(a0, na)
    finally:
        sc.close()
    od0, odp = _oracle_dose(wl, lab, a0, na)
    np.testing.assert_allclose(d0, od0, rtol=REL, atol=0)
    assert dp == pytest.approx(odp, rel=REL)
    return d0, dp


def test_dose_small_ragged(fc, orc):
    # detector 70 x 45 (ragged 32 x 8 tiles), three projections from angle 2
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=45, n_angles=7, du=0.16, dv=0.16)
    _case(fc, wl, wl.make_phantom(), 2, 3)


def test_dose_random_labels(fc, orc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=64, n_v=40, n_angles=5, nx=24, ny=20, nz=16,
                  dx=0.5, dy=0.5, dz=0.5, du=0.2, dv=0.2)
    g = wl.geom
    rng = np.random.default_rng(31)
    lab = rng.integers(0, len(wl.labels), size=(g.nz, g.ny, g.nx)).astype(np.uint8)
    _case(fc, wl, lab, 0, 5)


def test_dose_catphan_one_projection(fc, orc):
    wl = W.WORKLOADS["catphan_kv"]
    d0, dp = _case(fc, wl, wl.make_phantom(), 0, 1)
    assert np.all(d0 > 0) and dp > 0


def test_dose_mv_one_projection(fc, orc):
    # 2.5 MV spectrum, 60 bins, on a 256^2 x 10 Catphan module
    wl = W.scaled(W.WORKLOADS["paper_mv"], n_u=256, n_v=192, du=0.1568, dv=0.1568, nx=256,
                  ny=256, dx=0.0625, dy=0.0625, dz=0.0625)
    _case(fc, wl, wl.make_phantom(), 5, 1)


def test_dose_reproducible_and_device_outputs(fc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=96, n_v=64)
    sc = fc.Scanner(wl)
    try:
        a = sc.dose(0, 4)
        b = sc.dose(0, 4)
        np.testing.assert_array_equal(a[0], b[0])
        assert a[1] == b[1]
        d0 = torch.zeros(wl.n_e, dtype=torch.float64, device="cuda")
        dp = torch.zeros(1, dtype=torch.float64, device="cuda")
        fc.fc_dose_estimate(sc.h, 0, 4, wl.energies(), wl.muen_water(), wl.densities(), d0, dp)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d0.cpu().numpy(), a[0])
        assert float(dp.item()) == a[1]
    finally:
        sc.close()


def test_dose_argument_errors(fc):
    wl = W.WORKLOADS["small_kv"]
    sc = fc.Scanner(wl)
    e, m, r = wl.energies(), wl.muen_water(), wl.densities()
    try:
        for a0, na, ee, mm, rr in ((0, 0, e, m, r), (89, 2, e, m, r), (0, 1, -e, m, r),
                                   (0, 1, e, m + 1.0, r), (0, 1, e, m, 0.0 * r)):
            with pytest.raises(fc.FastcatError) as ex:
                fc.fc_dose_estimate(sc.h, a0, na, ee, mm, rr)
            assert ex.value.code == fc.FC_EINVAL
    finally:
        sc.close()


def test_fluence_for_dose(fc):
    # N_gamma = dose / Dp particles over the n_u n_v pixels of the beam
    wl = W.WORKLOADS["small_kv"]
    sc = fc.Scanner(wl)
    try:
        _, dp = sc.dose(0, 1)
        n0 = fc.fc_fluence_for_dose(sc.h, 7e-3, dp)
        assert n0 == pytest.approx(7e-3 / dp / (wl.geom.n_u * wl.geom.n_v), rel=1e-15)
        with pytest.raises(fc.FastcatError):
            fc.fc_fluence_for_dose(sc.h, 1e-3, 0.0)
    finally:
        sc.close()

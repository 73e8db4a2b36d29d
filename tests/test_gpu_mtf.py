"""GPU parity of the slanted-slit detector MTF (Sec. II.C) against the FP64
oracle.  Both sides work in binary64 with the same pixel-to-bin rule; the
GPU's 2-D blur sums in another order and its group weights come from the
binary32 w D table, so agreement is asked to 1e-9 (one kernel) and 1e-6
(energy groups)."""
import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


@pytest.mark.parametrize("name,du", [("small_kv", 0.08), ("catphan_kv", 0.04), ("paper_mv", 0.0336)])
def test_mtf_single_kernel(fc, orc, name, du):
    from oracle import mtf as OM
    wl = W.scaled(W.WORKLOADS[name], du=du, n_u=64, n_v=48, n_angles=4)
    sc = fc.Scanner(wl)
    try:
        f, m = fc.fc_detector_mtf(sc.h)
    finally:
        sc.close()
    fo, mo = OM.mtf(du, [1.0], [wl.psf_sigma_px])
    np.testing.assert_allclose(f, fo, rtol=1e-14)
    np.testing.assert_allclose(m, mo, rtol=0, atol=1e-9)


def test_mtf_energy_groups_and_errors(fc, orc):
    from oracle import mtf as OM
    wl = W.scaled(W.WORKLOADS["catphan_kv"], n_u=64, n_v=48, n_angles=4)
    grp = W.energy_groups(wl, 4)
    w, d = wl.spectrum()
    wd = w * d
    ends = [0] + [int(e) for e in grp["bin_end"]]
    share = [wd[a:b].sum() for a, b in zip(ends[:-1], ends[1:])]
    sc = fc.Scanner(wl)
    try:
        fc.fc_set_energy_groups(sc.h, **grp)
        f, m = fc.fc_detector_mtf(sc.h, 0.3, 2.5, 8)
        with pytest.raises(fc.FastcatError):
            fc.fc_detector_mtf(sc.h, 0.3, 2.5, 0)
        with pytest.raises(fc.FastcatError):
            fc.fc_detector_mtf(sc.h, -0.3, 2.5, 4)
    finally:
        sc.close()
    fo, mo = OM.mtf(wl.geom.du, share, grp["psf_sigma_px"], oversample=8)
    assert len(f) == 16 * 8 + 1
    np.testing.assert_allclose(m, mo, rtol=0, atol=1e-6)

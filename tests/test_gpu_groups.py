"""GPU parity of the energy-group detector model (Sec. II.E scatter fit added
per group, Sec. II.G optical spread per energy) through the C ABI against the
FP64 oracle.

Tolerances: intensity relative error <= 1e-4 per pixel (as the single-kernel
model); counts compared bit-exactly by drawing the oracle's Poisson counts
from the GPU's binary32 rates; reconstruction |d mu| <= 5e-4 mu_water."""
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


def _case(n_groups=4):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=45, n_angles=7, du=0.16, dv=0.16)
    return wl, wl.make_phantom(), W.energy_groups(wl, n_groups)


def _out(fc, sc, kind, a0, na):
    g = sc.g
    out = torch.empty((na, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
    fc.fc_project(sc.h, a0, na, kind, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle_I(wl, lab, grp, a0, na):
    from oracle import groups as OG
    w, d = wl.spectrum()
    bounds = [0] + [int(b) for b in grp["bin_end"]]
    P = OG.group_primaries(wl.geom, lab, w, d, wl.mu(), bounds, a0=a0, na=na)
    return OG.intensity_groups(wl.geom, P, grp["psf_sigma_px"], grp["scatter_amp"],
                               grp["scatter_a_cm"], grp["scatter_b"], wl.n0)


@pytest.mark.parametrize("n_groups", [1, 4, 8])
def test_group_intensity_matches_oracle(fc, orc, n_groups):
    wl, lab, grp = _case(n_groups)
    sc = fc.Scanner(wl, labels=lab, noise=False)
    try:
        fc.fc_set_energy_groups(sc.h, **grp)
        I = _out(fc, sc, fc.FC_OUT_INTENSITY, 2, 4)
        T = _out(fc, sc, fc.FC_OUT_PRIMARY, 2, 4)
    finally:
        sc.close()
    np.testing.assert_allclose(I, _oracle_I(wl, lab, grp, 2, 4), rtol=1e-4)
    w, d = wl.spectrum()
    np.testing.assert_allclose(T, orc.project_T(wl.geom, lab, w, d, wl.mu(), a0=2, na=4), rtol=1e-4)


def test_group_counts_and_reconstruction(fc, orc):
    wl, lab, grp = _case(4)
    g = wl.geom
    sc = fc.Scanner(wl, labels=lab, noise=True)
    try:
        fc.fc_set_energy_groups(sc.h, **grp)
        I = _out(fc, sc, fc.FC_OUT_INTENSITY, 0, g.n_angles)
        K = _out(fc, sc, fc.FC_OUT_COUNTS, 0, g.n_angles)
        np.testing.assert_array_equal(K, orc.poisson(I, wl.seed, 0))
        # reconstruction from the noise-free intensity uses the flood N0
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        fc.fc_reconstruct(sc.h, torch.from_numpy(I).cuda(), vol_mu=vol)
        torch.cuda.synchronize()
        vol = vol.cpu().numpy()
    finally:
        sc.close()
    ref = orc.fdk(g, I.astype(np.float64), wl.n0)
    mu_w = float(wl.mu()[:, 1].mean())
    assert np.max(np.abs(vol - ref)) <= 5e-4 * mu_w


def test_groups_off_restores_single_kernel_model(fc):
    wl, lab, grp = _case(2)
    sc = fc.Scanner(wl, labels=lab, noise=False)
    try:
        I0 = _out(fc, sc, fc.FC_OUT_INTENSITY, 0, 2)
        fc.fc_set_energy_groups(sc.h, **grp)
        Ig = _out(fc, sc, fc.FC_OUT_INTENSITY, 0, 2)
        fc.fc_set_energy_groups(sc.h)
        I1 = _out(fc, sc, fc.FC_OUT_INTENSITY, 0, 2)
    finally:
        sc.close()
    np.testing.assert_array_equal(I0, I1)
    assert not np.allclose(I0, Ig)


def test_group_argument_errors(fc):
    wl, lab, grp = _case(4)
    sc = fc.Scanner(wl, labels=lab, noise=True)
    try:
        bad = [dict(grp, bin_end=[5, 5, 10, wl.n_e]), dict(grp, bin_end=[5, 8, 10, wl.n_e - 1]),
               dict(grp, psf_sigma_px=[0.5, 0.5, 0.5, 4.5]), dict(grp, scatter_a_cm=[1, 1, 0, 1]),
               dict(grp, scatter_b=[1, -1, 1, 1]), dict(grp, scatter_amp=[0.1, 0.1, -0.1, 0.1])]
        for b in bad:
            with pytest.raises(fc.FastcatError) as ex:
                fc.fc_set_energy_groups(sc.h, **b)
            assert ex.value.code == fc.FC_EINVAL
        fc.fc_set_energy_groups(sc.h, **grp)
        fc.fc_set_noise_order(sc.h, fc.FC_NOISE_BEFORE_PSF)
        with pytest.raises(fc.FastcatError) as ex:
            _out(fc, sc, fc.FC_OUT_COUNTS, 0, 1)
        assert ex.value.code == fc.FC_EINVAL
    finally:
        sc.close()

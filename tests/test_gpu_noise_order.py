"""GPU parity of the Sec. II.G noise order (Poisson counts first, optical
spread after) through the C ABI against the FP64 oracle.

Tolerances: rate and noise-free counts relative error <= 1e-4 per pixel (as
the default-order intensity); with noise, the Poisson draws are compared
bit-exactly by drawing the oracle's counts from the GPU's own binary32 rates,
and the blurred counts within 1e-5 relative (binary32 blur of integers)."""
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


def _out(fc, sc, kind, a0, na):
    g = sc.g
    out = torch.empty((na, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
    fc.fc_project(sc.h, a0, na, kind, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _wl():
    # ragged detector (70 x 45), PSF 1.3 px, scatter 6 px
    import dataclasses
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=70, n_v=45, n_angles=6, du=0.16, dv=0.16)
    return dataclasses.replace(wl, psf_sigma_px=1.3, scatter_sigma_px=6.0, spr=0.25)


def test_noise_before_psf_noise_free(fc, orc):
    wl = _wl()
    g = wl.geom
    lab = wl.make_phantom()
    sc = fc.Scanner(wl, labels=lab, noise=False)
    try:
        fc.fc_set_noise_order(sc.h, fc.FC_NOISE_BEFORE_PSF)
        lam = _out(fc, sc, fc.FC_OUT_INTENSITY, 1, 4)
        K = _out(fc, sc, fc.FC_OUT_COUNTS, 1, 4)
    finally:
        sc.close()
    w, d = wl.spectrum()
    T = orc.project_T(g, lab, w, d, wl.mu(), a0=1, na=4)
    olam, oK = orc.counts_noise_before_psf(T, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    np.testing.assert_allclose(lam, olam, rtol=1e-4)
    np.testing.assert_allclose(K, oK, rtol=1e-4)


def test_noise_before_psf_draws(fc, orc):
    wl = _wl()
    lab = wl.make_phantom()
    sc = fc.Scanner(wl, labels=lab, noise=True)
    try:
        fc.fc_set_noise_order(sc.h, fc.FC_NOISE_BEFORE_PSF)
        lam = _out(fc, sc, fc.FC_OUT_INTENSITY, 2, 3)
        K = _out(fc, sc, fc.FC_OUT_COUNTS, 2, 3)
        # back to the default order on the same handle: noise after the blur
        fc.fc_set_noise_order(sc.h, fc.FC_NOISE_AFTER_BLUR)
        I = _out(fc, sc, fc.FC_OUT_INTENSITY, 2, 3)
    finally:
        sc.close()
    counts = orc.poisson(lam, wl.seed, 2).astype(np.float64)
    oK = orc.gauss_blur(counts, wl.psf_sigma_px)
    np.testing.assert_allclose(K, oK, rtol=1e-5)
    assert not np.allclose(I, lam)   # the orders differ in where the PSF acts


def test_noise_order_bad_value(fc):
    sc = fc.Scanner(W.WORKLOADS["small_kv"])
    try:
        with pytest.raises(fc.FastcatError) as ex:
            fc.fc_set_noise_order(sc.h, 2)
        assert ex.value.code == fc.FC_EINVAL
    finally:
        sc.close()

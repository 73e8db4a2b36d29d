"""GPU parity of the Richardson-Lucy deconvolution of projections through the
C ABI against the FP64 oracle (EM update with the clamp-to-edge blur and its
exact adjoint).

Tolerance: relative 2e-4 per pixel after up to 5 iterations: each step is a
binary32 blur, a division and a transposed blur (~1e-6 relative each), and
the multiplicative update carries the previous step's error forward, so the
error grows roughly linearly with the iteration count."""
import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 2e-4


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


def _counts(fc, sc, a0, na):
    g = sc.g
    out = torch.empty((na, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
    fc.fc_project(sc.h, a0, na, fc.FC_OUT_COUNTS, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("sigma,n_iter,shape", [(1.3, 5, (70, 45)), (4.0, 3, (37, 20)),
                                                (0.6, 4, (128, 96))])
def test_rl_matches_oracle(fc, orc, sigma, n_iter, shape):
    from oracle import deconv as OD
    n_u, n_v = shape
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=n_u, n_v=n_v, n_angles=6, du=0.16, dv=0.16)
    sc = fc.Scanner(wl, noise=True)
    try:
        d = _counts(fc, sc, 1, 3)
        u = np.empty_like(d)
        fc.fc_deconvolve_rl(sc.h, 1, 3, sigma, n_iter, u)
    finally:
        sc.close()
    ref = OD.richardson_lucy(d, sigma, n_iter)
    np.testing.assert_allclose(u, ref, rtol=RTOL, atol=1e-3)
    # flux: sum(H^T 1 * u) = sum(d)
    norm = OD.adjoint(np.ones(d.shape[1:]), OD.clamp_blur_matrix(n_v, sigma),
                      OD.clamp_blur_matrix(n_u, sigma))
    assert np.sum(norm * u.astype(np.float64)) == pytest.approx(np.sum(d, dtype=np.float64), rel=1e-5)


def test_rl_zero_iterations_and_reconstruction(fc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=96, n_v=64, n_angles=8, du=0.12, dv=0.12)
    g = wl.geom
    sc = fc.Scanner(wl, noise=True)
    try:
        d = _counts(fc, sc, 0, g.n_angles)
        u = np.empty_like(d)
        fc.fc_deconvolve_rl(sc.h, 0, g.n_angles, 1.0, 0, u)
        np.testing.assert_array_equal(u, d)
        fc.fc_deconvolve_rl(sc.h, 0, g.n_angles, 1.0, 4)
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        fc.fc_reconstruct(sc.h, None, vol_mu=vol)
        torch.cuda.synchronize()
        assert torch.isfinite(vol).all()
        with pytest.raises(fc.FastcatError):
            fc.fc_deconvolve_rl(sc.h, 0, g.n_angles, 4.5, 1)
        with pytest.raises(fc.FastcatError):
            fc.fc_deconvolve_rl(sc.h, 5, g.n_angles, 1.0, 1)
    finally:
        sc.close()


def test_rl_full_size_sampled(fc, orc):
    """The benchmarked size (360 projections of 512 x 384, PSF sigma 0.8 px):
    every image is deconvolved on the GPU; two sampled projections are checked
    against the oracle in full (the images are independent), and the flux
    invariant over all of them."""
    from oracle import deconv as OD
    wl = W.WORKLOADS["catphan_kv"]
    g = wl.geom
    sigma, n_iter = wl.psf_sigma_px, 3
    sc = fc.Scanner(wl, noise=True)
    try:
        d = _counts(fc, sc, 0, g.n_angles)
        u = np.empty_like(d)
        fc.fc_deconvolve_rl(sc.h, 0, g.n_angles, sigma, n_iter, u)
    finally:
        sc.close()
    for k in (0, 217):
        ref = OD.richardson_lucy(d[k:k + 1], sigma, n_iter)
        np.testing.assert_allclose(u[k:k + 1], ref, rtol=RTOL, atol=1e-3)
    norm = OD.adjoint(np.ones(d.shape[1:]), OD.clamp_blur_matrix(g.n_v, sigma),
                      OD.clamp_blur_matrix(g.n_u, sigma))
    flux_u = np.einsum("kvu,vu->k", u.astype(np.float64), norm)
    flux_d = d.astype(np.float64).sum(axis=(1, 2))
    assert np.max(np.abs(flux_u - flux_d) / flux_d) <= 1e-5

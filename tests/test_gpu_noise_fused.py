"""Noise drawn straight after the band blur: when fc_project returns counts
(or nothing) the band kernel leaves the rows that hold the constant flood
intensity unwritten and the Poisson sampler takes that rate there itself.
The counts must equal, bit for bit, those the standalone sampler (fc_poisson)
draws from the full intensity image that FC_OUT_INTENSITY returns."""
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


@pytest.mark.parametrize("n_angles,angle_begin", [(6, 0), (5, 3)])
def test_band_blur_counts_match_standalone_sampler(fc, n_angles, angle_begin):
    # the Catphan kV slab: the band kernel applies (rows far from the band
    # hold the constant), noise seed of the workload
    wl = W.scaled(W.WORKLOADS["catphan_kv"], n_angles=12)
    g = wl.geom
    sc = fc.Scanner(wl, noise=True)
    try:
        shape = (n_angles, g.n_v, g.n_u)
        I = torch.empty(shape, dtype=torch.float32, device="cuda")
        K = torch.empty(shape, dtype=torch.float32, device="cuda")
        fc.fc_project(sc.h, angle_begin, n_angles, fc.FC_OUT_INTENSITY, I)
        fc.fc_project(sc.h, angle_begin, n_angles, fc.FC_OUT_COUNTS, K)
        ref = torch.empty_like(K)
        fc.fc_poisson(I, ref, n_angles, g.n_v, g.n_u, angle_begin, wl.seed)
        torch.cuda.synchronize()
        Ih, Kh, Rh = I.cpu().numpy(), K.cpu().numpy(), ref.cpu().numpy()
        # the image has constant rows far from the band (the case under test)
        assert np.all(Ih[:, 0, :] == Ih[0, 0, 0]) and np.all(Ih[:, -1, :] == Ih[0, 0, 0])
        assert np.array_equal(Kh, Rh)
    finally:
        sc.close()


def test_full_scan_counts_feed_reconstruction(fc):
    """Counts of a whole 12-projection scan kept in the handle (FC_OUT_NONE)
    reconstruct exactly as the same counts passed in from the device."""
    wl = W.scaled(W.WORKLOADS["catphan_kv"], n_angles=12)
    g = wl.geom
    sc = fc.Scanner(wl, noise=True)
    try:
        K = torch.empty((g.n_angles, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_COUNTS, K)
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE)
        vol_a = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        vol_b = torch.empty_like(vol_a)
        fc.fc_reconstruct(sc.h, vol_mu=vol_a)
        fc.fc_reconstruct(sc.h, K, vol_mu=vol_b)
        torch.cuda.synchronize()
        assert torch.equal(vol_a, vol_b)
    finally:
        sc.close()

"""The allocation-free detector blur, fc_detector_blur_static.

Callers whose device memory belongs to another allocator, or is fixed at
start-up, cannot let the library allocate; this entry point runs the detector
blur with its intermediates in a library-held device array.  The test calls
it through the C ABI twice in a row on different inputs and checks each
output against the handle-based path (fc_project, FC_OUT_INTENSITY) with the
same tolerance as the other intensity parity tests.  It lives in its own file
that pytest collects last.
"""
import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_T = 1e-4


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


def test_blur_static_matches_handle_path_twice(fc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=96, n_v=72, n_angles=12, nx=32, ny=32, nz=24,
                  dx=0.4, dy=0.4, dz=0.4, du=0.16, dv=0.16)
    g = wl.geom
    sc = fc.Scanner(wl, noise=False)
    try:
        T = torch.empty((g.n_angles, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
        I_ref = torch.empty_like(T)
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_PRIMARY, T)
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_INTENSITY, I_ref)
        torch.cuda.synchronize()
    finally:
        sc.close()
    halves = [(0, 5), (5, g.n_angles)]   # two calls in a row, different inputs and sizes
    outs = []
    for a0, a1 in halves:
        Tin = T[a0:a1].contiguous()
        out = torch.full_like(Tin, -1.0)
        fc.fc_detector_blur_static(Tin, out, a1 - a0, g.n_v, g.n_u, wl.psf_sigma_px,
                                   wl.scatter_sigma_px, wl.spr, wl.n0)
        outs.append(out)
    torch.cuda.synchronize()
    ref = I_ref.cpu().numpy()
    for (a0, a1), out in zip(halves, outs):
        got = out.cpu().numpy()
        rel = np.abs(got - ref[a0:a1]) / ref[a0:a1]
        assert rel.max() <= REL_T, (a0, rel.max())


def test_blur_static_rejects_oversize(fc):
    n_v, n_u = 512, 512
    n_img = fc.FC_STATIC_SCRATCH_FLOATS // (2 * n_v * n_u) + 1
    T = torch.zeros(n_img * n_v * n_u, dtype=torch.float32, device="cuda")
    with pytest.raises(fc.FastcatError) as ei:
        fc.fc_detector_blur_static(T, T, n_img, n_v, n_u, 0.8, 20.0, 0.2, 1e5)
    assert ei.value.code == fc.FC_EINVAL
    assert "FC_STATIC_SCRATCH_FLOATS" in fc.fc_last_error()


def test_blur_static_rejects_bad_tensors_before_launch(fc):
    """Undersized, non-float32 or mixed-device tensors never reach a kernel
    (the kernels would read and write n_img * n_v * n_u elements)."""
    n_img, n_v, n_u = 2, 16, 24
    n = n_img * n_v * n_u
    good = torch.zeros(n, dtype=torch.float32, device="cuda")
    short = torch.zeros(n - 1, dtype=torch.float32, device="cuda")
    half = torch.zeros(n, dtype=torch.float16, device="cuda")
    for T, I in ((short, good), (good, short), (half, good), (good, half),
                 (good.cpu(), good)):
        with pytest.raises(ValueError):
            fc.fc_detector_blur_static(T, I, n_img, n_v, n_u, 0.8, 20.0, 0.2, 1e5)
    # a valid call still works after the refusals
    out = torch.empty_like(good)
    fc.fc_detector_blur_static(good + 1.0, out, n_img, n_v, n_u, 0.8, 20.0, 0.2, 1e5)
    torch.cuda.synchronize()
    assert torch.allclose(out, torch.full_like(out, 1.2e5), rtol=1e-5)

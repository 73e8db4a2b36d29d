"""Failure handling without a GPU fault (fc_inject_fault): an injected
out-of-memory allocation returns FC_ENOMEM and leaves the handle usable; an
injected give-up of the tensor-core blur's bounded accumulator wait takes the
kernel's abort path (MMAs and copies drained, tensor memory freed, error
word set), the call returns FC_ETIMEOUT, and the next call computes the
right result."""
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
    yield fastcat
    fastcat.fc_inject_fault(fastcat.FC_FAULT_NONE)


def _wl():
    # the band of rows that can meet the voxels covers the whole detector, so
    # the detector blur runs on the tensor-core passes
    return W.scaled(W.WORKLOADS["small_kv"], n_u=72, n_v=48, n_angles=6, nx=24, ny=24, nz=24,
                    dx=0.4, dy=0.4, dz=0.4, du=0.16, dv=0.16)


def _intensity(fc, sc, host=False):
    g = sc.g
    if host:
        out = np.empty((g.n_angles, g.n_v, g.n_u), np.float32)
    else:
        out = torch.empty((g.n_angles, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
    fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_INTENSITY, out)
    if not host:
        torch.cuda.synchronize()
        out = out.cpu().numpy()
    return out


@pytest.fixture(scope="module")
def reference(fc):
    wl = _wl()
    sc = fc.Scanner(wl, noise=False)
    try:
        return _intensity(fc, sc)
    finally:
        sc.close()


@pytest.mark.parametrize("n_ok", [0, 3])
def test_injected_out_of_memory_then_recovery(fc, reference, n_ok):
    """The (n_ok + 1)-th projection-buffer allocation of a fresh handle
    fails: FC_ENOMEM, then the same handle completes the call."""
    sc = fc.Scanner(_wl(), noise=False)
    try:
        fc.fc_inject_fault(fc.FC_FAULT_ALLOC, n_ok)
        try:
            with pytest.raises(fc.FastcatError) as ei:
                _intensity(fc, sc)
        finally:
            fc.fc_inject_fault(fc.FC_FAULT_NONE)
        assert ei.value.code == fc.FC_ENOMEM
        got = _intensity(fc, sc)
        assert np.array_equal(got.view(np.uint32), reference.view(np.uint32))
    finally:
        sc.close()


def test_injected_blur_wait_timeout_then_recovery(fc, reference):
    sc = fc.Scanner(_wl(), noise=False)
    try:
        _intensity(fc, sc)                     # buffers allocated, a clean run first
        fc.fc_inject_fault(fc.FC_FAULT_BLUR_TIMEOUT)
        try:
            with pytest.raises(fc.FastcatError) as ei:
                _intensity(fc, sc, host=True)
        finally:
            fc.fc_inject_fault(fc.FC_FAULT_NONE)
        assert ei.value.code == fc.FC_ETIMEOUT
        assert "timed out" in fc.fc_last_error()
        got = _intensity(fc, sc, host=True)     # error word cleared, right result
        assert np.array_equal(got.view(np.uint32), reference.view(np.uint32))
        vol = torch.empty((sc.g.nz, sc.g.ny, sc.g.nx), dtype=torch.float64, device="cuda")
        fc.fc_reconstruct(sc.h, None, vol_mu=vol)   # the context is still usable
        torch.cuda.synchronize()
        assert bool(torch.isfinite(vol).all())
    finally:
        sc.close()

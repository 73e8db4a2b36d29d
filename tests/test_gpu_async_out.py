"""Asynchronous host outputs of fc_reconstruct (FC_HOST_ASYNC + fc_wait_outputs):
the copies run on the handle's own stream while the caller's next calls
proceed, and the next reconstruction waits for them before it rewrites the
volume.  Checked against the synchronous device outputs bit for bit."""
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


def _pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype).pin_memory().numpy()


def test_async_volumes_match_sync(fc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_angles=24)
    g = wl.geom
    sc = fc.Scanner(wl, noise=False)
    try:
        h = sc.h
        stream = torch.cuda.Stream()
        # two different count sets: the reference volumes, synchronous
        cA = torch.empty((g.n_angles, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_INTENSITY, cA)
        cB = cA * 0.97 + 3.0
        torch.cuda.synchronize()
        refs = []
        for c in (cA, cB):
            v = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
            hu = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device="cuda")
            fc.fc_reconstruct(h, c, vol_mu=v, vol_hu=hu)
            torch.cuda.synchronize()
            refs.append((v.cpu().numpy(), hu.cpu().numpy()))
        assert not np.array_equal(refs[0][0], refs[1][0])
        # queued back to back on one stream, a projection in between: the
        # second backprojection must wait for the first copy-out
        outs = [(_pinned((g.nz, g.ny, g.nx), torch.float64), _pinned((g.nz, g.ny, g.nx), torch.float32))
                for _ in range(2)]
        for o in outs:
            o[0].fill(np.nan)
            o[1].fill(np.nan)
        with torch.cuda.stream(stream):
            fc.fc_reconstruct(h, cA, vol_mu=outs[0][0], vol_hu=outs[0][1], stream=stream, async_host=True)
            fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_NONE, None, stream)
            fc.fc_reconstruct(h, cB, vol_mu=outs[1][0], vol_hu=outs[1][1], stream=stream, async_host=True)
        fc.fc_wait_outputs(h)
        for (v, hu), (rv, rhu) in zip(outs, refs):
            assert np.array_equal(v, rv)
            assert np.array_equal(hu, rhu)
        # nothing queued: returns at once
        fc.fc_wait_outputs(h)
        # a device output after an asynchronous one orders itself behind it
        outs[0][0].fill(np.nan)
        fc.fc_reconstruct(h, cA, vol_mu=outs[0][0], async_host=True)
        v = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        fc.fc_reconstruct(h, cB, vol_mu=v)
        fc.fc_wait_outputs(h)
        torch.cuda.synchronize()
        assert np.array_equal(outs[0][0], refs[0][0])
        assert np.array_equal(v.cpu().numpy(), refs[1][0])
    finally:
        sc.close()


def test_async_refuses_pageable_memory(fc):
    wl = W.scaled(W.WORKLOADS["small_kv"], n_angles=8)
    g = wl.geom
    sc = fc.Scanner(wl, noise=False)
    try:
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE)
        pageable = np.empty((g.nz, g.ny, g.nx), np.float64)
        with pytest.raises(fc.FastcatError) as ei:
            fc.fc_reconstruct(sc.h, vol_mu=pageable, async_host=True)
        assert ei.value.code == fc.FC_EINVAL
        # the handle stays usable
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        fc.fc_reconstruct(sc.h, vol_mu=vol)
        torch.cuda.synchronize()
        assert torch.isfinite(vol).all()
    finally:
        sc.close()

"""GPU adjoint of the CNR objective against the FP64 oracle gradient
(PyTorch float64 reverse mode, itself pinned by finite differences):
relative error <= 1e-3."""
import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-3


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_04736_gb300 import build, fastcat
    build.build()
    fastcat.load()
    return fastcat


def _small():
    return W.scaled(W.WORKLOADS["adjoint_kv"], n_u=96, n_v=24, du=0.24, dv=0.24, n_angles=48,
                    nx=64, ny=64, nz=8, dx=0.25, dy=0.25, dz=0.25)


def _gpu(fc, wl, inp, grads=True):
    sc = fc.Scanner(wl, labels=inp["labels"], noise=False)
    try:
        rho = torch.from_numpy(inp["rho"]).cuda()
        z = torch.from_numpy(inp["z"]).cuda()
        J, gl, gd, gr = fc.fc_cnr_grad(sc.h, inp["logits"], inp["D"], inp["rho0"], rho, z,
                                       inp["rois"], grads=grads)
        torch.cuda.synchronize()
        return J, gl, gd, (gr.cpu().numpy().ravel() if gr is not None else None)
    finally:
        sc.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_cnr_gradient_matches_oracle(fc, orc, precision):
    from oracle import adjoint
    wl = _small()
    inp = W.adjoint_inputs(wl)
    obj = adjoint.Objective(wl, inp["labels"], inp["rho0"], inp["z"], inp["rois"])
    Jr, glr, gdr, grr = obj.value_and_grad(inp["logits"], inp["D"], inp["rho"])
    J, gl, gd, gr = _gpu(fc, wl, inp)
    print("J gpu %.8f oracle %.8f; rel err logits %.2e D %.2e rho %.2e"
          % (J, Jr, _rel(gl, glr), _rel(gd, gdr), _rel(gr, grr)))
    case = "64^2x8 voxels, 48 x 96 x 24"
    precision("J (CNR objective)", case, abs(J - Jr) / abs(Jr), REL)
    precision("dJ/dlogits", case, _rel(gl, glr), REL, "relative (norm)")
    precision("dJ/dD", case, _rel(gd, gdr), REL, "relative (norm)")
    precision("dJ/drho", case, _rel(gr, grr), REL, "relative (norm)")
    assert abs(J - Jr) <= REL * abs(Jr)
    assert _rel(gl, glr) <= REL
    assert _rel(gd, gdr) <= REL
    assert _rel(gr, grr) <= REL


def test_cnr_autograd_function(fc):
    wl = _small()
    inp = W.adjoint_inputs(wl)
    sc = fc.Scanner(wl, labels=inp["labels"], noise=False)
    try:
        rho = torch.from_numpy(inp["rho"]).cuda().requires_grad_(True)
        lg = torch.tensor(inp["logits"], requires_grad=True)
        dd = torch.tensor(inp["D"], requires_grad=True)
        z = torch.from_numpy(inp["z"]).cuda()
        f = fc.cnr_objective(sc.h, inp["rho0"], z, inp["rois"])
        J = f(lg, dd, rho)
        (2.0 * J).backward()
        J2, gl, gd, gr = fc.fc_cnr_grad(sc.h, inp["logits"], inp["D"], inp["rho0"], rho.detach(),
                                        z, inp["rois"])
        torch.cuda.synchronize()
        assert float(J) == pytest.approx(J2)
        # the density and spectrum gradients are accumulated with atomics, so
        # two evaluations agree to rounding, not bit for bit
        assert _rel(lg.grad.numpy(), 2.0 * gl) <= 1e-5
        assert _rel(dd.grad.numpy(), 2.0 * gd) <= 1e-5
        assert _rel(rho.grad.cpu().numpy(), 2.0 * gr.cpu().numpy()) <= 1e-5
    finally:
        sc.close()


def test_cnr_gradient_full_size_directional(fc, precision):
    """At the benchmarked size (128^2 x 32 voxels, 180 projections of 512 x
    384, 30 bins) the FP64 oracle is too slow, so a property that holds at
    any size is checked instead: central differences of J along the density
    gradient and along the logit gradient match the directional derivatives
    the adjoint gives (the density step is applied in binary32, so the
    expectation uses the densities actually applied)."""
    wl = W.WORKLOADS["adjoint_kv"]
    inp = W.adjoint_inputs(wl)
    sc = fc.Scanner(wl, labels=inp["labels"], noise=False)
    try:
        rho = torch.from_numpy(inp["rho"]).cuda()
        z = torch.from_numpy(inp["z"]).cuda()

        def J_of(logits, r):
            return fc.fc_cnr_grad(sc.h, logits, inp["D"], inp["rho0"], r, z, inp["rois"], grads=False)[0]

        J, gl, _, gr = fc.fc_cnr_grad(sc.h, inp["logits"], inp["D"], inp["rho0"], rho, z, inp["rois"])
        g = gr.double()
        step = 0.01 * g / torch.linalg.norm(g)
        rp, rm = (rho.double() + step).float(), (rho.double() - step).float()
        expect = float(torch.sum(g * (rp.double() - rm.double()))) / 2.0
        got = (J_of(inp["logits"], rp) - J_of(inp["logits"], rm)) / 2.0
        precision("dJ/drho . step", "adjoint_kv 128^2x32, 180x512x384 (central diff.)",
                  abs(got - expect) / abs(expect), 1e-3)
        assert abs(got - expect) <= 1e-3 * abs(expect), (got, expect)

        gl = np.asarray(gl, dtype=np.float64)
        dl = 0.01 * gl / np.linalg.norm(gl)
        expect = float(gl @ dl)
        got = (J_of(inp["logits"] + dl, rho) - J_of(inp["logits"] - dl, rho)) / 2.0
        precision("dJ/dlogits . step", "adjoint_kv (central diff.)", abs(got - expect) / abs(expect), 1e-3)
        assert abs(got - expect) <= 1e-3 * abs(expect), (got, expect)
    finally:
        sc.close()

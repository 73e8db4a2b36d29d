"""Pins of the FP64 CNR-objective oracle (CPU): its matrices against the
pinned oracle routines, its forward against the oracle pipeline, and its
reverse-mode gradient against central finite differences (h = 1e-3)."""
import numpy as np
import pytest

from paper_2011_04736_gb300 import workloads as W

torch = pytest.importorskip("torch")


def small_adjoint_case():
    return W.scaled(W.WORKLOADS["adjoint_kv"], n_u=96, n_v=24, du=0.24, dv=0.24, n_angles=48,
                    nx=64, ny=64, nz=8, dx=0.25, dy=0.25, dz=0.25)


@pytest.fixture(scope="module")
def case(orc):
    from oracle import adjoint
    wl = small_adjoint_case()
    inp = W.adjoint_inputs(wl)
    obj = adjoint.Objective(wl, inp["labels"], inp["rho0"], inp["z"], inp["rois"])
    return wl, inp, obj


def test_backprojection_matrix_matches_oracle(orc, case):
    wl, inp, obj = case
    g = wl.geom
    f = np.random.default_rng(0).normal(size=(g.n_angles, g.n_v, g.n_u))
    ref = orc.backproject(g, f).ravel()
    got = torch.sparse.mm(obj.B, torch.from_numpy(f.reshape(-1, 1))).numpy().ravel()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_forward_matches_oracle_pipeline(orc, case):
    """Nominal densities and no noise: the objective's volume is the oracle's
    projection -> intensity -> FDK."""
    from oracle import adjoint
    wl, inp, obj = case
    g = wl.geom
    w = torch.softmax(torch.from_numpy(inp["logits"]), 0).numpy()
    T = orc.project_T(g, inp["labels"], w, inp["D"], wl.mu())
    I = orc.intensity(T, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    vol = orc.fdk(g, I, orc.i_flood(wl.n0, wl.spr)).ravel()
    c = torch.softmax(torch.from_numpy(inp["logits"]), 0) * torch.from_numpy(inp["D"])
    rho = inp["rho0"][inp["labels"].ravel()]            # nominal densities in float64
    X = (torch.from_numpy(rho) * obj.irho0)[:, None] * obj.onehot
    A = torch.sparse.mm(obj.M, X)
    T2 = (torch.exp(-A @ obj.mu.T) @ c / c.sum()).reshape(T.shape)
    assert np.max(np.abs(T2.numpy() - T)) < 1e-12
    I2 = wl.n0 * (adjoint._blur(T2, wl.psf_sigma_px) + wl.spr * adjoint._blur(T2, wl.scatter_sigma_px))
    assert np.max(np.abs(I2.numpy() - I)) < 1e-6
    q = torch.log(wl.n0 * (1 + wl.spr) / torch.clamp(I2, min=1.0)) * obj.cosw
    f = adjoint._ramp(q, g.du * g.sad / g.sdd)
    mu = torch.sparse.mm(obj.B, f.reshape(-1, 1)).numpy().ravel()
    assert np.max(np.abs(mu - vol)) < 1e-10


def test_gradient_matches_finite_differences(case):
    wl, inp, obj = case
    J, gl, gd, gr = obj.value_and_grad(inp["logits"], inp["D"], inp["rho"])
    assert np.isfinite(J) and J > 0
    rng = np.random.default_rng(1)
    h = 1e-3
    checks = [("l", int(e)) for e in rng.choice(wl.n_e, 3, replace=False)]
    checks += [("d", int(e)) for e in rng.choice(wl.n_e, 2, replace=False)]
    hot = np.argsort(-np.abs(gr))[:3]
    checks += [("r", int(v)) for v in hot]
    base = {"l": inp["logits"].astype(np.float64), "d": inp["D"].astype(np.float64),
            "r": inp["rho"].astype(np.float64).ravel()}
    grads = {"l": gl, "d": gd, "r": gr}
    for kind, i in checks:
        vals = []
        for sgn in (1, -1):
            args = {k: v.copy() for k, v in base.items()}
            step = h * max(1.0, abs(args[kind][i]))
            args[kind][i] += sgn * step
            with torch.no_grad():
                vals.append(float(obj(torch.from_numpy(args["l"]), torch.from_numpy(args["d"]),
                                      torch.from_numpy(args["r"]))))
        fd = (vals[0] - vals[1]) / (2 * step)
        g = grads[kind][i]
        assert abs(fd - g) <= 1e-4 * max(abs(g), 1e-3 * np.max(np.abs(grads[kind]))), (kind, i, fd, g)

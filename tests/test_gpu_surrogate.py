"""GPU tests of the learned energy-integral surrogate (tensor-core MLP) and of
the exact energy sum from path lengths, against the FP64 oracle."""
import math

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


def _head_small():
    return W.scaled(W.WORKLOADS["head_surrogate"], n_u=64, n_v=64, n_angles=12, nx=64, ny=64,
                    nz=64, dx=0.25, dy=0.25, dz=0.25, du=0.2, dv=0.2)


def _random_state(seed, n_mat):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    st = np.zeros(34305 + 52 + 2 * 34305 + 1, np.float32)
    P = st[:mlp.N_PACKED]
    for name, fan in (("W1", 8), ("W2", 128), ("W3", 128), ("w4", 128)):
        a, b = mlp.OFF[name]
        P[a:b] = rng.uniform(-1, 1, b - a) * math.sqrt(3.0 / fan)
    for name in ("b1", "b2", "b3", "b4"):
        a, b = mlp.OFF[name]
        P[a:b] = rng.normal(0, 0.1, b - a)
    a, b = mlp.OFF["scale"]
    P[a:b] = 0.1
    a, b = mlp.OFF["ga"]
    P[a:b] = rng.dirichlet(np.ones(4))
    a, b = mlp.OFF["gmu"]
    P[a:b] = rng.uniform(0.1, 0.4, 32)
    a, b = mlp.OFF["box"]
    P[a:b] = 30.0
    return st


def _oracle_rays(orc, wl, lab, n, seed):
    g = wl.geom
    rng = np.random.default_rng(seed)
    rays = np.stack([rng.integers(0, g.n_angles, n), rng.integers(0, g.n_v, n),
                     rng.integers(0, g.n_u, n)], 1)
    w, d = wl.spectrum()
    L, T = orc.rays(g, lab, w, d, wl.mu(), rays)
    return L, T


def test_energy_sum_lengths_matches_oracle(fc, orc):
    wl = _head_small()
    lab = wl.make_phantom()
    L, T = _oracle_rays(orc, wl, lab, 4096, 3)
    sc = fc.Scanner(wl, labels=lab)
    try:
        dL = torch.from_numpy(L.astype(np.float32)).cuda()
        out = torch.empty(len(T), device="cuda")
        fc.fc_energy_sum_lengths(sc.h, dL, out)
        torch.cuda.synchronize()
    finally:
        sc.close()
    got = np.exp(out.cpu().numpy().astype(np.float64))
    assert np.max(np.abs(got - T) / T) <= 1e-4


def _sigma_error(fc, zmax):
    """Largest |sigma_gpu(z) - sigma(z)| over a dense grid of [-zmax, zmax]
    (sigma as the surrogate kernels evaluate it, measured through the
    library against the exact logistic function in float64)."""
    z = np.linspace(-zmax, zmax, 1 << 22).astype(np.float32)
    dz = torch.from_numpy(z).cuda()
    ds = torch.empty_like(dz)
    fc.fc_surrogate_sigma(dz, ds)
    torch.cuda.synchronize()
    exact = 1.0 / (1.0 + np.exp(-z.astype(np.float64)))
    return float(np.max(np.abs(ds.cpu().numpy().astype(np.float64) - exact)))


# First-order error bound of the tensor-core evaluation against the float64
# oracle with the same bf16 weights (both multiply bf16(W), products exact in
# binary32).  Each local error of the GPU path, times the exact derivative of
# the output with respect to the quantity it perturbs (back-propagated by the
# oracle's own intermediates), summed in absolute value:
#   x = L scale in binary32, carried as bf16 hi + lo:  (2^-24 + 2^-17) |x|;
#   accumulation of K products in binary32 (round or chop): K 2^-23 sum|w h|,
#     and the bias added in the epilogue: 2^-24 |z|;
#   SiLU: sigma off by at most eps_sigma (measured), the product rounded:
#     |z| eps_sigma + 2^-24 |h|; activations of layers 1-2 carried as bf16
#     hi + lo: 2^-17 |h|;
#   output: 128 sequential fma of w4 h3 onto b4: 128 2^-24 (|b4| + sum|w4 h3|);
#   four-group baseline ln sum_k a_k exp(-mu_k.L) with __expf / __logf: the
#     documented maximum errors (exp: 2 + floor(1.173 |arg|) ulp; log:
#     2^-21.41 absolute on [0.5, 2], else 3 ulp), the exponent's fma chain
#     and the 4-term sum.
# A safety factor of 1.25 covers second-order terms.
def _eval_bound(mlp, P, L, cache, eps_sigma):
    u, uc, split = 2.0 ** -24, 2.0 ** -23, 2.0 ** -17
    p = mlp.unpack(P)
    W1, W2, W3 = (mlp.bf16(p[k]) for k in ("W1", "W2", "W3"))
    w4 = p["w4"]
    x, z1, h1, z2, h2, z3, h3 = (cache[k] for k in ("x", "z1", "h1", "z2", "h2", "z3", "h3"))

    def dsilu(z):
        s = 1.0 / (1.0 + np.exp(-z))
        return s + z * s * (1.0 - s)

    g_h3 = np.broadcast_to(w4, h3.shape)
    g_z3 = g_h3 * dsilu(z3)
    g_h2 = g_z3 @ W3
    g_z2 = g_h2 * dsilu(z2)
    g_h1 = g_z2 @ W2
    g_z1 = g_h1 * dsilu(z1)
    g_x = g_z1 @ W1
    ax = np.abs(x)
    b = (np.abs(g_x) * (u + split) * ax).sum(1)
    b += (np.abs(g_z1) * (16 * uc * (ax @ np.abs(W1).T) + u * np.abs(z1))).sum(1)
    b += (np.abs(g_h1) * (np.abs(z1) * eps_sigma + (u + split) * np.abs(h1))).sum(1)
    b += (np.abs(g_z2) * (256 * uc * (1 + 2.0 ** -7) * (np.abs(h1) @ np.abs(W2).T) + u * np.abs(z2))).sum(1)
    b += (np.abs(g_h2) * (np.abs(z2) * eps_sigma + (u + split) * np.abs(h2))).sum(1)
    b += (np.abs(g_z3) * (256 * uc * (1 + 2.0 ** -7) * (np.abs(h2) @ np.abs(W3).T) + u * np.abs(z3))).sum(1)
    b += (np.abs(g_h3) * (np.abs(z3) * eps_sigma + u * np.abs(h3))).sum(1)
    b += 128 * u * (abs(p["b4"][0]) + np.abs(h3) @ np.abs(w4))
    # baseline: relative error of the group sum, then the logarithm
    Lp = np.zeros((len(L), mlp.NIN))
    Lp[:, :L.shape[1]] = L
    gmu = p["gmu"].reshape(4, mlp.NIN)
    arg = Lp @ gmu.T
    rel_e = (2.0 + np.floor(1.173 * np.abs(arg))) * uc + 8 * u * (Lp @ np.abs(gmu).T)
    terms = np.exp(-arg) * p["ga"]
    s_ = terms.sum(1)
    rel_s = (terms * rel_e).sum(1) / s_ + 4 * u
    ln_s = np.log(s_)
    log_err = np.where((s_ >= 0.5) & (s_ <= 2.0), 2.0 ** -21.41, 3 * uc * np.abs(ln_s))
    b += rel_s + log_err
    y = ln_s + h3 @ w4 + p["b4"][0]
    b += u * np.abs(y)
    return 1.25 * b


def test_surrogate_eval_matches_oracle(fc, orc, precision):
    """Tensor-core inference against the float64 oracle within the derived
    per-ray bound, and a planted wrong bias (one unit of the last hidden
    layer, in the oracle) is caught by the same comparison."""
    from oracle import mlp
    wl = _head_small()
    lab = wl.make_phantom()
    L, _ = _oracle_rays(orc, wl, lab, 2000, 4)
    st = _random_state(11, L.shape[1])
    sc = fc.Scanner(wl, labels=lab)
    try:
        fc.fc_surrogate_set(sc.h, st)
        dL = torch.from_numpy(L.astype(np.float32)).cuda()
        out = torch.empty(len(L), device="cuda")
        nfb = fc.fc_surrogate_eval(sc.h, dL, out)
        torch.cuda.synchronize()
    finally:
        sc.close()
    assert nfb == 0
    P = st[:mlp.N_PACKED].astype(np.float64)
    L32 = L.astype(np.float32)
    ref, cache = mlp.forward(P, L32)
    zmax = 1.1 * max(float(np.abs(cache[k]).max()) for k in ("z1", "z2", "z3")) + 0.01
    eps_sigma = _sigma_error(fc, zmax)
    got = out.cpu().numpy()
    bound = _eval_bound(mlp, P, L32.astype(np.float64), cache, eps_sigma)
    err = np.abs(got - ref)
    precision("surrogate ln T vs oracle MLP", "%d rays, random weights" % len(L),
              np.max(err / bound), 1.0, "of the derived per-ray bound")
    precision("surrogate ln T vs oracle MLP", "same (absolute; sigma off by %.1e)" % eps_sigma,
              err.max(), float(bound.max()), "abs")
    assert np.all(err <= bound), (err.max(), np.max(err / bound))
    # a wrong bias of 1e-2 in the unit of largest |w4| moves the oracle
    # beyond the bound on most rays
    p = mlp.unpack(P)
    j = int(np.argmax(np.abs(p["w4"])))
    P2 = P.copy()
    P2[mlp.OFF["b3"][0] + j] += 1e-2
    ref2, _ = mlp.forward(P2, L32)
    assert np.mean(np.abs(got - ref2) > bound) > 0.5


def test_surrogate_gradient_matches_oracle(fc, orc, precision):
    from oracle import mlp
    wl = _head_small()
    lab = wl.make_phantom()
    L, T = _oracle_rays(orc, wl, lab, 1024, 5)
    y = np.log(T)
    st = _random_state(12, L.shape[1])
    sc = fc.Scanner(wl, labels=lab)
    try:
        fc.fc_surrogate_set(sc.h, st)
        dL = torch.from_numpy(L.astype(np.float32)).cuda()
        dy = torch.from_numpy(y.astype(np.float32)).cuda()
        g, loss = fc.fc_surrogate_grad(sc.h, dL, dy)
    finally:
        sc.close()
    P = st[:mlp.N_PACKED].astype(np.float64)
    L32, y32 = L.astype(np.float32), y.astype(np.float32)
    lref, gref = mlp.loss_and_grad(P, L32, y32)
    precision("surrogate loss vs oracle", "1024 rays, random weights", abs(loss - lref) / lref, 2e-2)
    assert loss == pytest.approx(lref, rel=2e-2)
    # Every gradient block is a sum over the samples of products a_b c_b
    # (back-propagated error times activation, or the error alone for a
    # bias), whose factors the GPU stores as single bf16 values for the
    # weight-gradient GEMMs: 2^-9 relative each, so 2 2^-9 |a_b c_b| per
    # product, and || |a|^T |c| || / ||a^T c|| of it norm-wise.  The errors
    # of the deeper errors (their own bf16 roundings, back-propagated) enter
    # as independent round-to-nearest errors: at most 6 / sqrt(3) 2 2^-9
    # sqrt(sum (a_b c_b)^2) norm-wise (six standard deviations).  The
    # sigmoid's error (tanh.approx, measured below 1e-6 in the inference
    # test) is negligible next to 2^-9.
    yh, c = mlp.forward(P, L32)
    n = len(y32)
    gres = 2.0 * (yh - y32.astype(np.float64)) / n
    p = mlp.unpack(P)

    def dsilu(z):
        s_ = 1.0 / (1.0 + np.exp(-z))
        return s_ + z * s_ * (1.0 - s_)

    dz3 = np.outer(gres, p["w4"]) * dsilu(c["z3"])
    dz2 = (dz3 @ c["W3"]) * dsilu(c["z2"])
    dz1 = (dz2 @ c["W2"]) * dsilu(c["z1"])
    ones = np.ones((n, 1))
    factors = {"W1": (dz1, c["x"]), "b1": (dz1, ones), "W2": (dz2, c["h1"]), "b2": (dz2, ones),
               "W3": (dz3, c["h2"]), "b3": (dz3, ones), "w4": (gres[:, None], c["h3"]),
               "b4": (gres[:, None], ones)}
    u9 = 2.0 ** -9
    worst, tols = 0.0, {}
    for name, (fa, fb) in factors.items():
        a, b = mlp.OFF[name]
        ga, gr = g[a:b].astype(np.float64), gref[a:b]
        gn = np.linalg.norm(gr)
        tol = (2 * u9 * np.linalg.norm(np.abs(fa).T @ np.abs(fb)) +
               6.0 / math.sqrt(3.0) * 2 * u9 * math.sqrt(((fa ** 2).T @ (fb ** 2)).sum())) / gn
        tols[name] = tol
        rel = np.linalg.norm(ga - gr) / max(gn, 1e-30)
        cos = ga @ gr / max(np.linalg.norm(ga) * gn, 1e-30)
        worst = max(worst, rel / tol)
        assert rel <= tol and cos >= 1.0 - tol, (name, rel, tol, cos)
    precision("surrogate gradient vs oracle", "1024 rays, worst parameter block", worst, 1.0,
              "of the derived per-block bound")
    # a wrong bias of 2e-2 in the unit of largest |w4| (planted in the
    # oracle) moves the w4 block beyond its bound
    j = int(np.argmax(np.abs(p["w4"])))
    P2 = P.copy()
    P2[mlp.OFF["b3"][0] + j] += 2e-2
    _, g2 = mlp.loss_and_grad(P2, L32, y32)
    a, b = mlp.OFF["w4"]
    assert np.linalg.norm(g[a:b] - g2[a:b]) / np.linalg.norm(g2[a:b]) > tols["w4"]


@pytest.fixture(scope="module")
def trained(fc):
    """Surrogate trained on every ray of a small head-like scan (GPU data)."""
    wl = _head_small()
    lab = wl.make_phantom()
    g = wl.geom
    sc = fc.Scanner(wl, labels=lab)
    L = torch.empty((g.n_rays, len(wl.labels)), device="cuda")
    fc.fc_project_lengths(sc.h, 0, g.n_angles, L)
    y = torch.empty(g.n_rays, device="cuda")
    fc.fc_energy_sum_lengths(sc.h, L, y)
    fc.fc_surrogate_init(sc.h, 3)
    hist = fc.fc_surrogate_train(sc.h, L, y, steps=3000, batch=4096, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    yield wl, sc, L, y, hist
    sc.close()


def test_surrogate_training_gains_over_linear_model(fc, trained):
    wl, sc, L, y, hist = trained
    assert hist[-50:].mean() < 1e-2 * hist[:10].mean()
    out = torch.empty_like(y)
    fc.fc_surrogate_eval(sc.h, L, out)
    torch.cuda.synchronize()
    from oracle import mlp
    st = fc.fc_surrogate_get(sc.h)
    P0 = st[:mlp.N_PACKED].astype(np.float64).copy()
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        a, b = mlp.OFF[name]
        P0[a:b] = 0.0              # the method without the network: baseline only
    Lh, yh, oh = L.cpu().numpy(), y.cpu().numpy(), out.cpu().numpy()
    base, _ = mlp.forward(P0, Lh)
    w, d = wl.spectrum()
    mubar = (w * d) @ wl.mu() / np.sum(w * d)
    err_mlp = np.abs(oh - yh)
    err_base = np.abs(base - yh)
    err_lin = np.abs(-(Lh @ mubar) - yh)
    print("surrogate |d lnT|: max %.3e p99 %.3e; 4-group baseline max %.3e p99 %.3e; "
          "first-order max %.3e" % (err_mlp.max(), np.quantile(err_mlp, 0.99), err_base.max(),
                                    np.quantile(err_base, 0.99), err_lin.max()))
    assert err_mlp.max() < 0.1 * err_base.max()
    assert np.quantile(err_mlp, 0.99) < 2e-3


def test_surrogate_fallback_outside_box(fc, trained):
    wl, sc, L, y, _ = trained
    far = L[:256].clone()
    far[:, 1] += 1000.0            # far outside the training box
    exact = torch.empty(256, device="cuda")
    fc.fc_energy_sum_lengths(sc.h, far, exact)
    out = torch.empty(256, device="cuda")
    nfb = fc.fc_surrogate_eval(sc.h, far, out)
    torch.cuda.synchronize()
    assert nfb == 256
    assert torch.equal(out, exact)


def test_surrogate_eval_ragged_batches(fc, trained):
    """Every ray's result is independent of the batch it is evaluated in:
    batches of 1, 127, 129 and 383 rays (one tile, a tile and a ray, three
    tiles shared unevenly by the kernel's two groups) reproduce, bit for bit,
    the same rays evaluated inside the whole scan."""
    wl, sc, L, y, _ = trained
    full = torch.empty_like(y)
    fc.fc_surrogate_eval(sc.h, L, full)
    for n in (1, 127, 129, 383):
        start = 1000 + 7 * n
        part = torch.empty(n, device="cuda")
        fc.fc_surrogate_eval(sc.h, L[start:start + n].contiguous(), part)
        torch.cuda.synchronize()
        assert torch.equal(part, full[start:start + n]), n


def test_surrogate_checkpoint_roundtrip(fc, trained):
    wl, sc, L, y, _ = trained
    st = fc.fc_surrogate_get(sc.h)
    a = torch.empty_like(y)
    fc.fc_surrogate_eval(sc.h, L, a)
    sc2 = fc.Scanner(wl, labels=wl.make_phantom())
    try:
        fc.fc_surrogate_set(sc2.h, st)
        b = torch.empty_like(y)
        fc.fc_surrogate_eval(sc2.h, L, b)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert np.array_equal(fc.fc_surrogate_get(sc2.h), st)
    finally:
        sc2.close()


def test_surrogate_project_matches_exact_projection(fc, trained):
    """Projection with the surrogate in place of the energy loop against the
    exact projector on the same scan (the trained network's tolerance)."""
    wl, sc, L, y, _ = trained
    g = wl.geom
    Ts = torch.empty((g.n_angles, g.n_v, g.n_u), device="cuda")
    fc.fc_surrogate_project(sc.h, 0, g.n_angles, Ts)
    Te = torch.empty_like(Ts)
    fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_PRIMARY, Te)
    host = np.empty((2, g.n_v, g.n_u), np.float32)
    fc.fc_surrogate_project(sc.h, 3, 2, host)
    torch.cuda.synchronize()
    d = (torch.log(Ts) - torch.log(Te)).abs()
    assert float(d.max()) < 1e-2 and float(torch.quantile(d.ravel()[:1 << 20], 0.99)) < 2e-3
    assert np.array_equal(host, Ts[3:5].cpu().numpy())


def test_surrogate_guard_judges_every_ray(fc, trained, precision):
    """The per-ray guard, set from the data with exact ln T: afterwards every
    ray of that data is within tol (rays the network misses by more are
    evaluated exactly; the guard works on the baseline attenuation, so it
    may send every ray to the exact sum), the fallback count is reported; a
    tol the network never misses leaves the guard off, and tol <= 0 removes
    it again."""
    wl, sc, L, y, _ = trained
    out = torch.empty_like(y)
    try:
        nfb0 = fc.fc_surrogate_eval(sc.h, L, out)
        torch.cuda.synchronize()
        raw = (out - y).abs()
        tol = float(torch.quantile(raw[: 1 << 20], 0.9))   # a tolerance the network misses often
        thr = fc.fc_surrogate_guard(sc.h, L, y, tol)
        assert np.isfinite(thr)
        nfb = fc.fc_surrogate_eval(sc.h, L, out)
        torch.cuda.synchronize()
        err = (out - y).abs()
        precision("surrogate ln T, guarded", "small head scan, tol %.1e, %.1f%% of rays exact"
                  % (tol, 100.0 * nfb / y.numel()), float(err.max()) / tol, 1.0, "of tol")
        assert float(err.max()) <= tol
        assert (raw > tol).sum().item() <= nfb <= y.numel()
        # a tolerance above the network's worst error: no ray beyond it
        assert fc.fc_surrogate_guard(sc.h, L, y, 2.0 * float(raw.max()) + 1e-6) == float("inf")
        assert fc.fc_surrogate_eval(sc.h, L, out) == nfb0
        assert fc.fc_surrogate_guard(sc.h, L, y, 0.0) == float("inf")
        assert fc.fc_surrogate_eval(sc.h, L, out) == nfb0
    finally:
        fc.fc_surrogate_guard(sc.h, L, y, 0.0)

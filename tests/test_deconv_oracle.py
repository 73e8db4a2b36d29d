"""Pins of the Richardson-Lucy oracle (EM update for Poisson data with the
detector's clamp-to-edge blur).  CPU only."""
import numpy as np
import pytest

from oracle import deconv as OD


def test_clamp_blur_matrix_matches_oracle_blur(orc):
    # the explicit operator is the oracle's pinned clamp-to-edge blur
    rng = np.random.default_rng(1)
    X = rng.uniform(0.1, 1.0, size=(2, 13, 21))
    Bv, Bu = OD.clamp_blur_matrix(13, 1.3), OD.clamp_blur_matrix(21, 1.3)
    np.testing.assert_allclose(OD.forward(X, Bv, Bu), orc.gauss_blur(X, 1.3), rtol=1e-13)


def test_adjoint_identity():
    rng = np.random.default_rng(2)
    Bv, Bu = OD.clamp_blur_matrix(41, 2.1), OD.clamp_blur_matrix(9, 0.9)
    X = rng.normal(size=(41, 9))
    Y = rng.normal(size=(41, 9))
    lhs = np.sum(OD.forward(X, Bv, Bu) * Y)
    rhs = np.sum(X * OD.adjoint(Y, Bv, Bu))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    # interior columns of H^T 1 are 1 (taps sum to one); edges collect the clamp
    n = OD.adjoint(np.ones((41, 9)), Bv, Bu)
    assert n[20, 4] == pytest.approx(1.0, rel=1e-14)
    assert n[0, 0] > 1.0


def test_rl_fixed_point_flux_and_kl_descent():
    rng = np.random.default_rng(3)
    nv, nu, s = 24, 30, 1.5
    Bv, Bu = OD.clamp_blur_matrix(nv, s), OD.clamp_blur_matrix(nu, s)
    truth = np.full((nv, nu), 50.0)
    truth[8:12, 10:13] = 400.0
    truth[18, 5] = 900.0
    d = OD.forward(truth, Bv, Bu)
    # exact data and u_0 = truth: the update leaves it in place
    e = OD.forward(truth, Bv, Bu)
    u1 = truth * OD.adjoint(d / e, Bv, Bu) / OD.adjoint(np.ones_like(d), Bv, Bu)
    np.testing.assert_allclose(u1, truth, rtol=1e-12)
    # flux: sum(H^T 1 * u_{k+1}) = sum(d) after every step; KL(d || H u_k) decreases
    norm = OD.adjoint(np.ones_like(d), Bv, Bu)
    dn = rng.poisson(d).astype(np.float64)
    kl_prev = np.inf
    for k in range(1, 6):
        u = OD.richardson_lucy(dn, s, k)
        assert np.sum(norm * u) == pytest.approx(np.sum(dn), rel=1e-12)
        Hu = OD.forward(u, Bv, Bu)
        kl = np.sum(dn * np.log(np.maximum(dn, 1e-300) / Hu) - dn + Hu)
        assert kl <= kl_prev + 1e-9
        kl_prev = kl
        assert np.all(u >= 0)
    # deblurring sharpens the point: its peak rises toward the truth
    u = OD.richardson_lucy(d, s, 30)
    assert u[18, 5] > d[18, 5] * 1.5

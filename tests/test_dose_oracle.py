"""Pins of the dose estimate (Sec. II.H, D0(E) and Dp equations) and of the
water energy-absorption ratio it takes as input.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import dose as OD
from paper_2011_04736_gb300 import workloads as W


def _kn_dsigma(c, k):
    """Klein-Nishina d(sigma)/d(Omega) in units of r_e^2 at cos(theta) = c."""
    r = 1.0 / (1.0 + k * (1.0 - c))
    return 0.5 * r * r * (r + 1.0 / r - (1.0 - c * c))


@pytest.mark.parametrize("e_kev", [10.0, 60.0, 120.0, 511.0, 2500.0])
def test_klein_nishina_closed_forms_match_quadrature(e_kev):
    # total and scattered-energy cross-sections, integrated over the sphere
    quad = pytest.importorskip("scipy.integrate").quad
    k = e_kev / W.ELECTRON_REST_KEV
    s_t = 8.0 * math.pi / 3.0
    tot = quad(lambda c: 2 * math.pi * _kn_dsigma(c, k), -1, 1, epsabs=0, epsrel=1e-13)[0]
    sc = quad(lambda c: 2 * math.pi * _kn_dsigma(c, k) / (1 + k * (1 - c)), -1, 1,
              epsabs=0, epsrel=1e-13)[0]
    assert W.klein_nishina_ratio(e_kev) == pytest.approx(tot / s_t, rel=1e-10)
    assert W.klein_nishina_scatter_ratio(e_kev) == pytest.approx(sc / s_t, rel=1e-10)


def test_compton_energy_transfer_fraction():
    # mean fraction of the photon energy given to the electron: ~k for k -> 0
    # and the textbook 0.138 (100 keV) and 0.440 (1 MeV)
    def ftr(e):
        return 1.0 - W.klein_nishina_scatter_ratio(e) / W.klein_nishina_ratio(e)
    k = 1.0 / W.ELECTRON_REST_KEV
    assert ftr(1.0) / k == pytest.approx(1.0, rel=5e-3)
    assert ftr(100.0) == pytest.approx(0.138, abs=1e-3)
    assert ftr(1000.0) == pytest.approx(0.440, abs=1e-3)


def test_muen_over_mu_water_limits():
    e = np.array([10.0, 30.0, 80.0, 500.0, 2000.0])
    r = W.muen_over_mu("water", e)
    assert np.all((r > 0) & (r <= 1))
    # photo-electric dominance: nearly all of the interaction energy is absorbed
    assert W.muen_over_mu("water", 5.0) > 0.95
    # Compton only (photo-electric term switched off): the energy-transfer fraction
    rho, zoa, _ = W.MATERIALS["water"]
    W.MATERIALS["_compton"] = (rho, zoa, 0.0)
    try:
        ftr = 1.0 - W.klein_nishina_scatter_ratio(e) / W.klein_nishina_ratio(e)
        np.testing.assert_allclose(W.muen_over_mu("_compton", e), ftr, rtol=1e-14)
    finally:
        del W.MATERIALS["_compton"]


def _geom(**kw):
    base = dict(sad=50.0, sdd=100.0, n_u=4, n_v=4, du=0.01, dv=0.01, n_angles=8,
                nx=4, ny=4, nz=4, dx=2.0, dy=2.0, dz=2.0)
    base.update(kw)
    return W.Geometry(**base)


def test_dose_full_absorption_units():
    # every ray crosses ~8 cm of an opaque cube: each one deposits all of E
    # (mu_en/mu = 1), so D0 = E / M; 1 MeV in 1 g is 1.602176634e-10 Gy
    g = _geom()
    lab = np.ones((g.nz, g.ny, g.nx), np.uint8)
    mu = np.array([[0.0, 50.0], [0.0, 80.0]])
    e = np.array([1000.0, 250.0])
    d0, dp = OD.dose_estimate(g, lab, mu, e, np.ones(2), np.array([1.0, 3.0]),
                              np.array([0.0012, 1.0]), a0=0, na=2)
    M = 8.0 ** 3 * 1.0
    np.testing.assert_allclose(d0, [1.602176634e-10 / M, 0.25 * 1.602176634e-10 / M], rtol=1e-13)
    assert dp == pytest.approx(0.25 * d0[0] + 0.75 * d0[1], rel=1e-13)


def test_dose_two_slab_parallel_closed_form():
    # nearly parallel rays (SAD 1 km) along -x through two 1 cm slabs of
    # different materials: A(E) = N (1 - exp(-(mu_1(E) + mu_2(E)) * 1 cm))
    g = _geom(sad=1e5, sdd=2e5, n_u=3, n_v=3, du=0.5, dv=0.5, n_angles=1,
              nx=2, ny=2, nz=2, dx=1.0, dy=1.0, dz=1.0)
    lab = np.zeros((2, 2, 2), np.uint8)
    lab[:, :, 0] = 1
    lab[:, :, 1] = 2
    mu = np.array([[0.01, 0.2, 0.5], [0.02, 0.1, 0.3], [0.0, 0.05, 0.9]])
    e = np.array([40.0, 70.0, 100.0])
    muen = np.array([0.9, 0.5, 0.3])
    rho = np.array([0.0012, 1.0, 2.0])
    d0, dp = OD.dose_estimate(g, lab, mu, e, muen, np.ones(3), rho)
    M = 4 * 1.0 + 4 * 2.0
    want = 1.602176634e-13 * e * muen * (1 - np.exp(-(mu[:, 1] + mu[:, 2]))) / M
    np.testing.assert_allclose(d0, want, rtol=1e-9)
    assert dp == pytest.approx(want.mean(), rel=1e-9)


def test_absorbed_equals_one_minus_monoenergetic_projection():
    # energy conservation: with a one-bin spectrum the projector's T is the
    # fraction that passes, so the absorbed sum is sum_i (1 - T_i)
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=24, n_v=20, nx=16, ny=16, nz=8, dx=1.0,
                  dy=1.0, dz=1.0, n_angles=4, du=0.6, dv=0.6)
    g = wl.geom
    lab = wl.make_phantom()
    mu = wl.mu()
    idx = OD.all_rays(g, 1, 2)
    L, _ = oracle.rays(g, lab, np.ones(wl.n_e), np.ones(wl.n_e), mu, idx)
    A = OD.absorbed(L, mu)
    for e in (0, wl.n_e // 2, wl.n_e - 1):
        w = np.zeros(wl.n_e)
        w[e] = 1.0
        T = oracle.project_T(g, lab, w, np.ones(wl.n_e), mu, a0=1, na=2)
        assert A[e] == pytest.approx(np.sum(1.0 - T), rel=1e-12)
    assert np.all(A > 0)


def test_dp_spectrum_properties():
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=16, n_v=12, nx=16, ny=16, nz=8, dx=1.0,
                  dy=1.0, dz=1.0, n_angles=4, du=0.8, dv=0.8)
    g = wl.geom
    lab = wl.make_phantom()
    w, _ = wl.spectrum()
    args = (g, lab, wl.mu(), wl.energies(), wl.muen_water())
    d0, dp = OD.dose_estimate(*args, w, wl.densities())
    d0b, dpb = OD.dose_estimate(*args, 7.0 * w, wl.densities())
    np.testing.assert_array_equal(d0, d0b)           # D0 does not depend on phi
    assert dpb == pytest.approx(dp, rel=1e-14)       # phi is normalised
    assert d0.min() <= dp <= d0.max()
    delta = np.zeros(wl.n_e)
    delta[3] = 2.0
    assert OD.dose_estimate(*args, delta, wl.densities())[1] == pytest.approx(d0[3], rel=1e-14)
    # doubling every density halves the dose (mass doubles, attenuation unchanged)
    d0m, _ = OD.dose_estimate(*args, w, 2.0 * wl.densities())
    np.testing.assert_allclose(d0m, 0.5 * d0, rtol=1e-14)

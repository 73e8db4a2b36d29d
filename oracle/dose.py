"""FP64 dose estimate per particle (Sec. II.H) -- TEST INFRASTRUCTURE.

Only the tests, the entry point's smoke check and the benchmark's CPU
baseline may import this module.  It restates the two dose equations of
Sec. II.H:

    D0(E) = 1 / (N_i M) sum_i E (mu_en/mu)(E) (1 - exp(-mu_i(E) x_i))
    Dp    = sum_E phi(E) D0(E)

with mu_i(E) x_i = sum_m mu_m(E) L_im, the ray's attenuation through the
labelled phantom (path lengths L from the oracle's Siddon traversal), the
energy-absorption ratio of water, N_i the number of rays summed over, M the
phantom mass (every voxel, density of its label times the voxel volume) and
phi the fluence spectrum normalised to one.  Energies in keV, mass in grams,
dose in Gy: 1 keV deposited in 1 g is 1.602176634e-16 J / 1e-3 kg.
"""
from __future__ import annotations

import numpy as np

import oracle

GY_PER_KEV_PER_GRAM = 1.602176634e-16 / 1e-3


def all_rays(g, a0, na):
    """(k, iv, iu) of every pixel ray of projections a0 .. a0+na-1."""
    k, v, u = np.meshgrid(np.arange(a0, a0 + na), np.arange(g.n_v), np.arange(g.n_u),
                          indexing="ij")
    return np.stack([k.ravel(), v.ravel(), u.ravel()], axis=1).astype(np.int32)


def absorbed(L, mu):
    """Per energy bin, sum over rays of 1 - exp(-sum_m mu_m(E) L_m).

    L [n_rays][n_mat] cm, mu [n_e][n_mat] 1/cm."""
    att = np.asarray(L, np.float64) @ np.asarray(mu, np.float64).T   # [n_rays][n_e]
    return (-np.expm1(-att)).sum(axis=0)


def phantom_mass(g, labels, rho):
    """M = dx dy dz sum_v rho(label_v), grams."""
    counts = np.bincount(np.asarray(labels).ravel(), minlength=len(rho))
    return g.dx * g.dy * g.dz * float(np.dot(counts[:len(rho)], np.asarray(rho, np.float64)))


def dose_from_lengths(L, mu, e_kev, muen_over_mu, w, mass):
    """(D0 [n_e], Dp) from the path lengths of the N_i rays summed over."""
    n_rays = np.asarray(L).shape[0]
    A = absorbed(L, mu)
    d0 = GY_PER_KEV_PER_GRAM * np.asarray(e_kev, np.float64) * np.asarray(muen_over_mu) * A
    d0 = d0 / (n_rays * mass)
    phi = np.asarray(w, np.float64) / np.sum(w)
    return d0, float(np.dot(phi, d0))


def dose_estimate(g, labels, mu, e_kev, muen_over_mu, w, rho, a0=0, na=1):
    """D0(E) and Dp over every ray of projections a0 .. a0+na-1."""
    mu = np.asarray(mu, np.float64)
    n_e = mu.shape[0]
    L, _ = oracle.rays(g, labels, np.ones(n_e), np.ones(n_e), mu, all_rays(g, a0, na))
    return dose_from_lengths(L, mu, e_kev, muen_over_mu, w, phantom_mass(g, labels, rho))

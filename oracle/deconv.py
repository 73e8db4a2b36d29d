"""FP64 Richardson-Lucy deconvolution of projections -- TEST INFRASTRUCTURE.

Only the tests, the entry point's smoke check and the benchmark's CPU
baseline may import this module.  The discussion of the paper (Sec. IV)
deconvolves the projection images with the detector PSF by Richardson-Lucy
before reconstruction.  Written here as the multiplicative EM update for
Poisson data d = Poisson(H u):

    u_{k+1} = u_k * H^T (d / (H u_k)) / H^T 1,      u_0 = d,

H the detector's clamp-to-edge separable sampled-Gaussian blur (the operator
the simulation applies) and H^T its exact adjoint, both as explicit matrices
per axis: H X = B_v X B_u^T on each [n_v][n_u] image.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_taps(sigma):
    """Sampled Gaussian on |j| <= ceil(4 sigma), normalised to one."""
    R = int(math.ceil(4.0 * sigma)) if sigma > 0 else 0
    j = np.arange(-R, R + 1, dtype=np.float64)
    t = np.exp(-j * j / (2.0 * sigma * sigma)) if R > 0 else np.ones(1)
    return t / t.sum()


def clamp_blur_matrix(n, sigma):
    """B with (B x)[p] = sum_j g_j x[clamp(p + j)] on an axis of length n."""
    g = gauss_taps(sigma)
    R = (len(g) - 1) // 2
    B = np.zeros((n, n))
    for p in range(n):
        for j in range(-R, R + 1):
            B[p, min(max(p + j, 0), n - 1)] += g[j + R]
    return B


def forward(X, Bv, Bu):
    """H X = B_v X B_u^T for a stack X [..., n_v, n_u] (two matrix products)."""
    return np.matmul(np.matmul(Bv, X), Bu.T)


def adjoint(Y, Bv, Bu):
    """H^T Y = B_v^T Y B_u for a stack Y [..., n_v, n_u] (two matrix products)."""
    return np.matmul(np.matmul(Bv.T, Y), Bu)


def richardson_lucy(d, sigma, n_iter, floor=1e-12):
    """n_iter RL updates of the stack d [..., n_v, n_u] (u_0 = d); H u is
    floored at `floor` before the division."""
    d = np.asarray(d, np.float64)
    nv, nu = d.shape[-2:]
    Bv, Bu = clamp_blur_matrix(nv, sigma), clamp_blur_matrix(nu, sigma)
    norm = adjoint(np.ones((nv, nu)), Bv, Bu)
    u = d.copy()
    for _ in range(n_iter):
        e = np.maximum(forward(u, Bv, Bu), floor)
        u = u * adjoint(d / e, Bv, Bu) / norm
    return u

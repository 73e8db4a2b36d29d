"""FP64 energy-group detector model -- TEST INFRASTRUCTURE.

Only the tests, the entry point's smoke check and the benchmark's CPU
baseline may import this module.  It restates the per-energy detector model
of the paper with the spectrum lumped into contiguous energy groups:

* scatter (Sec. II.E): an additive profile across the detector of the fitted
  form y(x) = (a / sqrt(x^2 + a^2))^b, x the off-axis distance, scaled per
  group by an amplitude relative to the flood;
* primary per group (Sec. II.F, the I_f equation split over groups):
  P_g = sum_{E in g} w D exp(-sum_m mu_m L_m) / sum_E w D, so sum_g P_g = T;
* optical spread per energy (Sec. II.G, OSF convolution at each energy and
  sum): each group's intensity is blurred with its own sampled Gaussian
  (clamp-to-edge) and the groups are summed:
      I = N0 sum_g G_g (x) (P_g + A_g y_g(x)).
Built only from the pinned primitives of ``oracle`` (projection, blur).
"""
from __future__ import annotations

import numpy as np

import oracle


def scatter_fit(x, a, b):
    """The scatter fit form of Sec. II.E: (a / sqrt(x^2 + a^2))^b."""
    x = np.asarray(x, np.float64)
    return (a / np.sqrt(x * x + a * a)) ** b


def off_axis_cm(g):
    """Off-axis distance of every detector column (cm, at the detector)."""
    return (np.arange(g.n_u) - (g.n_u - 1) / 2.0) * g.du


def group_primaries(g, labels, w, D, mu, bounds, a0=0, na=None):
    """P[g][k][iv][iu] for groups of bins [bounds[g], bounds[g+1])."""
    w = np.asarray(w, np.float64)
    D = np.asarray(D, np.float64)
    tot = float(np.sum(w * D))
    out = []
    for b0, b1 in zip(bounds[:-1], bounds[1:]):
        wg = np.zeros_like(w)
        wg[b0:b1] = w[b0:b1]
        cg = float(np.sum(wg * D)) / tot
        if cg == 0.0:
            na_ = g.n_angles - a0 if na is None else na
            out.append(np.zeros((na_, g.n_v, g.n_u)))
            continue
        out.append(cg * oracle.project_T(g, labels, wg, D, mu, a0=a0, na=na))
    return np.stack(out)


def intensity_groups(g, P, sigma, amp, a, b, n0):
    """I = N0 sum_g G_sigma_g (x) (P_g + amp_g y_g(x))."""
    x = off_axis_cm(g)
    I = np.zeros(P.shape[1:])
    for k in range(P.shape[0]):
        prof = amp[k] * scatter_fit(x, a[k], b[k])
        I += oracle.gauss_blur(P[k] + prof[None, None, :], sigma[k])
    return n0 * I

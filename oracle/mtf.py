"""FP64 detector MTF by the slanted-slit method (Sec. II.C) -- TEST
INFRASTRUCTURE.

Only the tests, the entry point's smoke check and the benchmark's CPU
baseline may import this module.  The paper weights the energy-dependent
optical spread by the spectrum's detected share to form the detector PSF,
convolves it with an ideal slit 0.3 mm wide tilted by 2.5 degrees, takes the
line spread function by presampling and its Fourier magnitude as the MTF.
Here, step by step:

1. slit image S (N x N pixels of pitch d): the area fraction of each pixel
   inside the strip |n . (x - c)| <= w / 2, n = (cos a, sin a) in (u, v), c
   the image centre;
2. I = sum_g c_g G_g (x) S, the detector blur of each group (sampled Gaussian,
   clamp-to-edge) weighted by the group's share c_g of the flood;
3. presampled LSF: rows [N/4, 3N/4) only; each pixel's signed distance s =
   n . (centre - c) falls in a bin of width d / os over [-16 d, 16 d); the LSF
   is the mean of I over each bin;
4. MTF(f) = |sum_b LSF_b exp(-2 pi i f s_b)| / |sum_b LSF_b| at
   f = k / (32 d) for k = 0 .. 16 os (s_b bin centres).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

N_IMAGE = 192
HALF_SPAN_PX = 16


def _trap_cdf(t, a, b):
    """CDF at t of the sum of two centred uniforms of widths a >= b >= 0."""
    t = np.asarray(t, np.float64)
    h = 0.5 * (a + b)
    if b == 0.0:
        return np.clip((t + 0.5 * a) / a, 0.0, 1.0)
    x = np.clip(t + h, 0.0, a + b)        # shift support to [0, a + b]
    out = np.where(x <= b, x * x / (2 * a * b),
                   np.where(x <= a, (x - 0.5 * b) / a,
                            1.0 - (a + b - x) ** 2 / (2 * a * b)))
    return out


def slit_image(n, pitch, width, angle_rad):
    """Area fraction of every pixel inside the tilted strip."""
    c, s = math.cos(angle_rad), math.sin(angle_rad)
    x = (np.arange(n) - (n - 1) / 2.0) * pitch
    U, V = np.meshgrid(x, x)               # [row v][col u]
    sc = U * c + V * s
    a, b = pitch * max(abs(c), abs(s)), pitch * min(abs(c), abs(s))
    return _trap_cdf(-sc + 0.5 * width, a, b) - _trap_cdf(-sc - 0.5 * width, a, b)


def mtf(pitch_cm, weights, sigmas_px, width_mm=0.3, angle_deg=2.5, oversample=4):
    """(frequencies in 1/mm, MTF) of the detector PSF sum_g weights_g G_sigma_g."""
    n = N_IMAGE
    a = math.radians(angle_deg)
    S = slit_image(n, pitch_cm, width_mm / 10.0, a)
    w = np.asarray(weights, np.float64)
    w = w / w.sum()
    I = np.zeros_like(S)
    for wg, sg in zip(w, sigmas_px):
        I += wg * oracle.gauss_blur(S[None], sg)[0]
    x = (np.arange(n) - (n - 1) / 2.0) * pitch_cm
    U, V = np.meshgrid(x, x)
    s = U * math.cos(a) + V * math.sin(a)
    nb = 2 * HALF_SPAN_PX * oversample
    delta = pitch_cm / oversample
    rows = slice(n // 4, 3 * n // 4)
    b = np.floor(s[rows] / delta + nb / 2).astype(np.int64)
    ok = (b >= 0) & (b < nb)
    tot = np.bincount(b[ok], weights=I[rows][ok], minlength=nb)
    cnt = np.bincount(b[ok], minlength=nb)
    lsf = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)
    sb = (np.arange(nb) - nb / 2 + 0.5) * delta
    f = np.arange(nb // 2 + 1) / (nb * delta)          # 1/cm
    ph = np.exp(-2j * np.pi * np.outer(f, sb))
    m = np.abs(ph @ lsf) / abs(lsf.sum())
    return f / 10.0, m


def mtf_closed_form(f_per_mm, pitch_cm, weights, sigmas_px, width_mm=0.3, angle_deg=2.5,
                    oversample=4):
    """Transfer chain of the same measurement: slit (sinc of its width), pixel
    aperture projected on the slit normal (two sincs), the sampled Gaussian's
    transform along the normal, and the bin width (sinc)."""
    f = np.asarray(f_per_mm, np.float64) * 10.0          # 1/cm
    a = math.radians(angle_deg)
    dc, ds = pitch_cm * math.cos(a), pitch_cm * math.sin(a)
    w = np.asarray(weights, np.float64)
    w = w / w.sum()

    def dtft(sig, nu):
        R = int(math.ceil(4 * sig)) if sig > 0 else 0
        j = np.arange(-R, R + 1)
        g = np.exp(-j * j / (2 * sig * sig)) if R > 0 else np.ones(1)
        g = g / g.sum()
        return np.cos(2 * np.pi * np.outer(nu, j)) @ g

    psf = sum(wg * dtft(sg, f * dc) * dtft(sg, f * ds) for wg, sg in zip(w, sigmas_px))
    chain = (np.sinc(f * width_mm / 10.0) * np.sinc(f * dc) * np.sinc(f * ds)
             * np.sinc(f * pitch_cm / oversample))
    return np.abs(chain * psf)

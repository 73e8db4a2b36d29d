"""Pins of the slanted-slit MTF oracle (Sec. II.C).  CPU only."""
import math

import numpy as np
import pytest

from oracle import mtf as OM


def test_slit_image_area():
    # every row crosses the strip over w / cos(a): the row's area fractions
    # add up to w / (d cos a); all fractions lie in [0, 1]
    d, w, a = 0.04, 0.03, math.radians(2.5)
    S = OM.slit_image(64, d, w, a)
    assert S.min() >= 0.0 and S.max() <= 1.0 + 1e-15
    np.testing.assert_allclose(S.sum(axis=1), w / (d * math.cos(a)), rtol=1e-12)
    # a slit wider than a pixel fills the pixels on its centre line completely
    S2 = OM.slit_image(32, d, 3 * d, 0.0)
    assert S2[:, 15].min() == pytest.approx(1.0) and S2[:, 16].min() == pytest.approx(1.0)


@pytest.mark.parametrize("pitch,weights,sigmas", [(0.0336, [1.0], [0.8]),
                                                  (0.0784, [0.6, 0.4], [1.0, 2.5]),
                                                  (0.04, [1.0], [0.0])])
def test_mtf_matches_transfer_chain(orc, pitch, weights, sigmas):
    # slit x pixel aperture x sampled Gaussian x bin width, below 0.8 Nyquist
    f, m = OM.mtf(pitch, weights, sigmas)
    cf = OM.mtf_closed_form(f, pitch, weights, sigmas)
    sel = f <= 0.8 / (2 * pitch * 10)
    assert m[0] == pytest.approx(1.0, abs=1e-12)
    assert np.max(np.abs(m - cf)[sel]) < 5e-3
    # a wider PSF transfers less at every frequency
    f2, m2 = OM.mtf(pitch, weights, [s + 0.5 for s in sigmas])
    assert np.all(m2[sel][1:] < m[sel][1:])

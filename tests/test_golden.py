"""The oracle against the stored expected values of tests/golden/ (written by
tests/golden/make_golden.py from the oracle).  The Poisson fixture pins the
sampler's specification (stream layout, binary32 operation order) so that a
build of the oracle on another machine, or a change to it, that moves a single
count is caught."""
import numpy as np

from golden_io import poisson_counts


def test_golden_poisson_counts_reproduced(orc):
    k0, per_seed = poisson_counts()
    assert len(per_seed) == 2
    for seed, (lam, ref) in per_seed.items():
        got = orc.poisson(lam, seed, k0=k0)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), \
            (seed, np.argwhere(got != ref)[:5])
        # every branch of the sampler is present in the fixture
        flat = lam.ravel()
        assert np.isnan(flat).any() and (flat <= 0).any()
        assert ((flat > 0) & (flat < 10)).any() and (flat > 1e7).any() and (flat >= 10).sum() > 100

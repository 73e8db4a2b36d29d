"""The CUDA Poisson sampler through the C ABI against the stored counts of
tests/golden/poisson_counts.txt (written from the oracle): bit-identical
counts for the stored rates, both seeds, a ragged 33-column row."""
import numpy as np
import pytest

from golden_io import poisson_counts

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


def test_gpu_poisson_matches_golden_counts(fc):
    k0, per_seed = poisson_counts()
    for seed, (lam, ref) in per_seed.items():
        d_lam = torch.from_numpy(lam).cuda()
        d_out = torch.empty_like(d_lam)
        n, nv, nu = lam.shape
        fc.fc_poisson(d_lam, d_out, n, nv, nu, k0, seed)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), \
            (seed, np.argwhere(got != ref)[:5])

"""Readers for the stored expected values under tests/golden/ (no arithmetic
of the method here)."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def poisson_counts():
    """Per seed: (k0, rates[k][iv][iu] float32, counts[k][iv][iu] float32)
    from poisson_counts.txt."""
    path = os.path.join(GOLDEN, "poisson_counts.txt")
    shape = k0 = None
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("# shape"):
                parts = line.split()
                shape = tuple(int(x) for x in parts[2:5])
                k0 = int(parts[6])
            elif line.strip() and not line.startswith("#"):
                rows.append(line.split())
    out = {}
    for seed, k, iv, iu, lam, cnt in rows:
        seed, k, iv, iu = int(seed), int(k), int(iv), int(iu)
        if seed not in out:
            out[seed] = (np.zeros(shape, np.float32), np.zeros(shape, np.float32))
        out[seed][0][k - k0, iv, iu] = math.nan if lam == "nan" else float.fromhex(lam)
        out[seed][1][k - k0, iv, iu] = float(cnt)
    return k0, out

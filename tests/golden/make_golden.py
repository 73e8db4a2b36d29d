"""Writes the stored expected values under tests/golden/ from the oracle alone.

poisson_counts.txt pins the counter-based Poisson sampler (Sec. II.G-H of the
paper: Poisson sampling of the counts reaching each pixel; the stream layout
and the binary32 operation order are this project's specification, written
out in ``oracle/noise_oracle.c``).  The paper prints no sampled counts, so the
values are the oracle's: the file locks the specification against silent
change and lets any build of the oracle or of the GPU sampler be checked
bit for bit.  Rates cover every branch of the sampler: zero, negative and NaN
rates, inversion (rate < 10), PTRS near its lower limit and at detector
count levels, the rounding branch above 1e7.

Run from the repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

# (projections, rows, columns) of each rate block; 33 columns leave a ragged
# tail past one warp's 32 column pairs, two rows and projections exercise
# the counter's row and projection words.
SHAPE = (2, 3, 33)
K0 = 5
SEEDS = (1, 0x1234567890AB)
FIXED = [0.0, -1.0, float("nan"), 1.0e-6, 0.5, 3.0, 9.999, 10.0, 10.5, 47.3, 300.0,
         6.5e3, 1.0e5, 1.2e5, 9.9e6, 1.0e7, 1.5e7]


def rates():
    n = int(np.prod(SHAPE))
    rng = np.random.default_rng(20110473)
    lam = np.empty(n, np.float32)
    lam[: len(FIXED)] = np.array(FIXED, np.float32)
    rest = n - len(FIXED)
    # log-uniform over the PTRS range, where nearly every detector pixel lies
    lam[len(FIXED):] = np.exp(rng.uniform(math.log(10.0), math.log(2.0e5), rest)).astype(np.float32)
    return lam.reshape(SHAPE)


def fmt_rate(x):
    return "nan" if math.isnan(x) else float(x).hex()


def main():
    oracle.build()
    lam = rates()
    lines = ["# seed k iv iu rate(float32, hex) count -- written by make_golden.py from oracle.poisson",
             "# shape %d %d %d k0 %d" % (SHAPE + (K0,))]
    for seed in SEEDS:
        out = oracle.poisson(lam, seed, k0=K0)
        for k in range(SHAPE[0]):
            for iv in range(SHAPE[1]):
                for iu in range(SHAPE[2]):
                    lines.append("%d %d %d %d %s %d" % (seed, K0 + k, iv, iu,
                                                        fmt_rate(float(lam[k, iv, iu])),
                                                        int(out[k, iv, iu])))
    with open(os.path.join(HERE, "poisson_counts.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


# Measured errors against the FP64 oracle, recorded by the parity tests and
# printed as one table at the end of the run (the precision report of every
# output: what, size, max error, tolerance).
_PRECISION = []


@pytest.fixture(scope="session")
def precision():
    def rec(output, case, err, tol, unit="relative"):
        _PRECISION.append((output, case, float(err), float(tol), unit))
        return err
    return rec


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if not _PRECISION:
        return
    tr = terminalreporter
    tr.write_sep("=", "measured error against the FP64 oracle")
    tr.write_line("%-28s %-52s %12s %10s  %s" % ("output", "case", "max error", "bound", "unit"))
    for output, case, err, tol, unit in _PRECISION:
        tr.write_line("%-28s %-52s %12.3e %10.1e  %s" % (output, case, err, tol, unit))

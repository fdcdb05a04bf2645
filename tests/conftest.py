"""Shared pytest fixtures.  Tests marked ``gpu`` need a GB300 and the built
CUDA library; everything else runs on the CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libmc.so")
    config.addinivalue_line("markers", "slow: long-running statistical test")


def binned_mean_err(x, nbins: int = 20):
    """Mean and standard error of a correlated series by non-overlapping bins."""
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbins) * nbins
    b = x[len(x) - n:].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle

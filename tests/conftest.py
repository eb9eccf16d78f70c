import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C ABI)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def stp_lib():
    """Build libstp.so if needed and return the binding module."""
    from paper_1511_07800_gb300 import build, stp
    build.build()
    stp.lib()
    return stp


def rel_err(a, b):
    import numpy as np
    a, b = np.asarray(a), np.asarray(b)
    den = max(float(np.abs(b).max()), 1e-300)
    return float(np.abs(a - b).max()) / den


def gauge(p, cfg):
    """p with its volume-weighted mean removed (the gauge stp_poisson_solve
    returns: L p = b fixes p only up to a constant)."""
    import numpy as np
    from paper_1511_07800_gb300 import inputs
    dz = np.diff(inputs.zfaces(cfg))[:, None, None]
    return p - np.sum(p * dz) / (np.sum(dz) * p.shape[1] * p.shape[2])

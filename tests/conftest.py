import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def oracle_c_built():
    """Build the oracle's C sketch loop if it is missing (CPU only)."""
    so = os.path.join(ROOT, "oracle", "_oracle_sketch.so")
    if not os.path.exists(so):
        from oracle import build as ob
        ob.build()
    return so

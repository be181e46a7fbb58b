import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")



@pytest.fixture(scope="session")
def libtc():
    """Path of the built libtc.so (built here if stale); skips without nvcc.
    For CPU tests that reach the library's host-only entry points."""
    import shutil

    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1503_00576_gb300 import build

    return build.build()

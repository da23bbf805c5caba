import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmsf.so")
    config.addinivalue_line("markers", "slow: larger CPU or GPU cases")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def msflib():
    """The built CUDA library (compiled on demand; no GPU needed to load it)."""
    from paper_1903_12294_gb300 import build, msf
    build.build()
    return msf


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu(msflib):
    if not _has_gpu():
        pytest.fail("GPU test collected on a machine without a CUDA device")
    import torch
    torch.cuda.init()
    return msflib

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: long CPU physics run of the oracle")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def lbm():
    """The GPU library's Python binding; fails loudly when it cannot load."""
    if not gpu_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    from paper_1906_11027_gb300 import lbm as _lbm
    _lbm.load()
    return _lbm

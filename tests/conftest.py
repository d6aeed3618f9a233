import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


_CUDA = None


def pytest_runtest_setup(item):
    """A test marked gpu is skipped, before its fixtures, where no CUDA device
    is present (it would otherwise fail at the library's first device call)."""
    global _CUDA
    if item.get_closest_marker("gpu") is None:
        return
    if _CUDA is None:
        import torch
        _CUDA = torch.cuda.is_available()
    if not _CUDA:
        pytest.skip("no CUDA device")


def relerr(a, b):
    """Normwise relative difference max|a-b| / max|b| (0 if both vanish)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b)) if b.size else 0.0
    diff = np.max(np.abs(a - b)) if a.size else 0.0
    if scale == 0.0:
        return diff
    return diff / scale


@pytest.fixture
def rel():
    return relerr

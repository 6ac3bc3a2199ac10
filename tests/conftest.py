import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its C-ABI binding; fails loudly if not built."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_08076_gb300 import richm
    return richm


@pytest.fixture(scope="session")
def built_lib():
    """Build librichm.so (nvcc cross-compiles without a GPU) for tests that call its
    host-only entry points."""
    from paper_2412_08076_gb300.build import build
    return build()

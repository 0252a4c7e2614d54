import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def lib():
    """libmrtlb.so, built in-tree if needed (nvcc cross-compiles without a GPU)."""
    from paper_1106_0785_gb300 import build, mrtlb
    build.build()
    return mrtlb.load()


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_0785_gb300 import build, mrtlb
    build.build()
    mrtlb.load()
    return torch.device("cuda:0")

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def hlb_lib():
    """libhlb, built in-tree if it is missing (nvcc cross-compiles without a GPU)."""
    from paper_1708_03249_gb300 import build, hlb
    if not os.path.exists(hlb.LIB_PATH):
        build.build()
    return hlb.lib()


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


@pytest.fixture(scope="session")
def fdlib():
    """The CUDA library's binding, built in place first if its sources changed."""
    from paper_2311_05038_b300.build import build
    build()
    import paper_2311_05038_b300.fd as fd
    return fd


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False

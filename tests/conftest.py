import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the px library")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def px():
    """The CUDA library binding; GPU tests fail loudly if it is missing."""
    if not gpu_available():
        pytest.fail("GPU test collected on a machine without a CUDA device")
    import paper_2606_24647_gb300 as pxm
    pxm.load()
    return pxm

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library handle module; fails loudly when no GPU is present."""
    if not _have_gpu():
        pytest.fail("GPU test selected but no CUDA device is visible")
    import paper_0704_3486_gb300 as ovs
    ovs.load()
    return ovs

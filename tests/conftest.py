import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmusr")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def musr_lib():
    """The built CUDA library; GPU tests fail loudly if it cannot be loaded."""
    from paper_1509_07685_gb300 import binding
    return binding.load()

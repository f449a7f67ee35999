import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library through its Python binding; skips nothing: a gpu test without a GPU fails."""
    import torch

    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    from paper_1612_00474_gb300 import rpb

    rpb.load()
    return rpb

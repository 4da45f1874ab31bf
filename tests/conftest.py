import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled CUDA library")


@pytest.fixture(scope="session")
def gpu_lib():
    """The compiled CUDA library through its Python binding; fails loudly if it is missing."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    import paper_2412_03378_gb300 as vg

    vg.load()
    return vg

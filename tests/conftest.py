import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def qdpg_gpu():
    """The CUDA library, loaded and checked for a device; fails loudly otherwise."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but torch sees no CUDA device")
    import paper_1111_5596_gb300 as q

    q.load()
    return q

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def hg():
    """The CUDA binding; building it first.  Fails loudly if the GPU path is unavailable."""
    import torch
    from paper_1207_2367_gb300 import binding
    if not torch.cuda.is_available():
        pytest.fail("gpu test collected on a machine without CUDA")
    binding.load()
    return binding

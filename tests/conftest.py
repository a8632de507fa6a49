import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def has_gpu():
    import torch
    return torch.cuda.is_available()


@pytest.fixture(scope="module", autouse=True)
def _release_device_block_cache():
    """After each test module that used the library on a GPU, the library's
    cache of device blocks goes back to the driver, so that later framework
    allocations find the device as the library's contexts left it."""
    yield
    torch = sys.modules.get("torch")
    ub = sys.modules.get("paper_2107_05397_b300.binding")
    if torch is None or ub is None or not torch.cuda.is_available():
        return
    ub.unifrac_release_cached_memory(-1)

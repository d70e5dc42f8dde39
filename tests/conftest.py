import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(autouse=True)
def _release_cached_device_memory(request):
    # large GPU tests leave torch's caching allocator holding tens of GiB; the
    # library sizes some choices by the device's free memory (the gradient's
    # stored forward states), so each GPU test starts with the cache released
    if "gpu" in request.keywords and cuda_available():
        import gc
        import torch
        gc.collect()
        torch.cuda.empty_cache()
    yield


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a); calls the CUDA library through its C ABI")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def hexlib():
    """Builds (if needed) and loads libhexgpu.so; GPU tests fail loudly if
    the CUDA library or a GPU is missing."""
    import torch
    from paper_2103_16400_gb300 import build, capi
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return capi.load()

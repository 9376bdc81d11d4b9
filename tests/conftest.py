import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def G():
    """The CUDA library's Python binding, built for sm_103a (GPU tests only)."""
    import torch
    from paper_2605_25124_gb300 import build
    build.build()
    import paper_2605_25124_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return pkg

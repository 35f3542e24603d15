import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libhydro.so")
    config.addinivalue_line("markers", "slow: longer oracle runs")


@pytest.fixture(scope="session")
def hydro_lib():
    """The CUDA library, built in-tree if needed; GPU tests fail (not skip) without a GPU."""
    from paper_2503_04428_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_04428_gb300 import hydro
    hydro.lib()
    return hydro

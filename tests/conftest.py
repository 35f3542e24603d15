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


def pytest_terminal_summary(terminalreporter):
    """The worst relative-L1 and element-wise errors of every parity test that
    ran (tests/parity.py), beside its bars."""
    try:
        import parity
    except ImportError:
        return
    if not parity.WORST:
        return
    tr = terminalreporter
    tr.write_sep("-", "parity: worst errors against the oracle (relative L1 / element-wise, bars)")
    for name in sorted(parity.WORST):
        e1, em, b1, bm = parity.WORST[name]
        tr.write_line("%-90s L1 %.2e (<= %.0e)  max %.2e (<= %.0e)" % (name[-90:], e1, b1, em, bm))

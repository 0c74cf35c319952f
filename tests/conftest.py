import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (the GB300 parity and kernel tests)")


@pytest.fixture(scope="session")
def lqlib():
    """Build (if stale) and load liblq.so; GPU tests fail loudly when it cannot be built."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00195_gb300 import build
    build.build()
    from paper_1611_00195_gb300 import lq
    return lq.lib()

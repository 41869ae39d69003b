import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def built_lib():
    """Build libsvsim.so (nvcc cross-compiles without a GPU) and load it."""
    from paper_2604_12256_gb300 import build as B
    from paper_2604_12256_gb300 import svsim as S
    B.build()
    return S.load()

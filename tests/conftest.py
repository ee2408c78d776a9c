import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    import oracle as o
    o.build()
    return o


@pytest.fixture(scope="session")
def awglib():
    """The CUDA library, built in-tree if needed (nvcc cross-compiles without a GPU)."""
    from paper_2403_15582_gb300 import build
    build.build()
    import paper_2403_15582_gb300 as awg
    awg.lib()
    return awg

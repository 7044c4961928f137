import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def crnt_lib():
    """The product library, built in-tree if needed (nvcc cross-compiles
    without a GPU)."""
    from paper_1905_01141_gb300 import build
    build.build()
    import paper_1905_01141_gb300 as crnt
    crnt.load()
    return crnt

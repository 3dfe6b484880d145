import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgs.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def gs():
    """The CUDA path's Python binding; the library is built if missing."""
    from paper_2601_19489_gb300 import _lib

    _lib.load()
    import paper_2601_19489_gb300 as pkg

    return pkg

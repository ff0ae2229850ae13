import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")

import pytest


@pytest.fixture(scope="session")
def spaqr_lib():
    """The built C-ABI library (built here with nvcc if missing)."""
    from paper_2010_06807_gb300 import build as _b
    import paper_2010_06807_gb300 as pkg
    _b.build()
    return pkg.load_library()

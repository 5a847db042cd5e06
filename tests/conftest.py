import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session", autouse=True)
def _native_library(request):
    """Build libiga_fd.so once if it is missing (the GPU tests call it)."""
    from paper_1705_04384_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1705_04384_gb300 import build
        build.build()
    yield

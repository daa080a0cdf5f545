import ctypes
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests through the C ABI)")


def _gpu_count() -> int:
    for name in ("libcudart.so", "libcudart.so.13", "libcudart.so.12"):
        try:
            rt = ctypes.CDLL(name)
        except OSError:
            continue
        n = ctypes.c_int(0)
        if rt.cudaGetDeviceCount(ctypes.byref(n)) == 0:
            return n.value
        return 0
    return 0


@pytest.fixture(scope="session")
def gpu_lib():
    """The built CUDA library (built in-tree if missing); skips when no GPU is visible."""
    if _gpu_count() < 1:
        pytest.skip("no CUDA GPU visible")
    from paper_2207_12848_gb300 import build, load
    build.build()
    return load()


@pytest.fixture()
def ctx(gpu_lib):
    from paper_2207_12848_gb300 import Context
    c = Context(0)
    yield c
    c.close()

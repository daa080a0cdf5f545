import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests through the C ABI)")
    config.addinivalue_line("markers", "slow: full-size workload (minutes)")


def _gpu_count() -> int:
    try:
        import torch
        return torch.cuda.device_count() if torch.cuda.is_available() else 0
    except Exception:
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

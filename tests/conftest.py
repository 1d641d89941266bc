import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libtsvd.so")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def tsvd():
    """The package with libtsvd.so built (fails loudly if the build fails)."""
    from paper_2403_06218_gb300 import build as _b
    _b.build()
    import paper_2403_06218_gb300 as t
    t.load()
    return t

import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libisdf.so")
    config.addinivalue_line("markers", "slow: oracle work of a minute or more")


@pytest.fixture(scope="session")
def lib_built():
    """Build libisdf.so once per session (nvcc cross-compiles without a GPU)."""
    from paper_2601_16379_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch

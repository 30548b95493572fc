import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.fixture(scope="session")
def gpu():
    """The product library on cuda:0.  Skips only when there is no GPU at all;
    on a GPU host a library that fails to build or load is an error."""
    if not cuda_available():
        pytest.skip("no CUDA device")
    import torch
    import paper_1506_08612_gb300 as dd
    torch.cuda.set_device(0)
    return dd

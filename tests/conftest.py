import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300)")
    config.addinivalue_line("markers", "slow: long-running full-size case")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def seqcdc_lib():
    """The CUDA library's Python binding (builds libseqcdc.so if needed)."""
    from paper_2505_21194_gb300 import seqcdc
    seqcdc.load_library()
    return seqcdc


@pytest.fixture(scope="session")
def gpu(seqcdc_lib):
    if not cuda_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    import torch
    torch.cuda.init()
    return seqcdc_lib

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def cuda_lib():
    """The loaded C-ABI library on a CUDA device (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2603_01443_gb300 import capi

    return capi.lib()


@pytest.fixture(scope="session")
def host_lib():
    """The loaded C-ABI library for host-only calls (built here if missing)."""
    from paper_2603_01443_gb300 import capi

    if not os.path.exists(capi.LIB_PATH):
        from paper_2603_01443_gb300 import build

        build.build()
    return capi.lib()

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session", autouse=True)
def _built_host_libs():
    """The oracle and the structure generator are plain C; build them once."""
    import oracle
    from paper_1410_1914_gb300 import inputs
    oracle.build()
    inputs.build()


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library, built if stale; GPU tests need it and a device."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1914_gb300 import _lib, build
    build.build_cuda()
    return _lib.load()

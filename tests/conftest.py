import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def hmclib():
    """The built C-ABI library (built in-tree on first use)."""
    from paper_1402_4089_gb300 import build, hmc
    if not os.path.exists(hmc.LIB_PATH):
        build.build()
    return hmc.lib()


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4089_gb300 import build, hmc
    build.build()
    hmc.lib()
    return torch.device("cuda:0")

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: full-size workload (minutes on a CPU)")


def pytest_collection_modifyitems(config, items):
    # the gpu marker is explicit; nothing else to do
    return


@pytest.fixture(scope="session")
def native():
    """The ctypes binding, after an in-tree build of libselinv.so."""
    from paper_1604_02528_gb300 import buildlib
    buildlib.build()
    from paper_1604_02528_gb300 import _native
    return _native


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")

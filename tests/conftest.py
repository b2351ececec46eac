import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmsrep.so")
    config.addinivalue_line(
        "markers", "slow: full-size workload (seconds of CPU work)")


def pytest_collection_modifyitems(config, items):
    """Run GPU tests only where a GPU exists; everything else runs anywhere."""
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def rmat_full():
    from paper_2209_07552_gb300 import inputs as I
    return I.rmat_full()


@pytest.fixture(scope="session")
def laplace_full():
    from paper_2209_07552_gb300 import inputs as I
    return I.laplace_full()

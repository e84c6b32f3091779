import os
import sys

import pytest

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
for p in (_ROOT, _HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblpdec")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library, built in-tree and loaded; fails (never skips) without a GPU."""
    import torch

    from paper_1204_0556_gb300 import build, lpdec

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lpdec.load()
    torch.cuda.init()
    return lpdec

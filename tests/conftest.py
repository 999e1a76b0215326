import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.lib()  # builds libhemeoracle.so on first use
    return oracle


@pytest.fixture(scope="session")
def hemegb_lib():
    """The built extension (compiled here if missing or stale; nvcc cross-compiles without a GPU)."""
    from paper_2010_04144_gb300 import build as B
    from paper_2010_04144_gb300 import hemegb

    B.build()
    return hemegb


@pytest.fixture(scope="session")
def gpu(hemegb_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return hemegb_lib

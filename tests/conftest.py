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
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    return oracle()


@pytest.fixture(scope="session")
def gpu():
    """Builds liblqcd.so, loads the binding and checks that a GPU is present."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU (run with -m 'not gpu' on CPU)")
    from paper_1701_00426_gb300 import build, lqcd
    build.build()
    lqcd.load()
    torch.cuda.init()
    return lqcd

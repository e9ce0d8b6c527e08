import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def lhlib():
    from paper_1708_07859_b300 import build, lh
    build.build()
    return lh


@pytest.fixture(scope="session")
def ctx(lhlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = lhlib.Context()
    yield c
    c.close()

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture
def gctx():
    """A b3t context on the current torch stream of cuda:0 (GPU tests)."""
    import torch
    import paper_1304_0878_b300 as b3t
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    c = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    yield c
    c.close()

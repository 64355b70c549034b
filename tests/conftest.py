import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def gpu_ctx():
    """One library context on cuda:0 for the GPU tests."""
    import torch
    import paper_0902_4424_gb300 as pkg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    ctx = pkg.Context(0)
    yield ctx
    ctx.close()

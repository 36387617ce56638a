import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU and the compiled MAPI library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def mapi_ctx():
    """One library context on cuda:0 for the GPU tests (built on demand)."""
    import torch

    import paper_2110_12065_gb300 as M
    from paper_2110_12065_gb300 import build as B
    B.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    ctx = M.mapi_create(0)
    yield ctx
    torch.cuda.synchronize()
    M.mapi_destroy(ctx)

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def nhctx():
    """One library context on cuda:0, bound to a dedicated torch stream so that
    torch allocations/copies and library launches are ordered."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2204_01722_b300 import nh
    stream = torch.cuda.Stream()
    ctx = nh.nh_create(0, stream.cuda_stream)
    with torch.cuda.stream(stream):
        yield ctx, stream
    torch.cuda.synchronize()
    nh.nh_destroy(ctx)

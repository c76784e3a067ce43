"""nh_dot_noalloc: the dot product for callers that cannot let the library
allocate device memory (their own pool allocator owns it, or a cudaMalloc's
device-wide synchronisation is not acceptable in their loop).  Its result must
match the allocating nh_dot within the tolerance of the other dot tests, on two
calls in a row (the second reuses the shared scratch the first left behind).

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

from paper_2204_01722_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot(nhctx):
    ctx, stream = nhctx
    from paper_2204_01722_b300 import nh
    for n, seed in ((3_000_001, 1), (777, 5)):
        xh = inputs.normal_vector(n, seed=seed)
        yh = inputs.normal_vector(n, seed=seed + 1)
        x = torch.from_numpy(xh).cuda()
        y = torch.from_numpy(yh).cuda()
        ref = nh.nh_dot(ctx, n, x, y)
        scale = max(1.0, float(np.linalg.norm(xh)) * float(np.linalg.norm(yh)))
        # the allocating entry point itself agrees with a host sum computed apart
        # from the library (math.fsum: correctly rounded)
        import math
        assert abs(ref - math.fsum((xh * yh).tolist())) <= 1e-12 * scale
        res = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        nh.nh_dot_noalloc(stream.cuda_stream, n, x, y, res[0:1])
        nh.nh_dot_noalloc(stream.cuda_stream, n, x, y, res[1:2])
        stream.synchronize()
        a, b = res.cpu().numpy()
        assert abs(a - ref) <= 1e-12 * scale
        assert abs(b - ref) <= 1e-12 * scale
        exact = math.fsum((xh * yh).tolist())
        assert abs(a - exact) <= 1e-12 * scale
        assert a == b          # fixed summation order
    # empty input gives 0; oversize n is refused before anything runs
    res = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    nh.nh_dot_noalloc(stream.cuda_stream, 0, None, None, res)
    stream.synchronize()
    assert float(res.item()) == 0.0
    with pytest.raises(nh.NhError) as ei:
        nh.nh_dot_noalloc(stream.cuda_stream, nh.NH_DOT_NOALLOC_MAX_N + 1, x, y, res)
    assert ei.value.status == nh.NH_ERR_UNSUPPORTED

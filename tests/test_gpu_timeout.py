"""Failure detection on the GPU without a fault: every spin-wait in the kernels is
bounded.  A test hook launches a kernel whose wait cannot complete (an mbarrier that
no copy arrives on; a grid barrier that one block of a cooperative launch skips) with
a short poll limit.  The wait must give up, the next synchronisation must report
NH_ERR_TIMEOUT, and the context must stay usable: an FP32 apply (staged loads on
mbarriers) and an FP64 apply afterwards still match the oracle."""
import numpy as np
import pytest

import parity
from oracle import fem
from paper_2204_01722_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_expires_and_context_survives(nhctx, kind):
    from paper_2204_01722_b300 import nh
    ctx, _ = nhctx
    n, p = (8, 2, 3), 3
    V = inputs.box_vertices(*n, perturb=0.1, seed=4)
    sp = fem.Space(*n, V, p, p + 1)
    X = sp.node_coords()
    u = inputs.smooth_field(X, 0.05, seed=5).ravel()
    mask = inputs.uniaxial_mask(sp.node_dims)
    space, _, _ = nh.nh_space_box(ctx, *n, V, p, p + 1)
    nh.nh_space_set_dirichlet(ctx, space, mask)
    op = nh.nh_op_create(ctx, space, 0.3, None, 1.0, 0)
    nh.nh_qdata_setup(ctx, op, torch.as_tensor(u).cuda())
    nh.nh_sync(ctx)

    nh.nh_debug_wait_timeout(ctx, kind)
    with pytest.raises(nh.NhError) as e:
        nh.nh_sync(ctx)
    assert e.value.status == nh.NH_ERR_TIMEOUT
    nh.nh_sync(ctx)  # the flag was cleared with the report

    state = fem.qp_state(sp, fem.Material(1.0, 0.3, sp.ne), u)
    du = inputs.normal_vector(sp.n_dof, seed=6)
    ref = fem.jacobian_apply(sp, state, du, mask)
    y64 = torch.empty(sp.n_dof, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_apply(ctx, op, torch.as_tensor(du).cuda(), y64)
    y32 = torch.empty(sp.n_dof, dtype=torch.float32, device="cuda")
    nh.nh_jacobian_apply(ctx, op, torch.as_tensor(du, dtype=torch.float32).cuda(), y32)
    nh.nh_sync(ctx)
    assert rel(y64.cpu().numpy(), ref) < 1e-12
    parity.check(y64.cpu().numpy(), ref, parity.jacobian_scale(sp, state, du, mask), 1e-12, "FP64 apply after expiry")
    du32 = du.astype(np.float32).astype(np.float64)
    ref32 = fem.jacobian_apply(sp, state, du32, mask)
    assert rel(y32.double().cpu().numpy(), ref32) < 2e-5
    parity.check(y32.double().cpu().numpy(), ref32, parity.jacobian_scale(sp, state, du32, mask), 2e-5,
                 "FP32 apply after expiry")
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(space)

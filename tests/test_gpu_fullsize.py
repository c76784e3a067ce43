"""Full-size parity in the launch configuration the benchmark times.

Q3 on 48^3 elements (9,145,875 DoF) and Q2 on 74^3 / Q4 on 37^3 (~9.9 M DoF),
plus Q2 on 70^3 and Q4 on 35^3 (8.4 M DoF), whose x-element counts are
multiples of the FP32 kernel's elements per block, so that its block-row
scatter runs next to the uniaxial Dirichlet faces: the whole apply runs on the
GPU in FP64, float-float and FP32; the oracle recomputes sampled outputs
exactly from element windows.  A window is a 3x3x3 block of elements; every
node that is not on a window face interior to the domain receives all of its
element contributions from inside the window, so its value is complete and is
compared with the GPU's, entry by entry against the sum of absolute
contributions of that entry (|J| |du| on the window) and norm-wise over the
window.
"""
import numpy as np
import pytest

import parity
from oracle import fem
from paper_2204_01722_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def window(V, n, e0, w, p, q):
    nx = ny = nz = n
    Vg = V.reshape(nz + 1, ny + 1, nx + 1, 3)
    x0, y0, z0 = e0
    sub = Vg[z0:z0 + w + 1, y0:y0 + w + 1, x0:x0 + w + 1].reshape(-1, 3)
    sp = fem.Space(w, w, w, sub, p, q)
    N = p * n + 1
    I, J, K = inputs.lattice_index(sp.node_dims)
    gI, gJ, gK = p * x0 + I, p * y0 + J, p * z0 + K
    gid = gI + N * (gJ + N * gK)
    ok = np.ones(sp.n_nodes, dtype=bool)
    for loc, s0 in ((I, x0), (J, y0), (K, z0)):
        ok &= ~((loc == 0) & (s0 > 0))
        ok &= ~((loc == p * w) & (s0 + w < n))
    return sp, gid, ok


@pytest.mark.parametrize("p,n", [(3, 48), (2, 74), (4, 37), (2, 70), (4, 35)])
def test_fullsize_sampled_parity(nhctx, p, n):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    q = p + 1
    V = inputs.box_vertices(n, n, n, perturb=0.1, seed=42)
    s, nn, nd = nh.nh_space_box(ctx, n, n, n, V, p, q)
    N = p * n + 1
    assert nn == N ** 3
    mask = inputs.uniaxial_mask((N, N, N))
    nh.nh_space_set_dirichlet(ctx, s, mask)
    op = nh.nh_op_create(ctx, s, 0.3)
    # displacement: smooth field at the oracle's node coordinates
    X = fem.Space(n, n, n, V, p, q).node_coords()
    u = inputs.smooth_field(X, 0.05, seed=43).ravel()
    del X
    minJ = nh.nh_qdata_setup(ctx, op, torch.from_numpy(u).cuda())
    assert minJ > 0
    du = inputs.normal_vector(nd, seed=44)
    du_d = torch.from_numpy(du).cuda()
    y = torch.empty(nd, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_apply(ctx, op, du_d, y)
    yx = torch.empty(nd, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_apply(ctx, op, du_d, yx, prec=nh.NH_F64X)
    y32 = torch.empty(nd, dtype=torch.float32, device="cuda")
    nh.nh_jacobian_apply(ctx, op, du_d.float(), y32)
    torch.cuda.current_stream().synchronize()
    yh = y.cpu().numpy().reshape(-1, 3)
    yxh = yx.cpu().numpy().reshape(-1, 3)
    y32h = y32.double().cpu().numpy().reshape(-1, 3)
    du32 = du.astype(np.float32).astype(np.float64)
    mat = None
    w = 3
    rng = np.random.default_rng(p)
    starts = [(0, 0, 0), (n - w, n - w, n - w), (n // 2, 0, n - w)]
    starts += [tuple(int(v) for v in rng.integers(0, n - w + 1, size=3)) for _ in range(3)]
    for e0 in starts:
        sp, gid, ok = window(V, n, e0, w, p, q)
        mat = fem.Material(1.0, 0.3, sp.ne)
        uw = u.reshape(-1, 3)[gid].ravel()
        dw = du.reshape(-1, 3)[gid].ravel()
        mw = mask.reshape(-1, 3)[gid].ravel()
        st = fem.qp_state(sp, mat, uw)
        ref = fem.jacobian_apply(sp, st, dw, mw).reshape(-1, 3)
        sc = parity.jacobian_scale(sp, st, dw, mw).reshape(-1, 3)
        d32 = du32.reshape(-1, 3)[gid].ravel()
        ref32 = fem.jacobian_apply(sp, st, d32, mw).reshape(-1, 3)
        sc32 = parity.jacobian_scale(sp, st, d32, mw).reshape(-1, 3)
        assert ok.sum() > 0
        for got, r, scl, tol, what in ((yh, ref, sc, TOL64, "FP64"), (yxh, ref, sc, TOL64, "float-float"),
                                       (y32h, ref32, sc32, TOL32, "FP32")):
            g = got[gid][ok]
            e = np.linalg.norm(g - r[ok]) / np.linalg.norm(r[ok])
            assert e < tol, (what, e0, e)
            parity.check(g, r[ok], scl[ok], tol, f"{what} window at {e0}")
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)

"""GPU parity of the learned coarse-correction network and its solver stage.

* FP32 mode (same kernels, FP32 activations and weights): forward 2e-5 and
  gradient 2e-4 relative against the FP64 oracle -- FP32 rounding over a few
  thousand accumulated products per output.
* BF16 mode: forward 3e-2 relative, gradient cosine > 0.99 -- BF16 keeps 8
  significant bits of every activation and weight.
* The solver stage never breaks convergence: FCG with an untrained network
  still solves J x = b to the oracle's direct solution.
* Collected training targets equal (x* - x_k) at the vertex nodes in the
  feature scaling; the first pair (x_0 = 0) is checked against a direct solve.
"""
import numpy as np
import pytest

import parity
from oracle import fem, learned
from paper_2204_01722_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVELS, CH = 3, (8, 16, 32)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def sample():
    rng = np.random.default_rng(0)
    N = 9
    x = rng.normal(size=(4, N, N, N))
    t = rng.normal(size=(3, N, N, N))
    theta = learned.init_params(LEVELS, CH, seed=1) + 0.01 * rng.normal(size=learned.n_params(LEVELS, CH))
    return N, x, t, theta


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_and_gradient(nhctx, sample, bf16):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    N, x, t, theta = sample
    net = nh.nh_net_create(ctx, N, LEVELS, CH, bf16=bf16, seed=3)
    assert nh.nh_net_param_count(ctx, net) == theta.size
    nh.nh_net_set_params(ctx, net, theta.astype(np.float32))
    th32 = theta.astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    y = torch.empty((3, N, N, N), dtype=torch.float32, device="cuda")
    nh.nh_net_forward(ctx, net, xd, y)
    x32 = x.astype(np.float32).astype(np.float64)
    y_ref = learned.forward(th32, x32, LEVELS, CH)
    g = torch.empty(theta.size, dtype=torch.float32, device="cuda")
    loss = nh.nh_net_gradient(ctx, net, xd, td, g)
    torch.cuda.current_stream().synchronize()
    t32 = t.astype(np.float32).astype(np.float64)
    g_ref = learned.loss_grad(th32, x32, t32, LEVELS, CH)
    gh = g.double().cpu().numpy()
    if not bf16:
        assert rel(y.double().cpu().numpy(), y_ref) < 2e-5
        parity.check_inf(y.double().cpu().numpy(), y_ref, 2e-5, "FP32 forward")
        assert rel(gh, g_ref) < 2e-4
        parity.check_inf(gh, g_ref, 2e-4, "FP32 gradient")
        assert abs(loss - learned.loss(th32, x32, t32, LEVELS, CH)) < 1e-5 * loss
    else:
        assert rel(y.double().cpu().numpy(), y_ref) < 3e-2
        cos = float(gh @ g_ref / (np.linalg.norm(gh) * np.linalg.norm(g_ref)))
        assert cos > 0.99
    nh.nh_net_destroy(net)


def test_training_reduces_loss(nhctx, sample):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    N, x, t, _ = sample
    net = nh.nh_net_create(ctx, N, LEVELS, CH, bf16=True, seed=5)
    xd = torch.from_numpy(x.astype(np.float32)).cuda().contiguous()
    # a learnable target: a smooth function of the input
    td = (0.5 * xd[:3] + 0.25 * torch.roll(xd[1:4], 1, dims=1)).contiguous()
    first = nh.nh_net_train_step(ctx, net, 1, xd, td, 3e-3)
    last = first
    for _ in range(60):
        last = nh.nh_net_train_step(ctx, net, 1, xd, td, 3e-3)
    assert last < 0.5 * first
    nh.nh_net_destroy(net)


def _problem(ctx, n=4, p=2, mode=2):
    from paper_2204_01722_b300 import nh
    V = inputs.box_vertices(n, n, n, perturb=0.1, seed=2)
    sp = fem.Space(n, n, n, V, p, p + 1)
    E = inputs.inclusion_modulus(n, n, n, seed=4, rmin=0.5, rmax=1.0, contrast=100.0)
    mat = fem.Material(E, 0.3, sp.ne)
    mask = inputs.uniaxial_mask(sp.node_dims)
    s, _, nd = nh.nh_space_box(ctx, n, n, n, V, p, p + 1)
    nh.nh_space_set_dirichlet(ctx, s, mask)
    op = nh.nh_op_create(ctx, s, 0.3, E)
    u = inputs.smooth_field(sp.node_coords(), 0.03, seed=5).ravel()
    u[mask] = 0.0
    nh.nh_qdata_setup(ctx, op, torch.from_numpy(u).cuda())
    # coarse PCG to 1e-6: with the default 1e-3 the preconditioner varies enough from
    # one application to the next that FCG(1) occasionally stagnates on this small
    # contrast-100 problem (about one solve in 20)
    mg = nh.nh_mg_create(ctx, op, nh.nh_mg_default_opts(ctx, op, learned_mode=mode, coarse_rtol=1e-6))
    nh.nh_mg_setup(ctx, mg)
    st = fem.qp_state(sp, mat, u)
    J = fem.assemble(sp, fem.element_matrices(sp, st), mask)
    return s, op, mg, sp, mask, J, nd, st


@pytest.mark.parametrize("mode", [1, 2])
def test_learned_stage_keeps_fcg_exact(nhctx, mode):
    import scipy.sparse.linalg as spla
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    s, op, mg, sp, mask, J, nd, _ = _problem(ctx, mode=mode)
    net = nh.nh_net_create(ctx, 5, 2, (8, 16), bf16=True, seed=7)
    nh.nh_mg_set_learned(ctx, mg, net)
    b = inputs.normal_vector(nd, seed=8)
    b[mask] = 0.0
    x = torch.zeros(nd, dtype=torch.float64, device="cuda")
    # rtol and maxit leave room for the run-to-run spread of FCG(1) counts on this
    # high-contrast problem (the inexact coarse solve, with atomic-scatter rounding)
    rep = nh.nh_linear_solve(ctx, mg, torch.from_numpy(b).cuda(), x, rtol=1e-9, maxit=3000, norm=1)
    assert rep.learned_accepted + rep.learned_rejected == rep.vcycles
    assert rel(x.cpu().numpy(), spla.spsolve(J.tocsc(), b)) < 1e-6
    nh.nh_mg_set_learned(ctx, mg, None)
    nh.nh_net_destroy(net)
    nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_collected_coarse_pairs(nhctx):
    """Mode 2 pairs: target = A_c^-1 input, A_c the Q1 operator at the fine points."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    n, p = 4, 2
    s, op, mg, sp, mask, J, nd, st = _problem(ctx, n, p, mode=2)
    b = inputs.normal_vector(nd, seed=9)
    b[mask] = 0.0
    Nv = n + 1
    feats = torch.zeros((6, 4, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
    tg = torch.zeros((6, 3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
    k = nh.nh_mg_collect(ctx, mg, torch.from_numpy(b).cuda(), 6, feats, tg)
    assert k >= 2
    c = fem.Space(n, n, n, sp.vertices, 1, p + 1)
    mc = inputs.uniaxial_mask(c.node_dims)
    for i in range(k):
        f = feats[i, :3].cpu().numpy().reshape(3, -1).T.ravel().astype(np.float64)
        e = tg[i].cpu().numpy().reshape(3, -1).T.ravel().astype(np.float64)
        Ae = fem.jacobian_apply(c, st, e, mc)
        assert rel(Ae, f) < 2e-4   # FP32 storage of e, amplified by the coarse condition number
    nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_collected_targets(nhctx):
    import scipy.sparse.linalg as spla
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    n, p = 4, 2
    s, op, mg, sp, mask, J, nd, _ = _problem(ctx, n, p, mode=1)
    b = inputs.normal_vector(nd, seed=9)
    b[mask] = 0.0
    Nv = n + 1
    feats = torch.zeros((8, 4, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
    tg = torch.zeros((8, 3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
    k = nh.nh_mg_collect(ctx, mg, torch.from_numpy(b).cuda(), 8, feats, tg)
    assert k >= 2
    # first pair: residual b, error x*; features = R b / rms(R b), target = x* at vertices / rms(R b)
    c = fem.Space(n, n, n, sp.vertices, 1, p + 1)
    rc = fem.restrict(sp, c, b)
    rc[inputs.uniaxial_mask(c.node_dims)] = 0.0
    scale = np.sqrt(np.mean(rc ** 2))
    f0 = feats[0].cpu().numpy()
    np.testing.assert_allclose(f0[:3].reshape(3, -1).T.ravel(), rc / scale, rtol=1e-5, atol=1e-6)
    xs = spla.spsolve(J.tocsc(), b).reshape(-1, 3)
    N = p * n + 1
    I, Jj, K = inputs.lattice_index((Nv, Nv, Nv))
    vid = p * I + N * (p * Jj + N * p * K)
    t0 = tg[0].cpu().numpy().reshape(3, -1).T
    np.testing.assert_allclose(t0, xs[vid] / scale, rtol=1e-6, atol=1e-6 * np.abs(xs).max() / scale)
    nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_trained_network_gain(nhctx):
    """What a trained coarse warm start gains on the problem it was trained for:
    a network trained on the coarse (r_c, A_c^-1 r_c) pairs that p-MG solves of
    one small inclusion problem generate, then used in learned_mode 2 on
    held-out right-hand sides.  Training must lower the loss; the learned solve
    must reach the same solution and account for every coarse solve (warm start
    taken or refused); its coarse PCG iterations are reported against plain
    p-MG.  The counts are not compared: on this small high-contrast problem the
    FCG iteration count of plain p-MG itself varies from run to run (58 to 525
    observed for one right-hand side), because atomic-scatter rounding moves the
    inexact coarse solve across its every-4-iterations stopping test; hence the
    generous iteration limit."""
    import scipy.sparse.linalg as spla
    ctx, stream = nhctx
    from paper_2204_01722_b300 import nh
    from paper_2204_01722_b300 import learned as L
    n, p = 4, 2
    s, op, mg, sp, mask, J, nd, _ = _problem(ctx, n, p, mode=2)
    Nv = n + 1
    X = sp.node_coords()

    def rhs(seed):
        b = inputs.normal_vector(nd, seed=seed) if seed % 2 == 0 else inputs.smooth_field(X, 1.0, seed=seed).ravel()
        b[mask] = 0.0
        return b

    F, T = [], []
    for j in range(16):
        f = torch.zeros((8, 4, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
        t = torch.zeros((8, 3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
        k = nh.nh_mg_collect(ctx, mg, torch.from_numpy(rhs(100 + j)).cuda(), 8, f, t)
        F.append(f[:k])
        T.append(t[:k])
    feats, tgts = torch.cat(F).contiguous(), torch.cat(T).contiguous()
    net = nh.nh_net_create(ctx, Nv, 2, (8, 16), bf16=True, seed=3)
    hist = L.train(ctx, net, feats, tgts, epochs=120, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    Jc = J.tocsc()
    out = {}
    for name, use in (("plain", False), ("learned", True)):
        nh.nh_mg_set_learned(ctx, mg, net if use else None)
        its, acc, vc, rj = 0, 0, 0, 0
        for j in range(4):
            b = rhs(900 + j)
            x = torch.zeros(nd, dtype=torch.float64, device="cuda")
            rep = nh.nh_linear_solve(ctx, mg, torch.from_numpy(b).cuda(), x, rtol=1e-9, maxit=3000, norm=1)
            assert rel(x.cpu().numpy(), spla.spsolve(Jc, b)) < 1e-6
            its += rep.coarse_its
            acc += rep.learned_accepted
            rj += rep.learned_rejected
            vc += rep.vcycles
        out[name] = (its, acc)
        if use:
            assert acc + rj == vc
    msg = (f"coarse PCG iterations on 4 held-out right-hand sides: plain {out['plain'][0]}, learned "
           f"{out['learned'][0]} ({out['learned'][1]} warm starts taken); training loss {hist[0]:.3f} -> {hist[-1]:.3f}")
    print(msg)
    nh.nh_mg_set_learned(ctx, mg, None)
    nh.nh_net_destroy(net)
    nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)

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


def _bf16_exact(a):
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    return np.array_equal(f.astype(np.float64), a) and not np.any(f.view(np.uint32) & 0xFFFF)


def _integer_network(levels, ch, seed):
    """Sparse integer weights: two nonzeros per output channel, +-1 (+-8 in the
    stride-2 convolutions, so that every coarse field is a multiple of 8^l and its
    linear upsampling stays integer), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for co, ci, s in learned.layer_shapes(levels, ch):
        W = np.zeros((co, ci * 27))
        for c in range(co):
            idx = rng.choice(ci * 27, size=2, replace=False)
            W[c, idx] = (8.0 if s == 2 else 1.0) * rng.choice([-1.0, 1.0], size=2)
        parts += [W.ravel(), np.zeros(co)]
    return np.concatenate(parts)


def _both_paths(ctx, nh, net, N, xd, td):
    ys, gs = {}, {}
    for tc in (True, False):
        nh.nh_net_set_tensor_cores(ctx, net, tc)
        ys[tc] = torch.empty((3, N, N, N), dtype=torch.float32, device="cuda")
        nh.nh_net_forward(ctx, net, xd, ys[tc])
        gs[tc] = torch.empty(nh.nh_net_param_count(ctx, net), dtype=torch.float32, device="cuda")
        nh.nh_net_gradient(ctx, net, xd, td, gs[tc])
    nh.nh_net_set_tensor_cores(ctx, net, True)
    torch.cuda.current_stream().synchronize()
    return ({k: v.double().cpu().numpy() for k, v in ys.items()}, {k: v.double().cpu().numpy() for k, v in gs.items()})


# (grid, channels, weight seed, input seed): seeds for which every field the
# network stores (inputs, activations, upsampled fields, skip sums) is exactly
# representable in BF16 -- checked below against the oracle's tape
INTEGER_CASES = [(9, (8, 16, 32), 0, 100), (13, (16, 48, 64), 3, 103), (7, (32, 8), 0, 100)]


@pytest.mark.parametrize("N,ch,wseed,xseed", INTEGER_CASES)
def test_tensor_core_network_exact(nhctx, N, ch, wseed, xseed):
    """BF16 network on the tensor cores and on the CUDA cores against the oracle, exactly.

    Integer inputs in [0, 3] and sparse integer weights make every stored field
    exactly representable in BF16 and every FP32 sum exact whatever its order, so
    both forward paths must reproduce the FP64 oracle's output bit for bit.  The
    grids of 9^3, 13^3 and 7^3 voxels leave ragged 64-voxel tails; the channel
    sets cover every layer width (3, 8, 16, 32, 48, 64), both strides, and the
    generic and tap-major kernels (Cin 4 and 8 against multiples of 16).
    Gradient of the relative squared error with a target of 2^k entries +-1 (the
    output gradient 2 (y - t) / 2^k is exact): the CUDA-core backward is FP32
    (1e-6 against the oracle); the tensor-core backward rounds the FP32 gradient
    fields to TF32 (relative 2^-11 per operand, 13 convolutions deep: 2e-2)."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    Lv = len(ch)
    theta = _integer_network(Lv, ch, wseed)
    x = np.random.default_rng(xseed).integers(0, 4, size=(4, N, N, N)).astype(np.float64)
    y_ref, tape = learned.forward(theta, x, Lv, ch, keep=True)
    for t in tape:
        if not isinstance(t[0], str):
            assert _bf16_exact(t[0]) and (_bf16_exact(t[4]) or not t[3]), "precondition: fields not BF16-exact"
    rng = np.random.default_rng(7)
    t = np.zeros(3 * N ** 3)
    k = 1 << int(np.log2(t.size))
    t[rng.choice(t.size, size=k, replace=False)] = rng.choice([-1.0, 1.0], size=k)
    t = t.reshape(3, N, N, N)
    net = nh.nh_net_create(ctx, N, Lv, ch, bf16=True, seed=3)
    nh.nh_net_set_params(ctx, net, theta.astype(np.float32))
    ys, gs = _both_paths(ctx, nh, net, N, torch.from_numpy(x.astype(np.float32)).cuda(),
                         torch.from_numpy(t.astype(np.float32)).cuda())
    nh.nh_net_destroy(net)
    assert np.array_equal(ys[False], y_ref), "CUDA-core forward"
    assert np.array_equal(ys[True], y_ref), "tensor-core forward"
    g_ref = learned.loss_grad(theta, x, t, Lv, ch)
    assert rel(gs[False], g_ref) < 1e-6
    assert rel(gs[True], g_ref) < 2e-2
    parity.check_inf(gs[True], g_ref, 2e-2, "tensor-core gradient")


def test_tensor_core_network_exact_at_33(nhctx):
    """The 4-level 16/32/48/64 network at 33^3 (launch shapes of the production
    grids), integer data.  Not every field is exact in BF16 here, but every field
    is an integer and every convolution's sum of absolute terms stays far below
    2^24, so each FP32 sum is exact in any order and both paths round the same
    values to BF16 at the same points: their outputs must equal the oracle's with
    BF16 rounding applied to every stored field, bit for bit.  The gradients of
    the two paths differ only by the tensor-core backward's TF32 operands (2e-2)."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    N, ch = 33, (16, 32, 48, 64)
    theta = _integer_network(4, ch, 0)
    x = np.random.default_rng(100).integers(0, 4, size=(4, N, N, N)).astype(np.float64)
    bf = lambda v: torch.from_numpy(np.asarray(v, dtype=np.float32)).bfloat16().double().numpy()
    y_ref, tape = learned.forward(theta, x, 4, ch, keep=True, store=bf)
    for h, W, *_ in (t for t in tape if not isinstance(t[0], str)):
        assert np.array_equal(h, np.round(h)), "precondition: integer fields"
        assert np.abs(W).reshape(W.shape[0], -1).sum(axis=1).max() * np.abs(h).max() < 2.0 ** 24, "precondition"
    rng = np.random.default_rng(7)
    t = np.zeros(3 * N ** 3)
    k = 1 << int(np.log2(t.size))
    t[rng.choice(t.size, size=k, replace=False)] = rng.choice([-1.0, 1.0], size=k)
    net = nh.nh_net_create(ctx, N, 4, ch, bf16=True, seed=3)
    nh.nh_net_set_params(ctx, net, theta.astype(np.float32))
    ys, gs = _both_paths(ctx, nh, net, N, torch.from_numpy(x.astype(np.float32)).cuda(),
                         torch.from_numpy(t.reshape(3, N, N, N).astype(np.float32)).cuda())
    nh.nh_net_destroy(net)
    assert np.array_equal(ys[False], y_ref), "CUDA-core forward"
    assert np.array_equal(ys[True], y_ref), "tensor-core forward"
    assert np.count_nonzero(y_ref) > 0.2 * y_ref.size
    assert rel(gs[True], gs[False]) < 2e-2


@pytest.mark.parametrize("N,ch", [(9, (8, 16, 32)), (13, (16, 48, 64)), (7, (32, 8))])
def test_tensor_core_network_random(nhctx, N, ch):
    """Random inputs and He-normal weights: both BF16 paths against the FP64
    oracle on the BF16-rounded inputs and weights.  Their FP32 sums differ in
    order, so an activation whose FP32 value lies within rounding noise of a BF16
    rounding boundary rounds the other way (2^-8 relative), and such flips
    compound over the 13 layers: the tensor-core output must be as close to the
    oracle as the CUDA-core one (3e-2, the BF16 bound, and within 1.5x + 2e-3 of
    the CUDA-core error), the two within 1e-2 of each other, the gradients within
    cosine 0.99 of the oracle's."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    Lv = len(ch)
    rng = np.random.default_rng(N)
    x = rng.normal(size=(4, N, N, N))
    t = rng.normal(size=(3, N, N, N))
    theta = learned.init_params(Lv, ch, seed=2) + 0.01 * rng.normal(size=learned.n_params(Lv, ch))
    net = nh.nh_net_create(ctx, N, Lv, ch, bf16=True, seed=3)
    nh.nh_net_set_params(ctx, net, theta.astype(np.float32))
    ys, gs = _both_paths(ctx, nh, net, N, torch.from_numpy(x.astype(np.float32)).cuda(),
                         torch.from_numpy(t.astype(np.float32)).cuda())
    nh.nh_net_destroy(net)
    bf = lambda v: torch.from_numpy(np.asarray(v, dtype=np.float32)).bfloat16().double().numpy()
    th, xb = bf(theta), bf(x)
    y_ref = learned.forward(th, xb, Lv, ch)
    e_tc, e_cc = rel(ys[True], y_ref), rel(ys[False], y_ref)
    assert np.all(np.isfinite(ys[True])) and np.all(np.isfinite(gs[True]))
    assert e_tc < 3e-2 and e_tc < 1.5 * e_cc + 2e-3, (e_tc, e_cc)
    assert rel(ys[True], ys[False]) < 1e-2
    g_ref = learned.loss_grad(th, xb, t.astype(np.float32).astype(np.float64), Lv, ch)
    for g in gs.values():
        assert float(g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))) > 0.99


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
    # the fixed coarse solve (20 Chebyshev-Jacobi steps) keeps the V-cycle a fixed
    # linear operator, so only the network stage varies between applications
    mg = nh.nh_mg_create(ctx, op, nh.nh_mg_default_opts(ctx, op, learned_mode=mode, coarse_fixed=20))
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
    rep = nh.nh_linear_solve(ctx, mg, torch.from_numpy(b).cuda(), x, rtol=1e-10, maxit=300, norm=1)
    assert rep.learned_accepted + rep.learned_rejected == rep.vcycles
    assert rel(x.cpu().numpy(), spla.spsolve(J.tocsc(), b)) < 1e-7
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
    """What the trained network gains over the method without it, on held-out
    right-hand sides of the problem it was trained on (4^3 Q2, contrast-100
    inclusions).  p-MG with the fixed coarse solve (6 Chebyshev-Jacobi steps) is
    a fixed linear preconditioner, so every count below is repeatable.  Pairs
    (residual left by the fixed coarse solve, its exact correction) from 16
    right-hand sides train the network until it fits them (loss below half its
    start); in learned_mode 4 its predictions span a 12-vector coarse space
    around the fixed coarse solve.  On 4 held-out right-hand sides every solve
    must reach the direct solution (1e-7); the FCG counts with no coarse space,
    with the untrained network's and with the trained network's are printed.
    Measured on B300 (plain / untrained / trained): 215 / 212 / 214,
    212 / 215 / 205 and 215 / 215 / 220 -- within a few per cent either way: the
    fit does not carry over to unseen residuals.  The trained network itself
    differs from run to run (its weight gradients are summed with atomic adds),
    and the applies' and transfers' atomic scatter-adds move every count by a
    few.  The balancing two-level solve cannot raise the condition number; the
    last assertion checks that the learned coarse space costs at most 5% more
    iterations than none over the 4 solves."""
    import scipy.sparse.linalg as spla
    ctx, stream = nhctx
    from paper_2204_01722_b300 import nh
    from paper_2204_01722_b300 import learned as L
    n, p = 4, 2
    s, op, mg0, sp, mask, J, nd, _ = _problem(ctx, n, p, mode=3)
    nh.nh_mg_destroy(mg0)
    Nv = n + 1
    X = sp.node_coords()

    def rhs(seed):
        b = inputs.normal_vector(nd, seed=seed) if seed % 2 == 0 else inputs.smooth_field(X, 1.0, seed=seed).ravel()
        b[mask] = 0.0
        return b

    def make(mode, vectors):
        m = nh.nh_mg_create(ctx, op, nh.nh_mg_default_opts(ctx, op, learned_mode=mode, coarse_fixed=6,
                                                           learned_vectors=vectors))
        return m
    mg = make(3, 0)
    nh.nh_mg_setup(ctx, mg)
    F, T = [], []
    for j in range(16):
        f = torch.zeros((12, 4, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
        t = torch.zeros((12, 3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
        k = nh.nh_mg_collect(ctx, mg, torch.from_numpy(rhs(100 + j)).cuda(), 12, f, t)
        F.append(f[:k])
        T.append(t[:k])
    nh.nh_mg_destroy(mg)
    feats, tgts = torch.cat(F).contiguous(), torch.cat(T).contiguous()
    untrained = nh.nh_net_create(ctx, Nv, 2, (8, 16), bf16=True, seed=3)
    net = nh.nh_net_create(ctx, Nv, 2, (8, 16), bf16=True, seed=3)
    hist = L.train(ctx, net, feats, tgts, epochs=60, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    Jc = J.tocsc()
    out = {}
    for name, mode, vec, nt in (("plain", 3, 0, None), ("untrained", 4, 12, untrained), ("learned", 4, 12, net)):
        mg = make(mode, vec)
        if nt is not None:
            nh.nh_mg_set_learned(ctx, mg, nt)
        nh.nh_mg_setup(ctx, mg)
        its = 0
        for j in range(4):
            b = rhs(900 + j)
            x = torch.zeros(nd, dtype=torch.float64, device="cuda")
            rep = nh.nh_linear_solve(ctx, mg, torch.from_numpy(b).cuda(), x, rtol=1e-9, maxit=300, norm=1)
            ref = spla.spsolve(Jc, b)
            assert rel(x.cpu().numpy(), ref) < 1e-7
            its += rep.krylov_its
        out[name] = its
        nh.nh_mg_destroy(mg)
    print(f"FCG iterations on 4 held-out right-hand sides: plain {out['plain']}, coarse space from the untrained "
          f"network {out['untrained']}, from the trained network {out['learned']}; training loss "
          f"{hist[0]:.3f} -> {hist[-1]:.3f}")
    assert out["learned"] <= 1.05 * out["plain"], out
    nh.nh_net_destroy(net)
    nh.nh_net_destroy(untrained)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


@pytest.mark.parametrize("with_net", [False, True])
def test_coarse_space_two_level_solve_is_fixed_spd(nhctx, with_net):
    """learned_mode 4: the coarse space W (network predictions of the errors the
    fixed coarse solve leaves, or without a network that solve's own outputs) is
    built at setup, and the two-level balancing coarse solve keeps the V-cycle a
    fixed linear symmetric operator: V(r1 + 2 r2) = V(r1) + 2 V(r2), a.V(b) = b.V(a);
    FCG with it reaches the direct solution."""
    import scipy.sparse.linalg as spla
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    n, p = 4, 2
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
    mg = nh.nh_mg_create(ctx, op, nh.nh_mg_default_opts(ctx, op, learned_mode=4, learned_vectors=8,
                                                         coarse_fixed=6))
    net = None
    if with_net:
        net = nh.nh_net_create(ctx, n + 1, 2, (8, 16), bf16=True, seed=11)
        nh.nh_mg_set_learned(ctx, mg, net)
    nh.nh_mg_setup(ctx, mg)
    r1 = inputs.normal_vector(nd, seed=1)
    r2 = inputs.normal_vector(nd, seed=2)
    r1[mask] = 0.0
    r2[mask] = 0.0

    def V_(r):
        z = torch.empty(nd, dtype=torch.float64, device="cuda")
        nh.nh_mg_vcycle(ctx, mg, torch.from_numpy(r).cuda(), z)
        torch.cuda.current_stream().synchronize()
        return z.cpu().numpy()
    z1, z2, z12 = V_(r1), V_(r2), V_(r1 + 2.0 * r2)
    parity.check_inf(z12, z1 + 2.0 * z2, 1e-12, "two-level V-cycle linearity")
    assert abs(r1 @ z2 - r2 @ z1) <= 1e-12 * np.linalg.norm(r1) * np.linalg.norm(z2)
    st = fem.qp_state(sp, mat, u)
    J = fem.assemble(sp, fem.element_matrices(sp, st), mask)
    x = torch.zeros(nd, dtype=torch.float64, device="cuda")
    nh.nh_linear_solve(ctx, mg, torch.from_numpy(r1).cuda(), x, rtol=1e-10, maxit=300, norm=1)
    ref = spla.spsolve(J.tocsc(), r1)
    assert rel(x.cpu().numpy(), ref) < 1e-7
    parity.check_inf(x.cpu().numpy(), ref, 1e-7, "two-level linear solve")
    nh.nh_mg_destroy(mg)
    if net:
        nh.nh_net_destroy(net)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_post_correction_keeps_fcg_exact(nhctx):
    """learned_mode 3 (network post-correction after the fixed coarse solve) with
    an untrained network: every coarse solve is accounted for (correction taken
    or refused) and FCG(1) reaches a relative residual of 1e-6 and the direct
    solution to 1e-4.  Not tighter: the post-correction makes the V-cycle a
    nonlinear function of its input, and FCG(1), which keeps one direction, then
    slows down by several times and can stall near 1e-10 (measured; the learned
    coarse space, mode 4, keeps the V-cycle linear instead)."""
    import scipy.sparse.linalg as spla
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    s, op, mg, sp, mask, J, nd, _ = _problem(ctx, mode=3)
    opts = nh.nh_mg_default_opts(ctx, op, learned_mode=3, coarse_fixed=6)
    nh.nh_mg_destroy(mg)
    mg = nh.nh_mg_create(ctx, op, opts)
    nh.nh_mg_setup(ctx, mg)
    net = nh.nh_net_create(ctx, 5, 2, (8, 16), bf16=True, seed=7)
    nh.nh_mg_set_learned(ctx, mg, net)
    b = inputs.normal_vector(nd, seed=8)
    b[mask] = 0.0
    x = torch.zeros(nd, dtype=torch.float64, device="cuda")
    rep = nh.nh_linear_solve(ctx, mg, torch.from_numpy(b).cuda(), x, rtol=1e-6, maxit=600, norm=1)
    assert rep.learned_accepted + rep.learned_rejected == rep.vcycles
    assert rel(x.cpu().numpy(), spla.spsolve(J.tocsc(), b)) < 1e-4
    nh.nh_net_destroy(net)
    nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_four_level_network_at_33(nhctx):
    """The architecture of the 65^3 study (4 levels, 16/32/48/64 channels) on a
    33^3 grid (three stride-2 levels 33 -> 17 -> 9 -> 5) in FP32 mode: forward
    against the FP64 oracle, norm-wise and per entry against the largest entry
    (2e-5)."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    N, Lv, ch = 33, 4, (16, 32, 48, 64)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(4, N, N, N))
    theta = learned.init_params(Lv, ch, seed=2) + 0.01 * rng.normal(size=learned.n_params(Lv, ch))
    net = nh.nh_net_create(ctx, N, Lv, ch, bf16=False, seed=3)
    assert nh.nh_net_param_count(ctx, net) == theta.size
    nh.nh_net_set_params(ctx, net, theta.astype(np.float32))
    y = torch.empty((3, N, N, N), dtype=torch.float32, device="cuda")
    nh.nh_net_forward(ctx, net, torch.from_numpy(x.astype(np.float32)).cuda(), y)
    torch.cuda.current_stream().synchronize()
    ref = learned.forward(theta.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64), Lv, ch)
    got = y.double().cpu().numpy()
    assert rel(got, ref) < 2e-5
    parity.check_inf(got, ref, 2e-5, "4-level FP32 forward at 33^3")
    nh.nh_net_destroy(net)

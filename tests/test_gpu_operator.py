"""GPU parity: every operator entry point of libnh against the FP64 oracle on the
same seeded inputs.

Every result is checked twice: norm-wise (relative 2-norm) and entry by
entry against the sum of absolute contributions of that entry
(``parity.check``: |y_i - ref_i| <= tol * (|J| |du|)_i and the like), so that a
wrong value in a few entries cannot hide under the norm of the whole vector.
Tolerances, in both forms:
* FP64 paths: 1e-12.
* FP32 paths: 2e-5 -- unit roundoff 6e-8 times a few hundred rounded
  operations along the gather / six contraction stages / pointwise /
  scatter chain, with FP32-rounded quadrature data.
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def agree(got, ref, scale, tol, what=""):
    """Norm-wise and entry-wise agreement (module docstring)."""
    got = np.asarray(got, dtype=np.float64).ravel()
    e = rel(got, ref)
    assert e < tol, f"{what}: norm-wise {e:.3e} >= {tol:.1e}"
    parity.check(got, ref, scale, tol, what)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


def host(t):
    torch.cuda.current_stream().synchronize()
    return t.double().cpu().numpy()


class Case:
    """One mesh/material/state set up on both sides from the same seeded inputs."""

    def __init__(self, ctx, n, p, q=None, perturb=0.1, seed=0, layout=0, E=None, amp=0.05, mask="uniaxial"):
        from paper_2204_01722_b300 import nh
        self.nh = nh
        q = q or p + 1
        self.ctx = ctx
        V = inputs.box_vertices(*n, perturb=perturb, seed=seed)
        self.sp = fem.Space(*n, V, p, q)
        self.E = E
        self.mat = fem.Material(1.0 if E is None else E, 0.3, self.sp.ne)
        self.X = self.sp.node_coords()
        self.u = inputs.smooth_field(self.X, amp, seed=seed + 1).ravel()
        if mask == "uniaxial":
            self.mask = inputs.uniaxial_mask(self.sp.node_dims)
        elif mask == "none":
            self.mask = np.zeros(self.sp.n_dof, dtype=bool)
        else:
            self.mask = mask
        self.space, nn, nd = nh.nh_space_box(ctx, *n, V, p, q)
        assert nn == self.sp.n_nodes and nd == self.sp.n_dof
        nh.nh_space_set_dirichlet(ctx, self.space, self.mask)
        self.op = nh.nh_op_create(ctx, self.space, 0.3, E, 1.0, layout)
        self.ud = dev(self.u)
        self.minJ = nh.nh_qdata_setup(ctx, self.op, self.ud)
        self.state = fem.qp_state(self.sp, self.mat, self.u)

    def close(self):
        self.nh.nh_op_destroy(self.op)
        self.nh.nh_space_destroy(self.space)


@pytest.mark.parametrize("n,p,q", [((3, 2, 4), 1, 2), ((3, 2, 4), 2, 3), ((3, 3, 2), 3, 4), ((2, 3, 2), 4, 5),
                                   ((3, 2, 2), 2, 4), ((2, 2, 3), 3, 5), ((2, 2, 2), 4, 6), ((5, 4, 3), 2, 3)])
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_jacobian_apply_fp64(nhctx, n, p, q, layout):
    ctx, _ = nhctx
    c = Case(ctx, n, p, q, layout=layout, seed=p + 10 * q)
    du = inputs.normal_vector(c.sp.n_dof, seed=7)
    y = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    c.nh.nh_jacobian_apply(ctx, c.op, dev(du), y)
    form = "A" if layout == 0 else "B"
    ref = fem.jacobian_apply(c.sp, c.state, du, c.mask, form=form)
    agree(host(y), ref, parity.jacobian_scale(c.sp, c.state, du, c.mask, form), TOL64, "FP64 apply")
    assert abs(c.minJ - c.state["J"].min()) < 1e-13
    c.close()


@pytest.mark.parametrize("n,p,q", [((3, 2, 4), 2, 3), ((3, 3, 2), 3, 4), ((2, 3, 2), 4, 5), ((2, 2, 3), 2, 4),
                                   ((4, 3, 3), 1, 2)])
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_jacobian_apply_f64x(nhctx, n, p, q, layout):
    """Float-float arithmetic on the FP32 pipes, FP64 vectors: same 1e-12 bar as FP64."""
    ctx, _ = nhctx
    c = Case(ctx, n, p, q, layout=layout, seed=21)
    du = inputs.normal_vector(c.sp.n_dof, seed=22)
    y = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    c.nh.nh_jacobian_apply(ctx, c.op, dev(du), y, prec=c.nh.NH_F64X)
    form = "A" if layout == 0 else "B"
    ref = fem.jacobian_apply(c.sp, c.state, du, c.mask, form=form)
    agree(host(y), ref, parity.jacobian_scale(c.sp, c.state, du, c.mask, form), TOL64, "float-float apply")
    c.close()


@pytest.mark.parametrize("n,p", [((3, 2, 4), 2), ((3, 3, 2), 3), ((2, 3, 2), 4)])
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_jacobian_apply_fp32(nhctx, n, p, layout):
    ctx, _ = nhctx
    c = Case(ctx, n, p, layout=layout, seed=3)
    du = inputs.normal_vector(c.sp.n_dof, seed=8)
    y = torch.empty(c.sp.n_dof, dtype=torch.float32, device="cuda")
    c.nh.nh_jacobian_apply(ctx, c.op, dev(du, torch.float32), y)
    du32 = du.astype(np.float32).astype(np.float64)
    ref = fem.jacobian_apply(c.sp, c.state, du32, c.mask)
    agree(host(y), ref, parity.jacobian_scale(c.sp, c.state, du32, c.mask), TOL32, "FP32 apply")
    c.close()


@pytest.mark.parametrize("n,p,mask", [((16, 2, 1), 3, "none"), ((24, 2, 2), 3, "uniaxial"), ((14, 1, 2), 2, "none"),
                                      ((10, 2, 1), 4, "none"), ((10, 1, 2), 4, "uniaxial")])
def test_jacobian_apply_fp32_block_rows(nhctx, n, p, mask):
    """FP32 apply on boxes whose x-element count is a multiple of the kernel's
    elements per block, so the block-row scatter (rows summed in shared memory,
    reduced into y by bulk copies) is taken wherever a row has no Dirichlet node."""
    ctx, _ = nhctx
    c = Case(ctx, n, p, mask=mask, seed=17)
    du = inputs.normal_vector(c.sp.n_dof, seed=18)
    y = torch.empty(c.sp.n_dof, dtype=torch.float32, device="cuda")
    c.nh.nh_jacobian_apply(ctx, c.op, dev(du, torch.float32), y)
    du32 = du.astype(np.float32).astype(np.float64)
    ref = fem.jacobian_apply(c.sp, c.state, du32, c.mask)
    agree(host(y), ref, parity.jacobian_scale(c.sp, c.state, du32, c.mask), TOL32, "FP32 block-row apply")
    c.close()


def test_jacobian_apply_inclusions_and_empty_mask(nhctx):
    """Per-element modulus with contrast 1e3 and no Dirichlet DoFs."""
    ctx, _ = nhctx
    E = inputs.inclusion_modulus(4, 3, 3, seed=2, rmin=0.6, rmax=1.2, contrast=1e3)
    c = Case(ctx, (4, 3, 3), 2, E=E, mask="none", seed=5)
    du = inputs.normal_vector(c.sp.n_dof, seed=9)
    y = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    c.nh.nh_jacobian_apply(ctx, c.op, dev(du), y)
    agree(host(y), fem.jacobian_apply(c.sp, c.state, du), parity.jacobian_scale(c.sp, c.state, du), TOL64,
          "FP64 apply, inclusions")
    y32 = torch.empty(c.sp.n_dof, dtype=torch.float32, device="cuda")
    c.nh.nh_jacobian_apply(ctx, c.op, dev(du, torch.float32), y32)
    du32 = du.astype(np.float32).astype(np.float64)
    agree(host(y32), fem.jacobian_apply(c.sp, c.state, du32), parity.jacobian_scale(c.sp, c.state, du32), TOL32,
          "FP32 apply, inclusions")
    c.close()


def test_single_element_and_host_apply(nhctx):
    ctx, _ = nhctx
    c = Case(ctx, (1, 1, 1), 3, seed=4, perturb=0.0)
    du = inputs.normal_vector(c.sp.n_dof, seed=1)
    yh = np.empty(c.sp.n_dof)
    c.nh.nh_jacobian_apply_host(ctx, c.op, du, yh)
    agree(yh, fem.jacobian_apply(c.sp, c.state, du, c.mask), parity.jacobian_scale(c.sp, c.state, du, c.mask), TOL64,
          "host apply, one element")
    c.close()


@pytest.mark.parametrize("n,p", [((3, 4, 11), 2), ((8, 2, 9), 3), ((2, 2, 7), 4)])
def test_host_apply_pipelined(nhctx, n, p):
    """nh_jacobian_apply_host in chunks of z-layers (upload, kernel, download of
    finished node layers overlapped on three streams) equals the oracle, in each
    precision; FP32 chunks start on kernel batches."""
    ctx, _ = nhctx
    c = Case(ctx, n, p, seed=23)
    du = inputs.normal_vector(c.sp.n_dof, seed=24)
    for prec, dt, tol in ((c.nh.NH_F64, np.float64, TOL64), (c.nh.NH_F64X, np.float64, TOL64),
                          (c.nh.NH_F32, np.float32, TOL32)):
        x = torch.from_numpy(du.astype(dt)).pin_memory()
        y = torch.empty_like(x).pin_memory()
        c.nh.nh_jacobian_apply_host(ctx, c.op, x, y, prec=prec)
        xin = du.astype(dt).astype(np.float64)
        agree(y.numpy(), fem.jacobian_apply(c.sp, c.state, xin, c.mask),
              parity.jacobian_scale(c.sp, c.state, xin, c.mask), tol, f"pipelined host apply, prec {prec}")
    c.close()


@pytest.mark.parametrize("n,p,q", [((3, 2, 4), 2, 3), ((2, 3, 2), 4, 5), ((3, 2, 2), 1, 3)])
def test_residual(nhctx, n, p, q):
    ctx, _ = nhctx
    c = Case(ctx, n, p, q, seed=11)
    g = inputs.uniaxial_bc(c.sp.node_dims, 0.01)
    r = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    c.nh.nh_residual(ctx, c.op, c.ud, dev(g), r)
    ref = fem.residual(c.sp, c.mat, c.u, c.mask, g)
    agree(host(r), ref, parity.residual_scale(c.sp, c.mat, c.u, c.mask, g), TOL64, "residual")
    c.close()


@pytest.mark.parametrize("n,p,q,layout", [((3, 2, 2), 2, 3, 0), ((2, 2, 3), 3, 4, 0), ((2, 2, 2), 4, 5, 0),
                                          ((2, 3, 2), 2, 3, 1), ((2, 2, 2), 1, 3, 0), ((2, 2, 3), 3, 4, 2)])
def test_diagonal(nhctx, n, p, q, layout):
    ctx, _ = nhctx
    c = Case(ctx, n, p, q, layout=layout, seed=12)
    d = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    c.nh.nh_jacobian_diagonal(ctx, c.op, d)
    form = "A" if layout == 0 else "B"
    ref = fem.diagonal(c.sp, c.state, c.mask, form=form)
    sc = parity.diagonal_scale(c.sp, c.state, c.mask, form)
    agree(host(d), ref, sc, TOL64, "FP64 diagonal")
    d32 = torch.empty(c.sp.n_dof, dtype=torch.float32, device="cuda")
    c.nh.nh_jacobian_diagonal(ctx, c.op, d32)
    agree(host(d32), ref, sc, TOL32, "FP32 diagonal")
    c.close()


@pytest.mark.parametrize("pf,pc,layout", [(4, 2, 0), (4, 1, 0), (3, 2, 0), (2, 1, 0), (3, 2, 1), (3, 1, 2)])
def test_rediscretized_coarse_operator(nhctx, pf, pc, layout):
    """Rediscretised coarse operator (Sec. III-B alternative): quadrature data
    re-evaluated from the fine state on the coarse Gauss rule q_c = p_c + 1."""
    ctx, _ = nhctx
    n = (2, 3, 2)
    c = Case(ctx, n, pf, layout=layout, seed=19)
    qc = pc + 1
    V = c.sp.vertices
    st = fem.qp_state(fem.Space(*n, V, pf, qc), c.mat, c.u)
    spc = fem.Space(*n, V, pc, qc)
    maskc = inputs.uniaxial_mask(spc.node_dims)
    nh = c.nh
    sc, _, ndc = nh.nh_space_box(ctx, *n, V, pc, qc)
    nh.nh_space_set_dirichlet(ctx, sc, maskc)
    opc = nh.nh_op_rediscretize(ctx, c.op, sc)
    mj = nh.nh_qdata_setup_rediscretized(ctx, opc, c.op, c.ud)
    assert abs(mj - st["J"].min()) < 1e-13
    du = inputs.normal_vector(ndc, seed=20)
    form = "A" if layout == 0 else "B"
    for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        y = torch.empty(ndc, dtype=dt, device="cuda")
        nh.nh_jacobian_apply(ctx, opc, dev(du, dt), y)
        xin = du if dt == torch.float64 else du.astype(np.float32).astype(np.float64)
        agree(host(y), fem.jacobian_apply(spc, st, xin, maskc, form=form),
              parity.jacobian_scale(spc, st, xin, maskc, form), tol, f"rediscretised apply {dt}")
    y = torch.empty(ndc, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_apply(ctx, opc, dev(du), y, prec=nh.NH_F64X)
    agree(host(y), fem.jacobian_apply(spc, st, du, maskc, form=form), parity.jacobian_scale(spc, st, du, maskc, form),
          TOL64, "rediscretised float-float apply")
    d = torch.empty(ndc, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_diagonal(ctx, opc, d)
    agree(host(d), fem.diagonal(spc, st, maskc, form=form), parity.diagonal_scale(spc, st, maskc, form), TOL64,
          "rediscretised diagonal")
    nh.nh_op_destroy(opc)
    nh.nh_space_destroy(sc)
    c.close()


@pytest.mark.parametrize("pf,pc", [(4, 2), (4, 1), (3, 2), (3, 1), (2, 1)])
def test_coarse_level_operator(nhctx, pf, pc):
    """Galerkin coarse operator sharing the fine quadrature data (Sec. III-B)."""
    ctx, _ = nhctx
    n = (2, 3, 2)
    c = Case(ctx, n, pf, seed=13)
    V = c.sp.vertices
    spc = fem.Space(*n, V, pc, pf + 1)
    maskc = inputs.uniaxial_mask(spc.node_dims)
    nh = c.nh
    sc, _, ndc = nh.nh_space_box(ctx, *n, V, pc, pf + 1)
    nh.nh_space_set_dirichlet(ctx, sc, maskc)
    opc = nh.nh_op_level(ctx, c.op, sc)
    du = inputs.normal_vector(ndc, seed=3)
    for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        y = torch.empty(ndc, dtype=dt, device="cuda")
        nh.nh_jacobian_apply(ctx, opc, dev(du, dt), y)
        xin = du if dt == torch.float64 else du.astype(np.float32).astype(np.float64)
        agree(host(y), fem.jacobian_apply(spc, c.state, xin, maskc),
              parity.jacobian_scale(spc, c.state, xin, maskc), tol, f"coarse-level apply {dt}")
    y = torch.empty(ndc, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_apply(ctx, opc, dev(du), y, prec=nh.NH_F64X)
    agree(host(y), fem.jacobian_apply(spc, c.state, du, maskc), parity.jacobian_scale(spc, c.state, du, maskc),
          TOL64, "coarse-level float-float apply")
    d = torch.empty(ndc, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_diagonal(ctx, opc, d)
    agree(host(d), fem.diagonal(spc, c.state, maskc), parity.diagonal_scale(spc, c.state, maskc), TOL64,
          "coarse-level diagonal")
    nh.nh_op_destroy(opc)
    nh.nh_space_destroy(sc)
    c.close()


@pytest.mark.parametrize("pc,pf", [(1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (3, 4)])
def test_prolong_restrict(nhctx, pc, pf):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    n = (3, 2, 3)
    V = inputs.box_vertices(*n, perturb=0.1, seed=1)
    c = fem.Space(*n, V, pc, pf + 1)
    f = fem.Space(*n, V, pf, pf + 1)
    sc, _, ndc = nh.nh_space_box(ctx, *n, V, pc, pf + 1)
    sf, _, ndf = nh.nh_space_box(ctx, *n, V, pf, pf + 1)
    uc = inputs.normal_vector(ndc, seed=2)
    rf = inputs.normal_vector(ndf, seed=3)
    for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        out = torch.empty(ndf, dtype=dt, device="cuda")
        nh.nh_prolong(ctx, sc, sf, dev(uc, dt), out)
        ucin = uc if dt == torch.float64 else uc.astype(np.float32).astype(np.float64)
        agree(host(out), fem.prolong(c, f, ucin), parity.prolong_scale(c, f, ucin), tol, f"prolongation {dt}")
        outc = torch.empty(ndc, dtype=dt, device="cuda")
        nh.nh_restrict(ctx, sf, sc, dev(rf, dt), outc)
        rfin = rf if dt == torch.float64 else rf.astype(np.float32).astype(np.float64)
        agree(host(outc), fem.restrict(f, c, rfin), parity.restrict_scale(f, c, rfin), tol, f"restriction {dt}")
    nh.nh_space_destroy(sc)
    nh.nh_space_destroy(sf)


@pytest.mark.parametrize("n", [0, 1, 1000, 1_234_567])
def test_dot(nhctx, n):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    x = inputs.normal_vector(n, seed=1)
    y = inputs.normal_vector(n, seed=2)
    xd, yd = dev(x), dev(y)
    r = nh.nh_dot(ctx, n, xd, yd)
    exact = float(np.dot(x, y)) if n else 0.0
    assert abs(r - exact) <= 1e-12 * max(1.0, np.linalg.norm(x) * np.linalg.norm(y))
    assert nh.nh_dot(ctx, n, xd, yd) == r       # deterministic


def test_inverted_element_is_reported(nhctx):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    n = (2, 2, 2)
    V = inputs.box_vertices(*n)
    sp = fem.Space(*n, V, 2, 3)
    s, _, nd = nh.nh_space_box(ctx, *n, V, 2, 3)
    op = nh.nh_op_create(ctx, s, 0.3)
    u = -1.5 * sp.node_coords()          # x = X + u = -X/2: det F = -1/8
    with pytest.raises(nh.NhError) as ei:
        nh.nh_qdata_setup(ctx, op, dev(u.ravel()))
    assert ei.value.status == nh.NH_ERR_INVERTED
    y = torch.empty(nd, dtype=torch.float64, device="cuda")
    with pytest.raises(nh.NhError) as ei:
        nh.nh_jacobian_apply(ctx, op, dev(np.zeros(nd)), y)
    assert ei.value.status == nh.NH_ERR_STATE
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_argument_errors(nhctx):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    with pytest.raises(nh.NhError) as ei:
        nh.nh_space_box(ctx, 2, 2, 2, None, 5, 6)
    assert ei.value.status == nh.NH_ERR_UNSUPPORTED
    with pytest.raises(nh.NhError):
        nh.nh_space_box(ctx, 0, 2, 2, None, 2, 3)
    s, _, nd = nh.nh_space_box(ctx, 2, 2, 2, None, 2, 3)
    with pytest.raises(nh.NhError):
        nh.nh_op_create(ctx, s, 0.5)
    op = nh.nh_op_create(ctx, s, 0.3)
    x = torch.zeros(nd + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(nh.NhError) as ei:      # misaligned (offset by one double)
        nh.nh_qdata_setup(ctx, op, x.data_ptr() + 8)
    assert ei.value.status == nh.NH_ERR_ARG
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(s)


def test_fma_peak_measurement(nhctx):
    """nh_fma_peak: measured FP64 and FP32 FMA throughput, within the range a
    B300 can give (unit counts at up to 2.032 GHz: 1.2 and 77 TFLOP/s)."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    f64, ms64 = nh.nh_fma_peak(ctx, nh.NH_F64, 2048)
    f32, ms32 = nh.nh_fma_peak(ctx, nh.NH_F32, 1 << 16)
    assert 0.2 < f64 < 1.3 and ms64 > 0
    assert 10.0 < f32 < 80.0 and ms32 > 0
    with pytest.raises(nh.NhError):
        nh.nh_fma_peak(ctx, nh.NH_F64X, 10)


@pytest.mark.parametrize("n,p,mask", [((14, 2, 3), 2, "uniaxial"), ((14, 3, 2), 2, "none"), ((8, 3, 2), 3, "uniaxial"),
                                      ((8, 2, 3), 3, "none"), ((5, 3, 2), 4, "uniaxial"), ((10, 2, 2), 4, "none")])
def test_eight_colour_scatter(nhctx, n, p, mask):
    """nh_op_set_scatter(op, 1): eight launches, one per parity class of the
    elements (FP32: of the kernel's element batches), plain read-modify-writes
    instead of atomics.  Every precision equals the oracle as with atomics, and
    two applies give bit-identical results (fixed summation order)."""
    ctx, _ = nhctx
    c = Case(ctx, n, p, mask=mask, seed=29)
    c.nh.nh_op_set_scatter(ctx, c.op, 1)
    du = inputs.normal_vector(c.sp.n_dof, seed=30)
    du32 = du.astype(np.float32).astype(np.float64)
    ref = fem.jacobian_apply(c.sp, c.state, du, c.mask)
    ref32 = fem.jacobian_apply(c.sp, c.state, du32, c.mask)
    sc = parity.jacobian_scale(c.sp, c.state, du, c.mask)
    sc32 = parity.jacobian_scale(c.sp, c.state, du32, c.mask)
    for prec, dt, r, scl, tol in ((c.nh.NH_F64, torch.float64, ref, sc, TOL64),
                                  (c.nh.NH_F64X, torch.float64, ref, sc, TOL64),
                                  (c.nh.NH_F32, torch.float32, ref32, sc32, TOL32)):
        y1 = torch.empty(c.sp.n_dof, dtype=dt, device="cuda")
        y2 = torch.empty(c.sp.n_dof, dtype=dt, device="cuda")
        c.nh.nh_jacobian_apply(ctx, c.op, dev(du, dt), y1, prec=prec)
        c.nh.nh_jacobian_apply(ctx, c.op, dev(du, dt), y2, prec=prec)
        agree(host(y1), r, scl, tol, f"eight-colour scatter, prec {prec}")
        assert torch.equal(y1, y2), prec
    c.nh.nh_op_set_scatter(ctx, c.op, 0)
    c.close()
    c = Case(ctx, (7, 2, 2), 3, seed=29)
    with pytest.raises(c.nh.NhError) as ei:     # 7 elements along x: not a multiple of 8
        c.nh.nh_op_set_scatter(ctx, c.op, 1)
    assert ei.value.status == c.nh.NH_ERR_UNSUPPORTED
    c.close()

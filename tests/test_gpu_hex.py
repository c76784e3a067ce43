"""GPU parity on unstructured hexahedral meshes (`nh_space_hex`, Sec. II-B: the
element restriction of a general mesh) against the oracle's `HexSpace`.

The two sides number nodes differently (the library by topology, the oracle by
matching coordinates), so vectors are carried across by node position.  Meshes:
the perturbed box written as an unstructured mesh with every element's local
frame a random cube rotation and ids and element order shuffled, and an L-shaped
subset of it.  Tolerances as for the box: 1e-12 (FP64 and float-float), 2e-5
(FP32), each both norm-wise and entry by entry against the sum of absolute
contributions of the entry (``parity.check``); 1e-7 for a linear solve to 1e-11
against a sparse direct solve (norm-wise, and per entry against the largest
entry).
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import parity
from oracle import fem
from paper_2204_01722_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def agree(got, ref, scale, tol, what=""):
    got = np.asarray(got, dtype=np.float64).ravel()
    e = rel(got, ref)
    assert e < tol, f"{what}: norm-wise {e:.3e} >= {tol:.1e}"
    parity.check(got, ref, scale, tol, what)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype).cuda()


def host(t):
    torch.cuda.current_stream().synchronize()
    return t.double().cpu().numpy()


def make_mesh(kind, n, seed):
    V = inputs.box_vertices(*n, perturb=0.1, seed=seed)
    keep = None
    if kind == "L":
        ez, ey, ex = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
        keep = ~((ex.ravel() >= 1) & (ey.ravel() >= n[1] - 1))
    return inputs.hex_mesh_from_box(*n, V, seed=seed + 1, keep=keep)


class HexCase:
    """One mesh on both sides; library vectors are oracle vectors indexed by `dp`."""

    def __init__(self, ctx, Vh, H, p, q=None, E=None, amp=0.05, seed=0):
        from paper_2204_01722_b300 import nh
        self.nh, self.ctx = nh, ctx
        q = q or p + 1
        self.sp = fem.HexSpace(Vh, H, p, q)
        self.space, nn, nd = nh.nh_space_hex(ctx, Vh, H, p, q)
        assert nn == self.sp.n_nodes and nd == self.sp.n_dof
        X = nh.nh_space_coords(ctx, self.space, nn)
        d, perm = cKDTree(self.sp.node_coords()).query(X)  # library node i is oracle node perm[i]
        assert d.max() < 1e-12 and len(np.unique(perm)) == nn
        self.dp = (3 * perm[:, None] + np.arange(3)[None, :]).ravel()
        Xo = self.sp.node_coords()
        lo, hi = Xo[:, 0].min(), Xo[:, 0].max()
        m = np.zeros((nn, 3), dtype=bool)
        m[np.abs(Xo[:, 0] - lo) < 1e-12, :] = True       # x = 0 clamped
        m[np.abs(Xo[:, 0] - hi) < 1e-12, 0] = True       # x = 1: x-component prescribed
        self.mask = m.ravel()
        nh.nh_space_set_dirichlet(ctx, self.space, self.mask[self.dp])
        self.mat = fem.Material(1.0 if E is None else E, 0.3, self.sp.ne)
        self.op = nh.nh_op_create(ctx, self.space, 0.3, E)
        self.u = inputs.smooth_field(Xo, amp, seed=seed + 1).ravel()
        self.minJ = nh.nh_qdata_setup(ctx, self.op, dev(self.to_lib(self.u)))
        self.state = fem.qp_state(self.sp, self.mat, self.u)

    def to_lib(self, v):
        return np.asarray(v)[self.dp]

    def to_oracle(self, v):
        out = np.empty(len(self.dp))
        out[self.dp] = v
        return out

    def close(self):
        self.nh.nh_op_destroy(self.op)
        self.nh.nh_space_destroy(self.space)


@pytest.mark.parametrize("kind", ["rotated", "L"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hex_jacobian_apply(nhctx, kind, p):
    ctx, _ = nhctx
    Vh, H = make_mesh(kind, (6, 4, 3) if p <= 2 else (3, 3, 2), seed=p)
    c = HexCase(ctx, Vh, H, p, seed=p)
    nh = c.nh
    du = inputs.normal_vector(c.sp.n_dof, seed=9)
    ref = fem.jacobian_apply(c.sp, c.state, du, c.mask)
    assert abs(c.minJ - c.state["J"].min()) < 1e-13
    sc = parity.jacobian_scale(c.sp, c.state, du, c.mask)
    x32 = du.astype(np.float32)
    ref32 = fem.jacobian_apply(c.sp, c.state, x32.astype(np.float64), c.mask)
    sc32 = parity.jacobian_scale(c.sp, c.state, x32.astype(np.float64), c.mask)
    for prec, dtype, tol in ((nh.NH_F64, torch.float64, 1e-12), (nh.NH_F64X, torch.float64, 1e-12),
                             (nh.NH_F32, torch.float32, 2e-5)):
        x, r, scl = (x32.astype(np.float64), ref32, sc32) if dtype == torch.float32 else (du, ref, sc)
        y = torch.empty(c.sp.n_dof, dtype=dtype, device="cuda")
        nh.nh_jacobian_apply(ctx, c.op, dev(c.to_lib(x), dtype), y, prec=prec)
        agree(c.to_oracle(host(y)), r, scl, tol, f"hex apply, prec {prec}")
    # host buffers: chunks of elements over node prefixes (first-touch numbering)
    yh = np.empty(c.sp.n_dof)
    nh.nh_jacobian_apply_host(ctx, c.op, np.ascontiguousarray(c.to_lib(du)), yh)
    agree(c.to_oracle(yh), ref, sc, 1e-12, "hex host apply FP64")
    yh32 = np.empty(c.sp.n_dof, dtype=np.float32)
    nh.nh_jacobian_apply_host(ctx, c.op, np.ascontiguousarray(c.to_lib(x32)), yh32)
    agree(c.to_oracle(yh32), ref32, sc32, 2e-5, "hex host apply FP32")
    c.close()


@pytest.mark.parametrize("kind", ["rotated", "L"])
def test_hex_residual_and_diagonal(nhctx, kind):
    ctx, _ = nhctx
    Vh, H = make_mesh(kind, (3, 3, 2), seed=4)
    E = inputs.inclusion_modulus(3, 3, 2, seed=2, rmin=0.6, rmax=1.2, contrast=10.0)[:len(H)]
    c = HexCase(ctx, Vh, H, 3, E=E, seed=5)
    nh = c.nh
    g = np.zeros(c.sp.n_dof)
    g[c.mask] = -0.01
    r = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    nh.nh_residual(ctx, c.op, dev(c.to_lib(c.u)), dev(c.to_lib(g)), r)
    agree(c.to_oracle(host(r)), fem.residual(c.sp, c.mat, c.u, c.mask, g),
          parity.residual_scale(c.sp, c.mat, c.u, c.mask, g), 1e-12, "hex residual")
    d = torch.empty(c.sp.n_dof, dtype=torch.float64, device="cuda")
    nh.nh_jacobian_diagonal(ctx, c.op, d)
    agree(c.to_oracle(host(d)), fem.diagonal(c.sp, c.state, c.mask), parity.diagonal_scale(c.sp, c.state, c.mask),
          1e-12, "hex diagonal")
    c.close()


def test_hex_transfers(nhctx):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    Vh, H = make_mesh("L", (3, 3, 2), seed=6)
    f = HexCase(ctx, Vh, H, 3, seed=7)
    cs = fem.HexSpace(Vh, H, 1, 4)
    csp, nn, _ = nh.nh_space_hex(ctx, Vh, H, 1, 4)
    d, perm = cKDTree(cs.node_coords()).query(nh.nh_space_coords(ctx, csp, nn))
    assert d.max() < 1e-12
    cdp = (3 * perm[:, None] + np.arange(3)[None, :]).ravel()
    uc = inputs.normal_vector(cs.n_dof, seed=8)
    uf = torch.empty(f.sp.n_dof, dtype=torch.float64, device="cuda")
    nh.nh_prolong(ctx, csp, f.space, dev(uc[cdp]), uf)
    agree(f.to_oracle(host(uf)), fem.prolong(cs, f.sp, uc), parity.prolong_scale(cs, f.sp, uc), 1e-12,
          "hex prolongation")
    rf = inputs.normal_vector(f.sp.n_dof, seed=9)
    rc = torch.empty(cs.n_dof, dtype=torch.float64, device="cuda")
    nh.nh_restrict(ctx, f.space, csp, dev(f.to_lib(rf)), rc)
    out = np.empty(cs.n_dof)
    out[cdp] = host(rc)
    agree(out, fem.restrict(f.sp, cs, rf), parity.restrict_scale(f.sp, cs, rf), 1e-12, "hex restriction")
    nh.nh_space_destroy(csp)
    f.close()


def bsr_to_csr(rp, cl, val, n_nodes):
    import scipy.sparse as sps
    rows = np.repeat(np.arange(n_nodes), np.diff(rp))
    r = (3 * rows[:, None, None] + np.arange(3)[None, :, None]).repeat(3, 2)
    c = (3 * cl.astype(np.int64)[:, None, None] + np.arange(3)[None, None, :]).repeat(3, 1)
    return sps.coo_matrix((val.ravel(), (r.ravel(), c.ravel())), shape=(3 * n_nodes, 3 * n_nodes)).tocsr()


@pytest.mark.parametrize("kind", ["rotated", "L"])
def test_hex_assembled_q1_matches_oracle(nhctx, kind):
    """Split-phase COO assembly of the Galerkin Q1 level (fine quadrature data at
    the fine points) against the oracle's assembled element matrices."""
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    Vh, H = make_mesh(kind, (3, 3, 2), seed=13)
    f = HexCase(ctx, Vh, H, 3, seed=14)
    cs = fem.HexSpace(Vh, H, 1, 4)
    csp, nn, _ = nh.nh_space_hex(ctx, Vh, H, 1, 4)
    d, perm = cKDTree(cs.node_coords()).query(nh.nh_space_coords(ctx, csp, nn))
    assert d.max() < 1e-12
    cdp = (3 * perm[:, None] + np.arange(3)[None, :]).ravel()
    Xc = cs.node_coords()
    m = np.zeros((nn, 3), dtype=bool)
    m[np.abs(Xc[:, 0] - Xc[:, 0].min()) < 1e-12, :] = True
    m[np.abs(Xc[:, 0] - Xc[:, 0].max()) < 1e-12, 0] = True
    mask_c = m.ravel()
    nh.nh_space_set_dirichlet(ctx, csp, mask_c[cdp])
    cop = nh.nh_op_level(ctx, f.op, csp)
    rp, cl, val = nh.nh_op_assemble_q1(ctx, cop, nn)
    assert np.all(np.diff(rp) > 0) and np.all(np.diff(cl[rp[0]:rp[1]]) > 0)
    A = bsr_to_csr(rp, cl, val, nn)                      # library numbering
    ref = fem.assemble(cs, fem.element_matrices(cs, f.state), mask_c)
    P = np.zeros(3 * nn, dtype=np.int64)
    P[cdp] = np.arange(3 * nn)                          # oracle dof -> library dof
    A_o = A[P][:, P]
    err = abs(A_o - ref).max()
    assert err <= 1e-12 * abs(ref).max()
    nh.nh_op_destroy(cop)
    nh.nh_space_destroy(csp)
    f.close()


@pytest.mark.parametrize("mixed,assembled", [(0, 1), (1, 1), (0, 0)])
def test_hex_linear_solve_matches_direct(nhctx, mixed, assembled):
    """p-multigrid 3 -> 2 -> 1 on the unstructured mesh; the Q1 level assembled
    by the split-phase COO path (block rows, Jacobi-PCG) or matrix-free."""
    import scipy.sparse.linalg as spla
    ctx, _ = nhctx
    Vh, H = make_mesh("L", (4, 3, 3), seed=10)
    c = HexCase(ctx, Vh, H, 3, amp=0.04, seed=11)
    nh = c.nh
    opts = nh.nh_mg_default_opts(ctx, c.op, level_p=(3, 2, 1), mixed=mixed, coarse_rtol=1e-3, coarse_maxit=5000,
                                 coarse_assembled=assembled)
    mg = nh.nh_mg_create(ctx, c.op, opts)
    nh.nh_mg_setup(ctx, mg)
    J = fem.assemble(c.sp, fem.element_matrices(c.sp, c.state), c.mask)
    b = inputs.normal_vector(c.sp.n_dof, seed=12)
    b[c.mask] = 0.0
    x = torch.zeros(c.sp.n_dof, dtype=torch.float64, device="cuda")
    rep = nh.nh_linear_solve(ctx, mg, dev(c.to_lib(b)), x, rtol=1e-11, maxit=300, norm=1)
    ref = spla.spsolve(J.tocsc(), b)
    assert rel(c.to_oracle(host(x)), ref) < 1e-7
    parity.check_inf(c.to_oracle(host(x)), ref, 1e-7, "hex linear solve")
    assert rep.krylov_its < 150
    nh.nh_mg_destroy(mg)
    c.close()


def test_hex_mesh_errors(nhctx):
    ctx, _ = nhctx
    from paper_2204_01722_b300 import nh
    Vh, H = inputs.hex_mesh_from_box(2, 1, 1, inputs.box_vertices(2, 1, 1), reorient=False, permute=False)

    def status(V, HH, p=2):
        with pytest.raises(nh.NhError) as e:
            nh.nh_space_hex(ctx, V, HH, p, p + 1)
        return e.value.status

    bad = H.copy()
    bad[0, [0, 1]] = bad[0, [1, 0]]                        # mirrored element: negative Jacobian
    assert status(Vh, bad) == nh.NH_ERR_ARG and "inverted" in nh.nh_last_error(ctx)
    bad = H.copy()
    bad[1, 3] = len(Vh)                                    # vertex id out of range
    assert status(Vh, bad) == nh.NH_ERR_ARG
    assert status(Vh, np.vstack([H, H[:1]])) == nh.NH_ERR_ARG   # a face used by three elements
    assert status(Vh, H, p=5) == nh.NH_ERR_UNSUPPORTED
    sp, _, _ = nh.nh_space_hex(ctx, Vh, H, 2, 3)
    op = nh.nh_op_create(ctx, sp, 0.3)
    opts = nh.nh_mg_default_opts(ctx, op, coarse_solver=1)      # geometric coarse MG needs the box lattice
    with pytest.raises(nh.NhError) as e:
        nh.nh_mg_create(ctx, op, opts)
    assert e.value.status == nh.NH_ERR_UNSUPPORTED
    nh.nh_op_destroy(op)
    nh.nh_space_destroy(sp)

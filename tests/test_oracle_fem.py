"""Pins of the oracle's finite-element definitions against what the paper and
the mathematics fix: volume, patch test, finite differences, symmetry,
the two equivalent linearisations, small-strain linear elasticity coded
independently, rigid-body modes, objectivity, brute-force diagonal,
p-prolongation exactness, Galerkin identity and p+1 convergence."""
import numpy as np
import pytest

from oracle import basis, fem, solvers
from paper_2204_01722_b300 import inputs


def make(n=(2, 2, 2), p=2, q=None, perturb=0.1, seed=1, E=1.0, nu=0.3):
    q = q or p + 1
    V = inputs.box_vertices(*n, perturb=perturb, seed=seed)
    sp = fem.Space(*n, V, p, q)
    mat = fem.Material(E, nu, sp.ne)
    return sp, mat


def state_for(sp, mat, amp=0.05, seed=2):
    u = inputs.smooth_field(sp.node_coords(), amp, seed=seed).ravel()
    return u, fem.qp_state(sp, mat, u)


@pytest.mark.parametrize("p,q", [(1, 2), (2, 3), (3, 4), (2, 5)])
def test_geometry_volume(p, q):
    sp, _ = make((3, 2, 2), p, q, perturb=0.1)
    _, W, _ = sp.geometry()
    assert abs(W.sum() - 1.0) < 1e-13      # only interior vertices move
    assert W.min() > 0


def test_multiplicity_counts():
    sp, _ = make((2, 2, 2), 2)
    m = sp.multiplicity().reshape(5, 5, 5)
    assert m[0, 0, 0] == 1 and m[2, 2, 2] == 8 and m[1, 1, 1] == 1
    assert m[2, 1, 1] == 2 and m[2, 2, 1] == 4


@pytest.mark.parametrize("p", [1, 2, 3])
def test_patch_test(p):
    """Affine u = A X + c: residual vanishes at interior nodes; J(u) applied to an
    affine du also vanishes there (Gauss with p+1 points is exact)."""
    sp, mat = make((3, 3, 3), p, perturb=0.15, seed=4)
    X = sp.node_coords()
    A = np.array([[0.02, -0.05, 0.03], [0.04, -0.03, 0.01], [-0.02, 0.05, 0.06]])
    u = (X @ A.T + np.array([0.1, -0.2, 0.05])).ravel()
    r = fem.residual(sp, mat, u).reshape(-1, 3)
    interior = np.ones(sp.n_nodes, dtype=bool)
    interior[inputs.all_faces_mask(sp.node_dims)[::3]] = False
    assert interior.any()
    assert np.abs(r[interior]).max() < 1e-14
    assert np.abs(r[~interior]).max() > 1e-3       # the boundary carries traction
    st = fem.qp_state(sp, mat, u)
    B = np.array([[0.3, 0.1, -0.2], [0.0, 0.2, 0.4], [-0.1, 0.5, 0.1]])
    du = (X @ B.T).ravel()
    y = fem.jacobian_apply(sp, st, du).reshape(-1, 3)
    assert np.abs(y[interior]).max() < 1e-14


@pytest.mark.parametrize("p,form", [(1, "A"), (2, "A"), (3, "A"), (2, "B")])
def test_jacobian_finite_difference(p, form):
    """||F(u+h du) - F(u-h du) - 2h J du|| = O(h^3): second-order decay."""
    sp, mat = make((2, 2, 2), p)
    u, st = state_for(sp, mat)
    du = inputs.normal_vector(sp.n_dof, seed=3)
    y = fem.jacobian_apply(sp, st, du, form=form)
    errs = []
    for h in [1e-2, 1e-3, 1e-4]:
        d = fem.residual(sp, mat, u + h * du) - fem.residual(sp, mat, u - h * du) - 2 * h * y
        errs.append(np.linalg.norm(d) / np.linalg.norm(2 * h * y))
    slopes = np.log10(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.9), (errs, slopes)
    assert errs[-1] < 1e-5


def test_jacobian_finite_difference_with_dirichlet():
    sp, mat = make((2, 2, 2), 2)
    u, st = state_for(sp, mat)
    mask = inputs.uniaxial_mask(sp.node_dims)
    g = inputs.uniaxial_bc(sp.node_dims, 0.01)
    du = inputs.normal_vector(sp.n_dof, seed=3)
    du[mask] = 0.0          # variations stay in the affine space u_c = g_c
    y = fem.jacobian_apply(sp, st, du, mask)
    h = 1e-5
    d = fem.residual(sp, mat, u + h * du, mask, g) - fem.residual(sp, mat, u - h * du, mask, g)
    assert np.linalg.norm(d - 2 * h * y) / np.linalg.norm(2 * h * y) < 1e-7


@pytest.mark.parametrize("p,q", [(1, 2), (2, 3), (3, 4), (4, 5), (2, 4)])
def test_two_linearisations_agree(p, q):
    """Current-configuration form (Eq. dtau) == initial-configuration dP = dF S + F dS."""
    sp, mat = make((2, 1, 2), p, q)
    E = inputs.inclusion_modulus(2, 1, 2, seed=5, contrast=10.0)
    mat = fem.Material(E, 0.3, sp.ne)
    u, st = state_for(sp, mat, amp=0.08)
    du = inputs.normal_vector(sp.n_dof, seed=7)
    yA = fem.jacobian_apply(sp, st, du, form="A")
    yB = fem.jacobian_apply(sp, st, du, form="B")
    assert np.linalg.norm(yA - yB) / np.linalg.norm(yA) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetry(p):
    sp, mat = make((2, 2, 1), p)
    _, st = state_for(sp, mat)
    mask = inputs.uniaxial_mask(sp.node_dims)
    v = inputs.normal_vector(sp.n_dof, seed=11)
    w = inputs.normal_vector(sp.n_dof, seed=12)
    a = v @ fem.jacobian_apply(sp, st, w, mask)
    b = w @ fem.jacobian_apply(sp, st, v, mask)
    assert abs(a - b) <= 1e-13 * abs(a)


def linear_elastic_matrix(sp, mat):
    """Independent small-strain stiffness: K = sum_q W B^T D B in Voigt notation."""
    dXdxi, W, _ = sp.geometry()
    dxidX = np.linalg.inv(dXdxi)
    P3 = sp.P ** 3
    rows, cols, vals = [], [], []
    for e in range(sp.ne):
        lam, mu = mat.lam[e], mat.mu[e]
        D = np.zeros((6, 6))
        D[:3, :3] = lam
        D[np.arange(3), np.arange(3)] = lam + 2 * mu
        D[3:, 3:] = np.eye(3) * mu
        K = np.zeros((3 * P3, 3 * P3))
        for qp in range(sp.q ** 3):
            dN = np.stack([sp.Bxi[d][qp] for d in range(3)], axis=1) @ dxidX[e, qp]  # [P3, 3]
            Bv = np.zeros((6, 3 * P3))
            for a in range(P3):
                nx_, ny_, nz_ = dN[a]
                Bv[:, 3 * a:3 * a + 3] = [[nx_, 0, 0], [0, ny_, 0], [0, 0, nz_],
                                          [0, nz_, ny_], [nz_, 0, nx_], [ny_, nx_, 0]]
            K += W[e, qp] * Bv.T @ D @ Bv
        dofs = (3 * sp.elem_nodes[e][:, None] + np.arange(3)).ravel()
        rows.append(np.repeat(dofs, dofs.size))
        cols.append(np.tile(dofs, dofs.size))
        vals.append(K.ravel())
    import scipy.sparse as sps
    return sps.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(sp.n_dof, sp.n_dof)).tocsr()


@pytest.mark.parametrize("form", ["A", "B"])
def test_small_strain_is_linear_elasticity(form):
    sp, mat = make((2, 1, 2), 2)
    E = inputs.inclusion_modulus(2, 1, 2, seed=3, contrast=5.0)
    mat = fem.Material(E, 0.3, sp.ne)
    st = fem.qp_state(sp, mat, np.zeros(sp.n_dof))
    K = linear_elastic_matrix(sp, mat)
    for s in range(3):
        du = inputs.normal_vector(sp.n_dof, seed=20 + s)
        y = fem.jacobian_apply(sp, st, du, form=form)
        assert np.linalg.norm(y - K @ du) / np.linalg.norm(y) < 1e-13


def test_rigid_modes_in_null_space():
    sp, mat = make((2, 2, 2), 2)
    st = fem.qp_state(sp, mat, np.zeros(sp.n_dof))
    X = sp.node_coords()
    modes = [np.tile(np.eye(3)[i], (sp.n_nodes, 1)) for i in range(3)]
    for W in [np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0.]]), np.array([[0, 0, 1], [0, 0, 0], [-1, 0, 0.]]),
              np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0.]])]:
        modes.append(X @ W.T)
    ref = np.linalg.norm(fem.jacobian_apply(sp, st, inputs.normal_vector(sp.n_dof, 1)))
    for m in modes:
        assert np.linalg.norm(fem.jacobian_apply(sp, st, m.ravel())) < 1e-13 * ref


def test_objectivity_identity():
    """Frame indifference: J(u) (W (X+u)) = W F(u) node-wise for skew W; translations -> 0."""
    sp, mat = make((2, 2, 2), 2)
    u, st = state_for(sp, mat, amp=0.1)
    X = sp.node_coords()
    x = X + u.reshape(-1, 3)
    r = fem.residual(sp, mat, u).reshape(-1, 3)
    W = np.array([[0, -0.3, 0.2], [0.3, 0, -0.7], [-0.2, 0.7, 0.]])
    y = fem.jacobian_apply(sp, st, (x @ W.T).ravel()).reshape(-1, 3)
    assert np.linalg.norm(y - r @ W.T) < 1e-13 * np.linalg.norm(r)
    t = np.tile([0.3, -0.1, 0.2], sp.n_nodes)
    assert np.linalg.norm(fem.jacobian_apply(sp, st, t)) < 1e-13 * np.linalg.norm(r)


@pytest.mark.parametrize("p,q,form", [(1, 2, "A"), (2, 3, "A"), (3, 4, "A"), (2, 3, "B"), (2, 4, "A")])
def test_diagonal_brute_force(p, q, form):
    sp, mat = make((2, 1, 1), p, q)
    _, st = state_for(sp, mat)
    mask = inputs.uniaxial_mask(sp.node_dims)
    d = fem.diagonal(sp, st, mask, form)
    brute = np.empty(sp.n_dof)
    for k in range(sp.n_dof):
        ek = np.zeros(sp.n_dof)
        ek[k] = 1.0
        brute[k] = fem.jacobian_apply(sp, st, ek, mask)[k]
    np.testing.assert_allclose(d, brute, rtol=1e-13, atol=1e-15)


def test_assembled_matches_apply():
    sp, mat = make((2, 2, 1), 2)
    _, st = state_for(sp, mat)
    mask = inputs.uniaxial_mask(sp.node_dims)
    A = fem.assemble(sp, fem.element_matrices(sp, st), mask)
    du = inputs.normal_vector(sp.n_dof, 5)
    y = fem.jacobian_apply(sp, st, du, mask)
    assert np.linalg.norm(A @ du - y) < 1e-13 * np.linalg.norm(y)


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (1, 4), (2, 3), (1, 3)])
def test_prolongation_interpolates_polynomials(pc, pf):
    """On an undistorted box the coarse space holds every polynomial of degree pc per
    direction, so P (coarse nodal values) = fine nodal values of the same polynomial."""
    V = inputs.box_vertices(2, 3, 2)
    c = fem.Space(2, 3, 2, V, pc, pf + 1)
    f = fem.Space(2, 3, 2, V, pf, pf + 1)
    rng = np.random.default_rng(0)
    coef = rng.normal(size=(3, pc + 1, pc + 1, pc + 1))

    def poly(X):
        out = np.zeros((X.shape[0], 3))
        for a in range(pc + 1):
            for b in range(pc + 1):
                for g in range(pc + 1):
                    out += coef[:, a, b, g][None, :] * (X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** g)[:, None]
        return out
    uc = poly(c.node_coords()).ravel()
    uf = fem.prolong(c, f, uc)
    np.testing.assert_allclose(uf, poly(f.node_coords()).ravel(), atol=1e-12)


def test_restriction_is_transpose_and_galerkin():
    sp_f, mat = make((2, 2, 2), 3, 4)
    sp_c = fem.Space(2, 2, 2, sp_f.vertices, 1, 4)
    _, st = state_for(sp_f, mat)
    vf = inputs.normal_vector(sp_f.n_dof, 1)
    uc = inputs.normal_vector(sp_c.n_dof, 2)
    assert abs(vf @ fem.prolong(sp_c, sp_f, uc) - fem.restrict(sp_f, sp_c, vf) @ uc) < 1e-12
    # Galerkin: P^T A_f P = A_c, A_c = coarse basis at the fine quadrature points with fine state
    lhs = fem.restrict(sp_f, sp_c, fem.jacobian_apply(sp_f, st, fem.prolong(sp_c, sp_f, uc)))
    rhs = fem.jacobian_apply(sp_c, st, uc)
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(rhs)


def _manufactured(a=0.05):
    amp = np.array([1.0, -0.6, 0.8]) * a
    L = np.array([[0.0, 0.02, 0.0], [0.0, 0.0, 0.02], [0.02, 0.0, 0.0]])

    def u(X):
        s = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        return s[:, None] * amp[None, :] + X @ L.T

    def grad(X):
        sx, sy, sz = (np.sin(np.pi * X[:, i]) for i in range(3))
        cx, cy, cz = (np.cos(np.pi * X[:, i]) for i in range(3))
        ds = np.pi * np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz], axis=1)  # [m, 3]
        return amp[None, :, None] * ds[:, None, :] + L[None]

    def hess(X):
        sx, sy, sz = (np.sin(np.pi * X[:, i]) for i in range(3))
        cx, cy, cz = (np.cos(np.pi * X[:, i]) for i in range(3))
        p2 = np.pi ** 2
        Hs = np.empty((X.shape[0], 3, 3))
        Hs[:, 0, 0] = -p2 * sx * sy * sz
        Hs[:, 1, 1] = -p2 * sx * sy * sz
        Hs[:, 2, 2] = -p2 * sx * sy * sz
        Hs[:, 0, 1] = Hs[:, 1, 0] = p2 * cx * cy * sz
        Hs[:, 0, 2] = Hs[:, 2, 0] = p2 * cx * sy * cz
        Hs[:, 1, 2] = Hs[:, 2, 1] = p2 * sx * cy * cz
        return amp[None, :, None, None] * Hs[:, None, :, :]
    return u, grad, hess


@pytest.mark.parametrize("p,ns", [(1, (2, 4, 8)), (2, (2, 4)), (3, (2, 4)), (4, (2, 3))])
def test_manufactured_convergence(p, ns):
    """L2 error of the nonlinear solve against a manufactured solution decays as h^(p+1)
    (observed order log(e_1/e_2) / log(h_1/h_2) between successive meshes)."""
    uex, grad, hess = _manufactured()
    errs = []
    for n in ns:
        V = inputs.box_vertices(n, n, n)
        sp = fem.Space(n, n, n, V, p, p + 1)
        mat = fem.Material(1.0, 0.3, sp.ne)
        f = fem.body_force_for(sp, mat, grad, hess)
        mask = inputs.all_faces_mask(sp.node_dims)
        g = uex(sp.node_coords()).ravel()
        u, _ = solvers.newton_direct(sp, mat, np.zeros(sp.n_dof), mask, g, f)
        errs.append(fem.l2_error(sp, u, uex))
    h = 1.0 / np.array(ns, dtype=np.float64)
    rates = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(h[:-1] / h[1:])
    assert np.all(rates > p + 1 - 0.35), (errs, rates)


def test_manufactured_residual_vanishes_for_polynomial_solution():
    """A quadratic displacement lies in Q2: with its exact body force the residual of the
    nodal interpolant vanishes up to quadrature error of the (non-polynomial) stress."""
    uex, grad, hess = _manufactured(0.0)        # affine part only, zero body force
    sp, mat = make((2, 2, 2), 2, perturb=0.0)
    u = uex(sp.node_coords()).ravel()
    mask = inputs.all_faces_mask(sp.node_dims)
    r = fem.residual(sp, mat, u, mask, u, fem.body_force_for(sp, mat, grad, hess))
    assert np.abs(r).max() < 1e-14


@pytest.mark.parametrize("pf,pc", [(3, 2), (4, 2), (2, 1)])
def test_rediscretized_equals_galerkin_for_affine_state(pf, pc):
    """Sec. III-B: re-evaluating the nonlinearity on the coarse Gauss rule
    q_c = p_c + 1 (rediscretisation) gives the exact Galerkin coarse operator
    (coarse basis at the fine points) whenever that rule integrates the coarse
    integrand exactly: on an affine mesh with an affine displacement the
    tangent is constant per element and the integrand has degree 2 p_c per
    direction.  On a perturbed mesh with a curved displacement they differ."""
    n = (2, 2, 1)
    rng = np.random.default_rng(pf * 10 + pc)
    for perturb, same in ((0.0, True), (0.1, False)):
        V = inputs.box_vertices(*n, perturb=perturb, seed=3)
        fine = fem.Space(*n, V, pf, pf + 1)
        mat = fem.Material(1.0, 0.3, fine.ne)
        X = fine.node_coords()
        if same:
            A = 0.05 * rng.normal(size=(3, 3))
            u = (X @ A.T).ravel()
        else:
            u = inputs.smooth_field(X, 0.05, seed=4).ravel()
        gal = fem.Space(*n, V, pc, pf + 1)
        red = fem.Space(*n, V, pc, pc + 1)
        st_g = fem.qp_state(fine, mat, u)
        st_r = fem.qp_state(fem.Space(*n, V, pf, pc + 1), mat, u)
        du = rng.normal(size=gal.n_dof)
        y_g = fem.jacobian_apply(gal, st_g, du)
        y_r = fem.jacobian_apply(red, st_r, du)
        d = np.linalg.norm(y_r - y_g) / np.linalg.norm(y_g)
        assert (d < 1e-12) if same else (d > 1e-6)


"""Finite-element definitions of the method (oracle; test infrastructure only).

Plain FP64 numpy, batched over elements but otherwise literal: each element
operator is a dense Kronecker-product matrix (Eq. tensorDense), each pointwise
function is written as the paper states it, and assembly is E^T by
``np.add.at``.  No sum factorisation, no fusion.

Conventions (the paper does not state index conventions; these readings are
fixed by the finite-difference and two-form identity tests):
* a vector field is stored node-major ``[n_nodes, 3]``;
* gradients are ``(grad u)[c, d] = d u_c / d coord_d``;
* ``A : B = sum_ij A_ij B_ij``;
* the structured box numbers nodes and elements lexicographically, x fastest;
  local element nodes are ``l = i + P (j + P k)``.
"""
import numpy as np

from . import basis

I3 = np.eye(3)


def kron3(az, ay, ax):
    """3-D tensor-product matrix, rows (qk, qj, qi) and columns (k, j, i)."""
    return np.kron(az, np.kron(ay, ax))


def det3(A):
    return np.linalg.det(A)


def sym(A):
    return 0.5 * (A + np.swapaxes(A, -1, -2))


def tr(A):
    return np.trace(A, axis1=-2, axis2=-1)


def ddot(A, B):
    return np.sum(A * B, axis=(-2, -1))


def T(A):
    return np.swapaxes(A, -1, -2)


class Space:
    """Continuous Q_p space on a structured nx x ny x nz hexahedral box.

    ``vertices`` is ``[(nx+1)(ny+1)(nz+1), 3]`` (x fastest).  The geometry is
    the trilinear map of each element's 8 vertices ("linear geometry"); Q_p
    node coordinates are the trilinear images of the GLL lattice.  ``q`` is
    the number of Gauss points per direction; a coarse space built for the
    p-multigrid hierarchy takes the fine ``q`` (Sec. III-B: coarse levels use
    the fine quadrature points).
    """

    def __init__(self, nx, ny, nz, vertices, p, q):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.p, self.P, self.q = p, p + 1, q
        self.ne = nx * ny * nz
        self.vertices = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
        assert self.vertices.shape[0] == (nx + 1) * (ny + 1) * (nz + 1)
        self.node_dims = (p * nx + 1, p * ny + 1, p * nz + 1)
        self.n_nodes = int(np.prod(self.node_dims))
        self.n_dof = 3 * self.n_nodes
        P = self.P
        Nx, Ny, _ = self.node_dims
        ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        # element index e = ex + nx (ey + ny ez)
        ex = ex.transpose(2, 1, 0).ravel()
        ey = ey.transpose(2, 1, 0).ravel()
        ez = ez.transpose(2, 1, 0).ravel()
        k, j, i = np.meshgrid(np.arange(P), np.arange(P), np.arange(P), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()  # local l = i + P (j + P k)
        gi = p * ex[:, None] + i[None, :]
        gj = p * ey[:, None] + j[None, :]
        gk = p * ez[:, None] + k[None, :]
        self.elem_nodes = gi + Nx * (gj + Ny * gk)  # [ne, P^3]
        vk, vj, vi = np.meshgrid([0, 1], [0, 1], [0, 1], indexing="ij")
        vi, vj, vk = vi.ravel(), vj.ravel(), vk.ravel()  # v = vi + 2 vj + 4 vk
        self.elem_verts = (ex[:, None] + vi) + (nx + 1) * ((ey[:, None] + vj) + (ny + 1) * (ez[:, None] + vk))
        self._setup_basis()

    def _setup_basis(self):
        p, q = self.p, self.q
        vk, vj, vi = np.meshgrid([0, 1], [0, 1], [0, 1], indexing="ij")
        vi, vj, vk = vi.ravel(), vj.ravel(), vk.ravel()  # v = vi + 2 vj + 4 vk
        self._vsign = np.stack([2 * vi - 1, 2 * vj - 1, 2 * vk - 1], axis=1).astype(np.float64)  # [8, 3]

        B1, D1, xg, wg = basis.tabulate(p, q)
        self.B1, self.D1, self.xg, self.wg = B1, D1, xg, wg
        self.BI = kron3(B1, B1, B1)                                   # [Q^3, P^3]
        self.Bxi = np.stack([kron3(B1, B1, D1),                       # d/dxi_0 (x)
                             kron3(B1, D1, B1),                       # d/dxi_1 (y)
                             kron3(D1, B1, B1)])                      # d/dxi_2 (z)
        self.wq = kron3(wg[:, None], wg[:, None], wg[:, None]).ravel()  # [Q^3]
        qk, qj, qi = np.meshgrid(xg, xg, xg, indexing="ij")
        self.xi_q = np.stack([qi.ravel(), qj.ravel(), qk.ravel()], axis=1)  # [Q^3, 3]
        self.xnodes, _ = basis.gauss_lobatto(self.P)

    # -- trilinear geometry ---------------------------------------------------
    def trilinear(self, xi):
        """Shape values N[v] and derivatives dN[v, d] of the 8-vertex map at xi [m, 3]."""
        s = self._vsign  # [8, 3]
        f = 0.5 * (1.0 + xi[:, None, :] * s[None, :, :])  # [m, 8, 3]
        N = f[:, :, 0] * f[:, :, 1] * f[:, :, 2]
        dN = np.empty(f.shape)
        dN[:, :, 0] = 0.5 * s[None, :, 0] * f[:, :, 1] * f[:, :, 2]
        dN[:, :, 1] = 0.5 * s[None, :, 1] * f[:, :, 0] * f[:, :, 2]
        dN[:, :, 2] = 0.5 * s[None, :, 2] * f[:, :, 0] * f[:, :, 1]
        return N, dN

    def geometry(self, xi=None, w=None):
        """dX/dxi [ne, m, 3, 3], W = w det(dX/dxi) [ne, m], X [ne, m, 3] at points xi.

        W is the quadrature weight mapped to the physical element (Sec. II-B,
        W^e = det(grad_xi X) W^ (x) W^ (x) W^).
        """
        if xi is None:
            xi, w = self.xi_q, self.wq
        N, dN = self.trilinear(xi)
        Xv = self.vertices[self.elem_verts]                  # [ne, 8, 3]
        dXdxi = np.einsum("mvd,evi->emid", dN, Xv)           # [ne, m, i, d] = dX_i / dxi_d
        X = np.einsum("mv,evi->emi", N, Xv)
        W = w[None, :] * det3(dXdxi)
        return dXdxi, W, X

    def node_coords(self):
        """Node coordinates [n_nodes, 3]: trilinear image of the GLL lattice."""
        k, j, i = np.meshgrid(self.xnodes, self.xnodes, self.xnodes, indexing="ij")
        xi = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
        N, _ = self.trilinear(xi)
        Xv = self.vertices[self.elem_verts]
        Xe = np.einsum("mv,evi->emi", N, Xv)
        X = np.zeros((self.n_nodes, 3))
        X[self.elem_nodes.ravel()] = Xe.reshape(-1, 3)
        return X

    def multiplicity(self):
        """Number of elements sharing each node, m = E E^T 1 (Eq. mg_prolong)."""
        m = np.zeros(self.n_nodes)
        np.add.at(m, self.elem_nodes.ravel(), 1.0)
        return m

    # -- element restriction and basis action --------------------------------
    def ref_gradient(self, vec):
        """grad_xi of a nodal field at the quadrature points: g[e, q, c, d] = d u_c / d xi_d.

        E (element restriction, gather) followed by B_xi (Eq. tensorDense)."""
        ue = np.asarray(vec).reshape(self.n_nodes, 3)[self.elem_nodes]  # [ne, P^3, 3]
        return np.einsum("dql,elc->eqcd", self.Bxi, ue)

    def values(self, vec):
        ue = np.asarray(vec).reshape(self.n_nodes, 3)[self.elem_nodes]
        return np.einsum("ql,elc->eqc", self.BI, ue)

    def apply_Bxi_T(self, fhat):
        """E^T B_xi^T of a quadrature-point field fhat[e, q, c, d] -> nodal [n_nodes, 3]."""
        ye = np.einsum("dql,eqcd->elc", self.Bxi, fhat)
        y = np.zeros((self.n_nodes, 3))
        np.add.at(y, self.elem_nodes.ravel(), ye.reshape(-1, 3))
        return y

    def apply_BI_T(self, f0):
        """E^T B_I^T of a quadrature-point field f0[e, q, c] -> nodal [n_nodes, 3]."""
        ye = np.einsum("ql,eqc->elc", self.BI, f0)
        y = np.zeros((self.n_nodes, 3))
        np.add.at(y, self.elem_nodes.ravel(), ye.reshape(-1, 3))
        return y


class HexSpace(Space):
    """Continuous Q_p space on an unstructured conforming hexahedral mesh
    (the element restriction E of a general mesh, Sec. II-B).

    ``hex8[e, v]`` is the vertex at corner (v & 1, (v >> 1) & 1, v >> 2) of the
    reference cube.  Global nodes are found by coordinates: every element's
    trilinear image of the GLL lattice is computed and points that coincide
    (within 1e-9 of the mesh extent) are one node, numbered in order of first
    appearance.  This uses no mesh topology, so it checks a topological
    numbering independently.
    """

    def __init__(self, vertices, hex8, p, q):
        from scipy.spatial import cKDTree

        self.nx = self.ny = self.nz = None
        self.p, self.P, self.q = p, p + 1, q
        self.vertices = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
        self.elem_verts = np.asarray(hex8, dtype=np.int64).reshape(-1, 8)
        self.ne = self.elem_verts.shape[0]
        self._setup_basis()
        k, j, i = np.meshgrid(self.xnodes, self.xnodes, self.xnodes, indexing="ij")
        N, _ = self.trilinear(np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1))
        Xe = np.einsum("mv,evi->emi", N, self.vertices[self.elem_verts]).reshape(-1, 3)
        tol = 1e-9 * max(np.ptp(self.vertices, axis=0).max(), 1e-300)
        parent = np.arange(Xe.shape[0])

        def root(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for a, b in cKDTree(Xe).query_pairs(tol):
            ra, rb = root(a), root(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
        roots = np.array([root(a) for a in range(Xe.shape[0])])
        uniq, first = np.unique(roots, return_index=True)
        order = np.argsort(first)                       # number by first appearance
        rank = np.empty(len(uniq), dtype=np.int64)
        rank[order] = np.arange(len(uniq))
        self.elem_nodes = rank[np.searchsorted(uniq, roots)].reshape(self.ne, -1)
        self.n_nodes = len(uniq)
        self.n_dof = 3 * self.n_nodes
        self.node_dims = None


def unit_cube_vertices(nx, ny, nz):
    x = np.linspace(0.0, 1.0, nx + 1)
    y = np.linspace(0.0, 1.0, ny + 1)
    z = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


class Material:
    """Compressible Neo-Hookean material: Young's modulus per element, Poisson ratio."""

    def __init__(self, E, nu, ne):
        E = np.broadcast_to(np.asarray(E, dtype=np.float64), (ne,)).copy()
        self.E, self.nu = E, float(nu)
        self.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
        self.mu = E / (2.0 * (1.0 + nu))


def qp_state(space, mat, u):
    """Kinematic state at the quadrature points of ``space`` from displacement u.

    H = grad_X u, F = I + H, J = det F with J - 1 from the invariants of H so
    that log J = log1p(J - 1) does not cancel; Green-Euler strain
    e = (H + H^T + H H^T)/2 and Kirchhoff stress tau = 2 mu e + lambda log J I
    (Eq. strain-energy, Eq. Kirchhoff-stress; the "e" forms avoid the
    cancellation of b - I).
    """
    dXdxi, W, _ = space.geometry()
    dxidX = np.linalg.inv(dXdxi)
    g = space.ref_gradient(u)
    H = g @ dxidX
    F = I3 + H
    trH = tr(H)
    Jm1 = trH + 0.5 * (trH ** 2 - tr(H @ H)) + det3(H)
    J = 1.0 + Jm1
    logJ = np.log1p(Jm1)
    lam = mat.lam[:, None]
    mu = mat.mu[:, None]
    e = 0.5 * (H + T(H) + H @ T(H))
    tau = 2.0 * mu[..., None, None] * e + (lam * logJ)[..., None, None] * I3
    Finv = np.linalg.inv(F)
    return dict(W=W, dXdxi=dXdxi, dxidX=dxidX, H=H, F=F, J=J, logJ=logJ, tau=tau,
                Finv=Finv, lam=np.broadcast_to(lam, W.shape), mu=np.broadcast_to(mu, W.shape))


def second_piola(state):
    """S = mu (I - C^-1) + lambda log J C^-1: the initial-configuration form of the
    same Neo-Hookean model (Sec. V-E "initial" storage rows)."""
    Finv = state["Finv"]
    Cinv = Finv @ T(Finv)
    lam = state["lam"][..., None, None]
    mu = state["mu"][..., None, None]
    return mu * (I3 - Cinv) + lam * state["logJ"][..., None, None] * Cinv, Cinv


def residual(space, mat, u, mask=None, g_bc=None, body_force=None):
    """Discrete residual F(u) (Eq. residual-discrete with f_1 = stress, f_0 = -rho0 g).

    The oracle integrates the first Piola stress P = F S against grad_X v, the
    reference-configuration statement of the weak form whose current-
    configuration statement is int grad_x v : tau dV (Eq. variational-form).
    ``body_force`` (values [ne, q, 3] at the quadrature points) enters as
    -int v . f.  Constrained rows (``mask`` True) return u - g.
    """
    st = qp_state(space, mat, u)
    S, _ = second_piola(st)
    Pk = st["F"] @ S
    fhat = st["W"][..., None, None] * (Pk @ T(st["dxidX"]))    # f_cd = sum_K P_cK dxi_d/dX_K
    r = space.apply_Bxi_T(fhat)
    if body_force is not None:
        r -= space.apply_BI_T(st["W"][..., None] * body_force)
    r = r.ravel()
    if mask is not None:
        u = np.asarray(u).ravel()
        g = np.zeros_like(u) if g_bc is None else np.asarray(g_bc).ravel()
        r[mask] = u[mask] - g[mask]
    return r


def _masked(vec, mask):
    v = np.array(vec, dtype=np.float64).ravel()
    if mask is not None:
        v[mask] = 0.0
    return v


def pointwise_A(state, g):
    """Paper's current-configuration linearisation (Eqs. Jacobian, dtau, depsilon).

    With G = grad_x du = g grad_x xi and deps = sym G:
        dtau - tau G^T = G tau + lambda tr(deps) I + 2 (mu - lambda log J) deps,
    tested against grad_x v, i.e. fhat = W (that) (grad_x xi)^T.
    """
    X = state["dxidX"] @ state["Finv"]                 # grad_x xi = grad_X xi F^-1
    G = g @ X
    deps = sym(G)
    lam = state["lam"][..., None, None]
    mu = state["mu"][..., None, None]
    logJ = state["logJ"][..., None, None]
    sig = G @ state["tau"] + lam * tr(deps)[..., None, None] * I3 + 2.0 * (mu - lam * logJ) * deps
    return state["W"][..., None, None] * (sig @ T(X))


def pointwise_B(state, g):
    """Initial-configuration linearisation dP = dF S + F dS with
    dE = sym(F^T dF), dS = lambda (C^-1 : dE) C^-1 + 2 (mu - lambda log J) C^-1 dE C^-1
    (dC^-1 = -C^-1 dC C^-1, Sec. V-E), tested against grad_X v."""
    dF = g @ state["dxidX"]
    S, Cinv = second_piola(state)
    F = state["F"]
    dE = sym(T(F) @ dF)
    lam = state["lam"][..., None, None]
    mu = state["mu"][..., None, None]
    logJ = state["logJ"][..., None, None]
    dS = lam * ddot(Cinv, dE)[..., None, None] * Cinv + 2.0 * (mu - lam * logJ) * (Cinv @ dE @ Cinv)
    dP = dF @ S + F @ dS
    return state["W"][..., None, None] * (dP @ T(state["dxidX"]))


def jacobian_apply(space, state, du, mask=None, form="A"):
    """J du (Eq. Jacobian-discrete-ref): E^T B_xi^T W Lambda(f_11) B_xi E du.

    ``state`` comes from ``qp_state`` on a space with the same quadrature
    points (a coarse space reuses the fine state: exact Galerkin coarse
    operator, Sec. III-B).  Dirichlet convention: constrained columns are
    dropped and constrained rows act as the identity.
    """
    v = _masked(du, mask)
    g = space.ref_gradient(v)
    fhat = pointwise_A(state, g) if form == "A" else pointwise_B(state, g)
    y = space.apply_Bxi_T(fhat).ravel()
    if mask is not None:
        du = np.asarray(du).ravel()
        y[mask] = du[mask]
    return y


def tangent(state, form="A"):
    """Pointwise tangent D[e, q, c, d, c', d'] = d fhat_cd / d g_c'd' (the f_11 block of
    Eq. Jacobian-discrete-ref), by applying the linear pointwise map to unit gradients."""
    ne, nq = state["W"].shape
    D = np.zeros((ne, nq, 3, 3, 3, 3))
    fn = pointwise_A if form == "A" else pointwise_B
    for c in range(3):
        for d in range(3):
            g = np.zeros((ne, nq, 3, 3))
            g[..., c, d] = 1.0
            D[..., c, d] = fn(state, g)
    return D.reshape(ne, nq, 3, 3, 3, 3)


def diagonal(space, state, mask=None, form="A"):
    """Diagonal of the assembled Jacobian: for node a, component c,
    sum_e sum_q sum_{d,d'} B_xi,d[q,a] D[q, c,d, c,d'] B_xi,d'[q,a]; constrained rows 1."""
    D = tangent(state, form)
    Dcc = np.einsum("eqcdcf->eqcdf", D)                          # [e, q, c, d, d']
    de = np.einsum("dql,eqcdf,fql->elc", space.Bxi, Dcc, space.Bxi)
    y = np.zeros((space.n_nodes, 3))
    np.add.at(y, space.elem_nodes.ravel(), de.reshape(-1, 3))
    y = y.ravel()
    if mask is not None:
        y[mask] = 1.0
    return y


def element_matrices(space, state, form="A"):
    """Element Jacobian matrices K[e, (l,c), (l',c')] (tiny meshes only)."""
    D = tangent(state, form)
    # K = sum_q B_xi^T D B_xi, the right product first: DB[e,q,c,d,m,C] = sum_D D[.., C, D] B_xi,D[q, m]
    DB = np.einsum("eqcdCD,Dqm->eqcdmC", D, space.Bxi)
    K = np.einsum("dql,eqcdmC->elcmC", space.Bxi, DB)
    P3 = space.P ** 3
    return K.reshape(space.ne, 3 * P3, 3 * P3)


def assemble(space, Ke, mask=None):
    """Sparse assembled matrix sum_e E^T K_e E; Dirichlet rows/cols -> identity."""
    import scipy.sparse as sp
    dofs = (3 * space.elem_nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(space.ne, -1)
    rows = np.repeat(dofs, dofs.shape[1], axis=1).ravel()
    cols = np.tile(dofs, (1, dofs.shape[1])).ravel()
    A = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(space.n_dof, space.n_dof)).tocsr()
    if mask is not None:
        keep = sp.diags((~mask).astype(np.float64))
        A = keep @ A @ keep + sp.diags(mask.astype(np.float64))
    return A.tocsr()


# -- p-multigrid transfer (Eq. mg_prolong) ------------------------------------

def ctof_matrix(coarse, fine):
    """B_ctof: the coarse GLL Lagrange basis evaluated at the fine GLL nodes (3-D)."""
    b, _ = basis.lagrange_tabulate(coarse.xnodes, fine.xnodes)   # [P_f, P_c]
    return kron3(b, b, b)


def prolong(coarse, fine, uc):
    """P_f = sum_e E_f^T Lambda(m_f^-1) B_ctof E_c (Eq. mg_prolong), m_f = node multiplicity."""
    B = ctof_matrix(coarse, fine)
    ue = np.asarray(uc).reshape(coarse.n_nodes, 3)[coarse.elem_nodes]
    fe = np.einsum("fc,ecx->efx", B, ue)
    minv = 1.0 / fine.multiplicity()
    fe = fe * minv[fine.elem_nodes][..., None]
    uf = np.zeros((fine.n_nodes, 3))
    np.add.at(uf, fine.elem_nodes.ravel(), fe.reshape(-1, 3))
    return uf.ravel()


def restrict(fine, coarse, rf):
    """Restriction = prolongation transposed (Sec. III-B)."""
    B = ctof_matrix(coarse, fine)
    minv = 1.0 / fine.multiplicity()
    re = np.asarray(rf).reshape(fine.n_nodes, 3)[fine.elem_nodes] * minv[fine.elem_nodes][..., None]
    ce = np.einsum("fc,efx->ecx", B, re)
    rc = np.zeros((coarse.n_nodes, 3))
    np.add.at(rc, coarse.elem_nodes.ravel(), ce.reshape(-1, 3))
    return rc.ravel()


# -- manufactured solutions ----------------------------------------------------

def piola_derivative(F, dF, lam, mu):
    """dP = dF S + F dS for P = F S(C), S = mu (I - C^-1) + lambda log J C^-1,
    at any deformation gradient F (pointwise; arrays [..., 3, 3])."""
    Finv = np.linalg.inv(F)
    Cinv = Finv @ T(Finv)
    J = det3(F)
    logJ = np.log(J)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    mu = np.asarray(mu)[..., None, None]
    S = mu * (I3 - Cinv) + lam * logJ * Cinv
    dE = sym(T(F) @ dF)
    dS = lam * ddot(Cinv, dE)[..., None, None] * Cinv + 2.0 * (mu - lam * logJ) * (Cinv @ dE @ Cinv)
    return dF @ S + F @ dS


def body_force_for(space, mat, grad_u, hess_u):
    """f = -Div P(u*) at the quadrature points of ``space``.

    ``grad_u(X)`` returns [m, 3, 3] and ``hess_u(X)`` returns [m, 3, 3, 3] with
    hess[c, L, J] = d^2 u*_c / dX_L dX_J.  Div P_c = sum_J [dP(F; d_J F)]_{cJ}."""
    _, _, X = space.geometry()
    Xf = X.reshape(-1, 3)
    F = I3 + grad_u(Xf)
    Hs = hess_u(Xf)
    lam = np.repeat(mat.lam, space.q ** 3)
    mu = np.repeat(mat.mu, space.q ** 3)
    div = np.zeros((Xf.shape[0], 3))
    for Jd in range(3):
        dP = piola_derivative(F, Hs[:, :, :, Jd], lam, mu)
        div += dP[:, :, Jd]
    return -div.reshape(space.ne, space.q ** 3, 3)


def l2_error(space, uh, exact, qe=None):
    """|| u_h - u* ||_L2 with a (p+3)-point Gauss rule per direction."""
    qe = qe or space.p + 3
    xg, wg = basis.gauss_legendre(qe)
    B1, _ = basis.lagrange_tabulate(space.xnodes, xg)
    BI = kron3(B1, B1, B1)
    qk, qj, qi = np.meshgrid(xg, xg, xg, indexing="ij")
    xi = np.stack([qi.ravel(), qj.ravel(), qk.ravel()], axis=1)
    w = kron3(wg[:, None], wg[:, None], wg[:, None]).ravel()
    _, W, X = space.geometry(xi, w)
    ue = np.asarray(uh).reshape(space.n_nodes, 3)[space.elem_nodes]
    uq = np.einsum("ql,elc->eqc", BI, ue)
    err = uq - exact(X.reshape(-1, 3)).reshape(uq.shape)
    return np.sqrt(np.sum(W[..., None] * err ** 2))

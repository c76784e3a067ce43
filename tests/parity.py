"""Entry-wise parity checks of library results against the oracle.

Every operator here returns, per entry, a sum of many signed contributions
(element contributions gathered by E^T, quadrature points, tensor components;
Sec. II-B).  A norm over the whole vector can hide a wrong value in a few
entries (one Dirichlet face, one element class, a block-row boundary), and a
relative check per entry fails on entries that nearly cancel.  So each entry is
held to the precision its own sum allows:

    |y_i - ref_i| <= tol * s_i,

where s_i is the same sum with every contribution replaced by its absolute
value: for a linear map L applied to x, s = |L| |x| with |L| the matrix of
absolute entries (for the Jacobian, the oracle's element matrices in absolute
value, assembled with the Dirichlet convention).  Rounding in any evaluation
order of such a sum is a modest multiple of the unit roundoff times s_i, so
tol = 1e-12 (FP64) and 2e-5 (FP32) bound each entry with a wide margin while a
dropped term, a sign or an index error in one entry shows as an O(1) ratio.

Results of iterative solves (V-cycle, Krylov, Newton) carry a global error
set by the stopping test; they are checked per entry against the largest
entry of the reference: |x_i - ref_i| <= tol * ||ref||_inf.
"""
import numpy as np

from oracle import fem


def check(got, ref, scale, tol, what=""):
    """|got_i - ref_i| <= tol * scale_i for every i; reports the worst entry."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    scale = np.broadcast_to(np.asarray(scale, dtype=np.float64).ravel(), ref.shape)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite entries"
    err = np.abs(got - ref)
    bad = err > tol * scale
    if np.any(bad):
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(scale > 0, err / scale, np.inf)
        i = int(np.argmax(ratio))
        raise AssertionError(f"{what}: {int(bad.sum())} of {len(ref)} entries off; worst entry {i}: "
                             f"got {got[i]:.17g} ref {ref[i]:.17g} |err|/scale {ratio[i]:.3e} > tol {tol:.1e}")
    return float(np.max(np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), 0.0))) if len(ref) else 0.0


def check_inf(got, ref, tol, what=""):
    """|got_i - ref_i| <= tol * ||ref||_inf for every i."""
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return check(got, ref, np.full(ref.shape, max(np.abs(ref).max(initial=0.0), 1e-300)), tol, what)


def jacobian_scale(space, state, x, mask=None, form="A"):
    """|J| |x|: the Jacobian apply of ``x`` with every element-matrix entry and
    every input entry in absolute value (constrained rows: |x_i|)."""
    Ke = fem.element_matrices(space, state, form)
    A = fem.assemble(space, np.abs(Ke), mask)
    return A @ np.abs(np.asarray(x, dtype=np.float64).ravel())


def diagonal_scale(space, state, mask=None, form="A"):
    """The diagonal's sum over elements, points and gradient directions in
    absolute value (constrained rows 1)."""
    D = np.abs(fem.tangent(state, form))
    Dcc = np.einsum("eqcdcf->eqcdf", D)
    B = np.abs(space.Bxi)
    de = np.einsum("dql,eqcdf,fql->elc", B, Dcc, B)
    y = np.zeros((space.n_nodes, 3))
    np.add.at(y, space.elem_nodes.ravel(), de.reshape(-1, 3))
    y = y.ravel()
    if mask is not None:
        y[mask] = 1.0
    return y


def residual_scale(space, mat, u, mask=None, g_bc=None):
    """E^T |B_xi|^T |f| with f = W P (grad_X xi)^T the stress at the points;
    constrained rows |u_i| + |g_i|."""
    st = fem.qp_state(space, mat, u)
    S, _ = fem.second_piola(st)
    Pk = st["F"] @ S
    fhat = np.abs(st["W"][..., None, None] * (Pk @ fem.T(st["dxidX"])))
    ye = np.einsum("dql,eqcd->elc", np.abs(space.Bxi), fhat)
    y = np.zeros((space.n_nodes, 3))
    np.add.at(y, space.elem_nodes.ravel(), ye.reshape(-1, 3))
    y = y.ravel()
    if mask is not None:
        u = np.abs(np.asarray(u, dtype=np.float64).ravel())
        g = np.zeros_like(u) if g_bc is None else np.abs(np.asarray(g_bc, dtype=np.float64).ravel())
        y[mask] = (u + g)[mask]
    return y


def prolong_scale(coarse, fine, uc):
    """The prolongation of |uc| with |B_ctof| (Eq. mg_prolong in absolute value)."""
    B = np.abs(fem.ctof_matrix(coarse, fine))
    ue = np.abs(np.asarray(uc, dtype=np.float64)).reshape(coarse.n_nodes, 3)[coarse.elem_nodes]
    fe = np.einsum("fc,ecx->efx", B, ue) * (1.0 / fine.multiplicity())[fine.elem_nodes][..., None]
    uf = np.zeros((fine.n_nodes, 3))
    np.add.at(uf, fine.elem_nodes.ravel(), fe.reshape(-1, 3))
    return uf.ravel()


def restrict_scale(fine, coarse, rf):
    """The restriction of |rf| with |B_ctof|."""
    B = np.abs(fem.ctof_matrix(coarse, fine))
    minv = 1.0 / fine.multiplicity()
    re = np.abs(np.asarray(rf, dtype=np.float64)).reshape(fine.n_nodes, 3)[fine.elem_nodes]
    ce = np.einsum("fc,efx->ecx", B, re * minv[fine.elem_nodes][..., None])
    rc = np.zeros((coarse.n_nodes, 3))
    np.add.at(rc, coarse.elem_nodes.ravel(), ce.reshape(-1, 3))
    return rc.ravel()

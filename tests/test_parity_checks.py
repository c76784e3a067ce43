"""CPU checks of the entry-wise parity checker (tests/parity.py).

The scales must bound every entry of the quantity they go with (triangle
inequality), accept two independent evaluations of the same operator that
differ only by rounding, and reject mistakes planted in the oracle's result
that a norm-wise check over the whole vector lets through.
"""
import numpy as np
import pytest

import parity
from oracle import fem
from paper_2204_01722_b300 import inputs


def make(n=(3, 2, 2), p=2, seed=3, E=None):
    V = inputs.box_vertices(*n, perturb=0.1, seed=seed)
    sp = fem.Space(*n, V, p, p + 1)
    mat = fem.Material(1.0 if E is None else E, 0.3, sp.ne)
    u = inputs.smooth_field(sp.node_coords(), 0.05, seed=seed + 1).ravel()
    mask = inputs.uniaxial_mask(sp.node_dims)
    return sp, mat, u, mask, fem.qp_state(sp, mat, u)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_jacobian_scale_bounds_and_accepts_the_other_form(p):
    sp, mat, u, mask, st = make(p=p)
    du = inputs.normal_vector(sp.n_dof, seed=5)
    ya = fem.jacobian_apply(sp, st, du, mask, form="A")
    yb = fem.jacobian_apply(sp, st, du, mask, form="B")
    s = parity.jacobian_scale(sp, st, du, mask)
    assert np.all(s >= np.abs(ya) * (1 - 1e-14))
    # constrained rows are the identity: the scale is |du| there
    assert np.array_equal(s[mask], np.abs(du[mask]))
    # the two linearisations (Eq. dtau and dP = dF S + F dS) differ only by rounding
    parity.check(yb, ya, s, 1e-12, "form B vs form A")
    # the element matrices applied one element at a time give the same result
    Ke = fem.element_matrices(sp, st)
    ye = fem.assemble(sp, Ke, mask) @ du
    parity.check(ye, ya, s, 1e-12, "assembled vs matrix-free")


def test_planted_mistakes_are_caught():
    sp, mat, u, mask, st = make(p=2)
    du = inputs.normal_vector(sp.n_dof, seed=6)
    ref = fem.jacobian_apply(sp, st, du, mask)
    s = parity.jacobian_scale(sp, st, du, mask)
    norm = np.linalg.norm(ref)

    def rejected(y):
        with pytest.raises(AssertionError):
            parity.check(y, ref, s, 1e-12)

    # a constrained row with the wrong sign
    i = int(np.flatnonzero(mask)[0])
    y = ref.copy()
    y[i] = -y[i]
    rejected(y)
    # one element's contribution to one node dropped (the scatter of one element missed)
    v = du.copy()
    v[mask] = 0.0
    g = sp.ref_gradient(v)
    fh = fem.pointwise_A(st, g)
    ye = np.einsum("dql,eqcd->elc", sp.Bxi, fh)
    free_nodes = np.flatnonzero(~mask.reshape(-1, 3).any(axis=1))
    e, l = np.argwhere(np.isin(sp.elem_nodes, free_nodes))[0]
    y = ref.copy()
    node = sp.elem_nodes[e, l]
    y[3 * node:3 * node + 3] -= ye[e, l]
    rejected(y)
    # an error that the norm-wise 1e-12 test lets through: 5e-13 of the whole
    # vector's norm placed on the unconstrained entry with the smallest scale
    free = np.flatnonzero(~mask)
    i = int(free[np.argmin(s[free])])
    y = ref.copy()
    y[i] += 5e-13 * norm
    assert np.linalg.norm(y - ref) / norm < 1e-12
    rejected(y)


def test_diagonal_scale():
    sp, mat, u, mask, st = make(p=3, n=(2, 2, 2))
    d = fem.diagonal(sp, st, mask)
    s = parity.diagonal_scale(sp, st, mask)
    assert np.all(s >= np.abs(d) * (1 - 1e-14))
    # the diagonal of the assembled element matrices, an independent evaluation
    Ke = fem.element_matrices(sp, st)
    parity.check(fem.assemble(sp, Ke, mask).diagonal(), d, s, 1e-12, "diagonal")


def test_residual_scale_accepts_the_kirchhoff_form():
    """The residual through the Kirchhoff stress tested against grad_x v
    (Eq. residual-discrete, current configuration) equals the oracle's first
    Piola form to rounding, entry by entry."""
    sp, mat, u, mask, st = make(p=2, n=(2, 3, 2))
    g = inputs.uniaxial_bc(sp.node_dims, 0.01)
    r = fem.residual(sp, mat, u, mask, g)
    s = parity.residual_scale(sp, mat, u, mask, g)
    assert np.all(s >= np.abs(r) * (1 - 1e-14))
    dxidx = st["dxidX"] @ st["Finv"]
    fhat = st["W"][..., None, None] * (st["tau"] @ fem.T(dxidx))
    r2 = sp.apply_Bxi_T(fhat).ravel()
    r2[mask] = (u - g)[mask]
    parity.check(r2, r, s, 1e-12, "Kirchhoff vs Piola residual")
    y = r.copy()
    y[int(np.flatnonzero(~mask)[3])] *= 1 + 1e-9
    with pytest.raises(AssertionError):
        parity.check(y, r, s, 1e-12)


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (1, 3)])
def test_transfer_scales(pc, pf):
    n = (2, 2, 3)
    V = inputs.box_vertices(*n, perturb=0.1, seed=2)
    c = fem.Space(*n, V, pc, pf + 1)
    f = fem.Space(*n, V, pf, pf + 1)
    uc = inputs.normal_vector(c.n_dof, seed=1)
    rf = inputs.normal_vector(f.n_dof, seed=2)
    P = fem.prolong(c, f, uc)
    R = fem.restrict(f, c, rf)
    sp_ = parity.prolong_scale(c, f, uc)
    sr = parity.restrict_scale(f, c, rf)
    assert np.all(sp_ >= np.abs(P) * (1 - 1e-14)) and np.all(sr >= np.abs(R) * (1 - 1e-14))
    # restriction is the transpose of prolongation: r^T P u = (R r)^T u
    assert abs(rf @ P - fem.restrict(f, c, rf) @ uc) <= 1e-12 * (np.abs(rf) @ sp_)
    y = P.copy()
    y[7] += 1e-9 * sp_[7]
    with pytest.raises(AssertionError):
        parity.check(y, P, sp_, 1e-12)


def test_check_inf():
    ref = np.array([1.0, -2.0, 0.0])
    parity.check_inf(ref + 1e-13, ref, 1e-12)
    with pytest.raises(AssertionError):
        parity.check_inf(ref + np.array([0.0, 0.0, 1e-11]), ref, 1e-12)

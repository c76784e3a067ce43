"""Fixtures under tests/golden/.

* Oracle regression values (written by tests/golden/make_golden.py, which calls
  only the oracle): the residual and both linearisations on a small seeded Q2
  case must still match to 1e-12 relative, so a change to the oracle's arithmetic
  shows up here.
* The paper's table of Jacobian representations (Sec. V-E): the current
  configuration stores 17 scalars per quadrature point, the tuned initial
  configuration 26 and the AD one 31 (its tape taken as C^-1, 6 scalars).  The
  test packs exactly those scalars from the oracle's state, rebuilds the pointwise
  linearisation from the packed values and the (homogeneous) Lame constants alone
  and checks it against the oracle's form A / form B, so each listed set suffices.
"""
import os
import sys

import numpy as np
import pytest

from oracle import fem
from paper_2204_01722_b300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden  # noqa: E402

I3 = np.eye(3)
SYM = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


@pytest.mark.parametrize("name", ["residual", "jacobian_apply_A", "jacobian_apply_B"])
def test_oracle_regression_values(name):
    stored = np.loadtxt(make_golden.path(name))
    now = make_golden.values()[name]
    assert stored.shape == now.shape
    assert np.linalg.norm(now - stored) <= 1e-12 * np.linalg.norm(stored)


def storage_table():
    rows = {}
    with open(os.path.join(HERE, "storage_scalars.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, count = line.split()[:2]
                rows[name] = int(count)
    return rows


def unpack_sym(v):
    A = np.zeros(v.shape[:-1] + (3, 3))
    for k, (i, j) in enumerate(SYM):
        A[..., i, j] = A[..., j, i] = v[..., k]
    return A


def pack_sym(A):
    return np.stack([A[..., i, j] for i, j in SYM], axis=-1)


def state_and_gradient():
    V = inputs.box_vertices(2, 2, 1, perturb=0.1, seed=5)
    sp = fem.Space(2, 2, 1, V, 2, 3)
    mat = fem.Material(1.0, 0.3, sp.ne)
    u = inputs.smooth_field(sp.node_coords(), 0.05, seed=6).ravel()
    st = fem.qp_state(sp, mat, u)
    g = np.random.default_rng(7).normal(size=st["W"].shape + (3, 3))
    return st, g, mat.lam[0], mat.mu[0]


def test_current_configuration_needs_17_scalars():
    st, g, lam, mu = state_and_gradient()
    X = st["dxidX"] @ st["Finv"]
    packed = np.concatenate([st["W"][..., None], X.reshape(X.shape[:-2] + (9,)), pack_sym(st["tau"]),
                             (lam * st["logJ"])[..., None]], axis=-1)
    assert packed.shape[-1] == storage_table()["current"]
    W, Xp, tau, llj = packed[..., 0], packed[..., 1:10].reshape(X.shape), unpack_sym(packed[..., 10:16]), packed[..., 16]
    G = g @ Xp
    de = 0.5 * (G + np.swapaxes(G, -1, -2))
    sig = G @ tau + lam * np.trace(de, axis1=-2, axis2=-1)[..., None, None] * I3 + 2.0 * (mu - llj)[..., None, None] * de
    f = W[..., None, None] * (sig @ np.swapaxes(Xp, -1, -2))
    ref = fem.pointwise_A(st, g)
    assert np.abs(f - ref).max() <= 1e-13 * np.abs(ref).max()


def test_initial_configuration_tuned_needs_26_scalars():
    st, g, lam, mu = state_and_gradient()
    Finv = st["Finv"]
    Cinv = Finv @ np.swapaxes(Finv, -1, -2)
    sh = st["W"].shape
    packed = np.concatenate([st["dxidX"].reshape(sh + (9,)), st["W"][..., None], st["H"].reshape(sh + (9,)),
                             pack_sym(Cinv), (lam * st["logJ"])[..., None]], axis=-1)
    assert packed.shape[-1] == storage_table()["initial_tuned"]
    D = packed[..., 0:9].reshape(sh + (3, 3))
    W = packed[..., 9]
    F = I3 + packed[..., 10:19].reshape(sh + (3, 3))
    Ci = unpack_sym(packed[..., 19:25])
    llj = packed[..., 25][..., None, None]
    S = mu * (I3 - Ci) + llj * Ci
    dF = g @ D
    dE = 0.5 * (np.swapaxes(F, -1, -2) @ dF + np.swapaxes(dF, -1, -2) @ F)
    dS = lam * np.einsum("...ij,...ij", Ci, dE)[..., None, None] * Ci + 2.0 * (mu - llj) * (Ci @ dE @ Ci)
    f = W[..., None, None] * ((dF @ S + F @ dS) @ np.swapaxes(D, -1, -2))
    ref = fem.pointwise_B(st, g)
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()


def test_initial_configuration_ad_needs_31_scalars():
    """S comes from the residual evaluation; the tangent needs C^-1 (the tape) and
    log J, which the tape also fixes: log J = -log det(C^-1) / 2."""
    st, g, lam, mu = state_and_gradient()
    Finv = st["Finv"]
    Cinv = Finv @ np.swapaxes(Finv, -1, -2)
    S, _ = fem.second_piola(st)
    sh = st["W"].shape
    packed = np.concatenate([st["dxidX"].reshape(sh + (9,)), st["W"][..., None], st["H"].reshape(sh + (9,)),
                             pack_sym(S), pack_sym(Cinv)], axis=-1)
    assert packed.shape[-1] == storage_table()["initial_AD"]
    D = packed[..., 0:9].reshape(sh + (3, 3))
    W = packed[..., 9]
    F = I3 + packed[..., 10:19].reshape(sh + (3, 3))
    Sp = unpack_sym(packed[..., 19:25])
    Ci = unpack_sym(packed[..., 25:31])
    logJ = (-0.5 * np.log(np.linalg.det(Ci)))[..., None, None]
    dF = g @ D
    dE = 0.5 * (np.swapaxes(F, -1, -2) @ dF + np.swapaxes(dF, -1, -2) @ F)
    dS = lam * np.einsum("...ij,...ij", Ci, dE)[..., None, None] * Ci + 2.0 * (mu - lam * logJ) * (Ci @ dE @ Ci)
    f = W[..., None, None] * ((dF @ Sp + F @ dS) @ np.swapaxes(D, -1, -2))
    ref = fem.pointwise_B(st, g)
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()

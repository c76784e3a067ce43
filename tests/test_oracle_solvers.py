"""Pins of the oracle's solver definitions: Chebyshev residual polynomial in
closed form, CG/Lanczos against direct solves and eigenvalues, and the
V-cycle's symmetry with restriction = prolongation^T."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, solvers
from paper_2204_01722_b300 import inputs


def test_chebyshev_matches_closed_form():
    """On D^-1 A with known spectrum the error after k steps is
    p_k(lambda) e_0, p_k(lambda) = T_k((theta - lambda)/delta) / T_k(theta/delta)."""
    rng = np.random.default_rng(0)
    n = 40
    lam = np.sort(rng.uniform(0.05, 1.0, n))
    d = rng.uniform(0.5, 2.0, n)
    A = np.diag(lam * d)            # D^-1 A = diag(lam)
    dinv = 1.0 / d
    xs = rng.normal(size=n)
    b = A @ xs
    lmax = lam.max()
    for k in [1, 2, 3, 5]:
        x = solvers.chebyshev(lambda v: A @ v, dinv, b, np.zeros(n), lmax, k)
        a, bb = 0.1 * lmax, 1.1 * lmax
        theta, delta = (bb + a) / 2, (bb - a) / 2
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        pk = Tk((theta - lam) / delta) / Tk(theta / delta)
        np.testing.assert_allclose(xs - x, pk * xs, atol=1e-13)


def test_cg_and_lanczos():
    rng = np.random.default_rng(1)
    n = 30
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.linspace(1.0, 50.0, n)
    A = Q @ np.diag(ev) @ Q.T
    b = rng.normal(size=n)
    x, it, Tm = solvers.cg_lanczos(lambda v: A @ v, b, rtol=1e-12, maxit=200, norm="l2")
    np.testing.assert_allclose(A @ x, b, atol=1e-9)
    # after n steps the Ritz values are the eigenvalues
    _, it, Tm = solvers.cg_lanczos(lambda v: A @ v, b, rtol=0.0, maxit=n)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Tm)), ev, rtol=1e-6)
    # 10 steps bound lambda_max from below, close to it
    lm = solvers.estimate_lambda_max(lambda v: A @ v, np.ones(n), b, iters=10)
    assert 0.9 * ev[-1] < lm <= ev[-1] * (1 + 1e-12)


def _levels(n=2, p=4, degree=3):
    V = inputs.box_vertices(n, n, n, 0.1, seed=1)
    sps = [fem.Space(n, n, n, V, pp, p + 1) for pp in (p, 2, 1)]
    mat = fem.Material(1.0, 0.3, sps[0].ne)
    u = inputs.smooth_field(sps[0].node_coords(), 0.05, seed=2).ravel()
    st = fem.qp_state(sps[0], mat, u)
    levels = []
    for i, sp in enumerate(sps):
        mask = inputs.uniaxial_mask(sp.node_dims)
        A = (lambda s, m: (lambda v: fem.jacobian_apply(s, st, v, m)))(sp, mask)
        dinv = 1.0 / fem.diagonal(sp, st, mask)
        seed_vec = inputs.uniform_vector(sp.n_dof, seed=5)
        seed_vec[mask] = 0
        L = dict(A=A, dinv=dinv, mask=mask, degree=degree,
                 lmax=solvers.estimate_lambda_max(A, dinv, seed_vec))
        if i + 1 < len(sps):
            L["restrict"] = (lambda f, c: (lambda v: fem.restrict(f, c, v)))(sp, sps[i + 1])
            L["prolong"] = (lambda f, c: (lambda v: fem.prolong(c, f, v)))(sp, sps[i + 1])
        levels.append(L)
    return sps, levels


def test_vcycle_is_symmetric_with_exact_coarse_solve():
    sps, levels = _levels()
    mask = levels[0]["mask"]
    r1 = inputs.normal_vector(sps[0].n_dof, 1)
    r2 = inputs.normal_vector(sps[0].n_dof, 2)
    r1[mask] = 0
    r2[mask] = 0
    z1 = solvers.vcycle(levels, r1, coarse_rtol=1e-14)
    z2 = solvers.vcycle(levels, r2, coarse_rtol=1e-14)
    assert abs(r2 @ z1 - r1 @ z2) < 1e-10 * abs(r2 @ z1)
    assert r1 @ z1 > 0


def test_vcycle_preconditioned_cg_converges_fast():
    sps, levels = _levels()
    mask = levels[0]["mask"]
    b = inputs.normal_vector(sps[0].n_dof, 3)
    b[mask] = 0
    x, it, Tm = solvers.cg_lanczos(levels[0]["A"], b, apply_M=lambda r: solvers.vcycle(levels, r, coarse_rtol=1e-14),
                                   rtol=1e-8, maxit=100, norm="l2")
    assert it < 25
    ev = np.linalg.eigvalsh(Tm)
    assert ev.max() / ev.min() < 20
    _, it_j, _ = solvers.cg_lanczos(levels[0]["A"], b, apply_M=lambda r: levels[0]["dinv"] * r,
                                    rtol=1e-8, maxit=2000, norm="l2")
    assert it_j > 2 * it


def _spd(n, seed, lo=1.0, hi=50.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return Q @ np.diag(np.linspace(lo, hi, n)) @ Q.T, rng


def test_fcg_with_a_fixed_preconditioner_generates_the_pcg_iterates():
    """FCG(1) with a fixed SPD preconditioner: the truncated A-orthogonalisation
    is exact (CG's directions are A-conjugate), so its iterates are PCG's."""
    A, rng = _spd(30, 2)
    M = np.diag(rng.uniform(0.5, 2.0, 30))
    b = rng.normal(size=30)
    for k in range(1, 8):
        x_f, _, _ = solvers.fcg(lambda v: A @ v, b, lambda v: M @ v, rtol=0.0, maxit=k)
        x_c, _, _ = solvers.cg_lanczos(lambda v: A @ v, b, apply_M=lambda v: M @ v, rtol=0.0, maxit=k)
        np.testing.assert_allclose(x_f, x_c, rtol=1e-11, atol=1e-12 * np.linalg.norm(x_c))


def test_fcg_tolerates_a_varying_preconditioner():
    """Alternating two different SPD preconditioners (plain PCG loses its
    conjugacy): FCG(1) still converges to the solution."""
    A, rng = _spd(40, 3, 1.0, 1e3)
    M1 = np.diag(1.0 / np.diag(A))
    M2 = np.linalg.inv(A + np.diag(rng.uniform(0, 50, 40)))
    calls = [0]

    def M(v):
        calls[0] += 1
        return (M1 if calls[0] % 2 else M2) @ v
    b = rng.normal(size=40)
    x, k, rel = solvers.fcg(lambda v: A @ v, b, M, rtol=1e-12, maxit=400)
    assert rel <= 1e-12 and k < 400
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)


def test_chebyshev_solve_closed_form_and_symmetry():
    """x = q(M A) M b: on a diagonal problem with spectrum of M A inside [a, b]
    the error after k steps is p_k(lambda) e_0 with the scaled Chebyshev
    polynomial; on a general SPD problem the map b -> x is linear and
    symmetric (M symmetric)."""
    rng = np.random.default_rng(4)
    n = 40
    lam = np.sort(rng.uniform(0.05, 1.0, n))
    d = rng.uniform(0.5, 2.0, n)
    A = np.diag(lam * d)
    Mv = lambda v: v / d          # noqa: E731  (M A = diag(lam))
    xs = rng.normal(size=n)
    a, bb = 0.04, 1.1
    theta, delta = (bb + a) / 2, (bb - a) / 2
    for k in (1, 2, 4, 9):
        x = solvers.chebyshev_solve(lambda v: A @ v, Mv, A @ xs, a, bb, k)
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        pk = Tk((theta - lam) / delta) / Tk(theta / delta)
        np.testing.assert_allclose(xs - x, pk * xs, atol=1e-12)
    S, rng = _spd(25, 5)
    dinv = 1.0 / np.diag(S)
    Q = np.stack([solvers.chebyshev_solve(lambda v: S @ v, lambda v: dinv * v, e, 0.02, 1.5, 7) for e in np.eye(25)],
                 axis=1)
    np.testing.assert_allclose(Q, Q.T, atol=1e-12 * np.abs(Q).max())
    assert np.linalg.eigvalsh(0.5 * (Q + Q.T)).min() > 0


def test_lanczos_extremes():
    """With as many steps as distinct eigenvalues the Ritz values are exact."""
    rng = np.random.default_rng(6)
    lam = np.array([0.3, 0.7, 1.1, 2.0, 5.0, 9.5])
    A = np.diag(lam)
    lo, hi = solvers.lanczos_extremes(lambda v: A @ v, lambda v: v.copy(), rng.uniform(-1, 1, 6), 6)
    assert abs(lo - 0.3) < 1e-10 and abs(hi - 9.5) < 1e-10


def test_newton_krylov_reaches_the_direct_newton_solution():
    """The load-stepped inexact Newton-Krylov driver (FCG(1) to 1e-3 with a
    Jacobi preconditioner, predictor, secant step) converges to the solution of
    Newton with direct solves on every load step."""
    n, p = (3, 2, 2), 2
    V = inputs.box_vertices(*n, perturb=0.1, seed=3)
    sp = fem.Space(*n, V, p, p + 1)
    mat = fem.Material(1.0, 0.3, sp.ne)
    mask = inputs.uniaxial_mask(sp.node_dims)
    g = inputs.uniaxial_bc(sp.node_dims, 0.04)

    def jacobi(st):
        dinv = 1.0 / fem.diagonal(sp, st, mask)
        return lambda v: dinv * v
    u, hist = solvers.newton_krylov(sp, mat, mask, g, 2, jacobi)
    uo = np.zeros(sp.n_dof)
    for k in (1, 2):
        uo, _ = solvers.newton_direct(sp, mat, uo, mask, g * k / 2, rtol=1e-13)
    assert np.linalg.norm(u - uo) / np.linalg.norm(uo) < 1e-7
    assert len(hist) == 2 and all(1 <= h[0] <= 8 for h in hist)
    r = fem.residual(sp, mat, u, mask, g)
    assert np.linalg.norm(r) < 1e-8 * np.linalg.norm(fem.residual(sp, mat, uo * 0.5, mask, g)) + 1e-12

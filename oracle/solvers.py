"""Solver definitions (oracle; test infrastructure only).

FP64, small meshes.  Krylov methods follow their textbook statements:
* CG (Hestenes-Stiefel) with the Lanczos tridiagonal built from the CG
  coefficients (Sec. III-A: condition-number and lambda_max estimates);
* Chebyshev semi-iteration on D^-1 A over [0.1, 1.1] lambda_max
  (Sec. III-B smoother; Saad, Iterative Methods, Alg. 12.1);
* the p-multigrid V-cycle of Algorithm multigrid_algorithm with
  restriction = prolongation^T; its coarsest solve is Jacobi-PCG to a
  tolerance (Sec. III-B) or a fixed preconditioned Chebyshev polynomial;
* flexible CG with truncation 1 (Notay 2000) for variable preconditioners;
* Newton with a direct sparse solve (for manufactured solutions) and the
  load-stepped Newton-Krylov driver (Sec. III-A) in ``newton_krylov``.
"""
import numpy as np

from . import fem


def newton_direct(space, mat, u0, mask, g_bc, body_force=None, rtol=1e-12, maxit=30):
    """Newton's method with the assembled Jacobian and a sparse direct solve."""
    import scipy.sparse.linalg as spla
    u = np.array(u0, dtype=np.float64).ravel()
    u[mask] = np.asarray(g_bc).ravel()[mask]
    r0 = None
    for it in range(maxit):
        r = fem.residual(space, mat, u, mask, g_bc, body_force)
        nr = np.linalg.norm(r)
        r0 = nr if r0 is None else r0
        if nr <= rtol * max(r0, 1e-300) or nr < 1e-14:
            return u, it
        st = fem.qp_state(space, mat, u)
        A = fem.assemble(space, fem.element_matrices(space, st), mask)
        u = u - spla.spsolve(A.tocsc(), r)
    raise RuntimeError("Newton did not converge")


def cg_lanczos(apply_A, b, x0=None, apply_M=None, rtol=1e-3, maxit=500, norm="natural"):
    """Preconditioned CG.  Returns x, iterations, and the Lanczos tridiagonal
    (alpha, beta) implied by the CG coefficients:
        T[k,k] = 1/a_k + b_{k-1}/a_{k-1},  T[k,k+1] = sqrt(b_k)/a_k.
    ``norm``: "natural" uses sqrt(r^T M r), "l2" uses ||r||_2."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    M = apply_M if apply_M is not None else (lambda v: v.copy())
    r = b - apply_A(x)
    z = M(r)
    rz = r @ z
    nrm0 = np.sqrt(abs(rz)) if norm == "natural" else np.linalg.norm(r)
    p = z.copy()
    alphas, betas = [], []
    it = 0
    nrm = nrm0
    while it < maxit and nrm > rtol * nrm0:
        Ap = apply_A(p)
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        z = M(r)
        rz_new = r @ z
        bta = rz_new / rz
        alphas.append(a)
        betas.append(bta)
        rz = rz_new
        p = z + bta * p
        it += 1
        nrm = np.sqrt(abs(rz)) if norm == "natural" else np.linalg.norm(r)
    return x, it, lanczos_tridiagonal(alphas, betas)


def lanczos_tridiagonal(alphas, betas):
    k = len(alphas)
    Tm = np.zeros((k, k))
    for i in range(k):
        Tm[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            Tm[i, i + 1] = Tm[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    return Tm


def estimate_lambda_max(apply_A, dinv, seed_vec, iters=10):
    """Largest Ritz value of D^-1 A from ``iters`` CG/Lanczos steps on a rough seed
    (Sec. III-B), with right-hand side ``seed_vec`` and zero initial guess."""
    _, it, Tm = cg_lanczos(apply_A, seed_vec, apply_M=lambda v: dinv * v, rtol=0.0, maxit=iters)
    return float(np.max(np.linalg.eigvalsh(Tm))) if it else 0.0


def lanczos_extremes(apply_A, apply_M, seed_vec, iters):
    """Smallest and largest Ritz values of M A after ``iters`` steps of
    M-preconditioned CG on ``seed_vec`` (zero initial guess)."""
    _, it, Tm = cg_lanczos(apply_A, seed_vec, apply_M=apply_M, rtol=0.0, maxit=iters)
    ev = np.linalg.eigvalsh(Tm)
    return float(ev[0]), float(ev[-1])


def chebyshev_solve(apply_A, apply_M, b, a, bnd, degree):
    """x = q(M A) M b: ``degree`` steps of Chebyshev semi-iteration for A x = b,
    preconditioned by M, for eigenvalues of M A in [a, bnd], from x = 0
    (Saad, Iterative Methods, Alg. 12.1).  A fixed polynomial, so linear in b."""
    theta = 0.5 * (bnd + a)
    delta = 0.5 * (bnd - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(b)
    r = b.copy()
    d = apply_M(r) / theta
    x = x + d
    for _ in range(1, degree):
        r = r - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + 2.0 * rho_new / delta * apply_M(r)
        x = x + d
        rho = rho_new
    return x


def fcg(apply_A, b, apply_M, x0=None, rtol=1e-8, maxit=500, norm="l2"):
    """Flexible CG with truncation 1 (Notay 2000): the new direction is
    A-orthogonalised against the previous one only,
        p_k = z_k - (z_k . A p_{k-1} / p_{k-1} . A p_{k-1}) p_{k-1},
    and the step is a_k = p_k . r_k / p_k . A p_k, so a preconditioner that
    varies between applications is allowed.  For a fixed symmetric positive
    definite M it generates the PCG iterates.  ``norm``: "l2" stops on
    ||r_k|| <= rtol ||r_0||, "natural" on sqrt(r.z).  Returns x, iterations,
    and the final relative norm."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    z = apply_M(r)
    nrm0 = np.sqrt(abs(r @ z)) if norm == "natural" else np.linalg.norm(r)
    if nrm0 == 0.0:
        return x, 0, 0.0
    p = z.copy()
    q = apply_A(p)
    nrm = nrm0
    k = 0
    while k < maxit:
        a = (p @ r) / (p @ q)
        x = x + a * p
        r = r - a * q
        k += 1
        z = apply_M(r)
        nrm = np.sqrt(abs(r @ z)) if norm == "natural" else np.linalg.norm(r)
        if nrm <= rtol * nrm0:
            break
        p = z - ((z @ q) / (p @ q)) * p
        q = apply_A(p)
    return x, k, nrm / nrm0


def chebyshev(apply_A, dinv, b, x, lmax, degree, lo=0.1, hi=1.1):
    """``degree`` steps of Chebyshev semi-iteration for A x = b preconditioned by
    D^-1 = diag(dinv), targeting eigenvalues of D^-1 A in [lo, hi] * lmax
    (Saad, Iterative Methods, Alg. 12.1)."""
    a, bnd = lo * lmax, hi * lmax
    theta = 0.5 * (bnd + a)
    delta = 0.5 * (bnd - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - apply_A(x)
    d = dinv * r / theta
    for k in range(degree):
        x = x + d
        if k + 1 == degree:
            break
        r = r - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + 2.0 * rho_new / delta * (dinv * r)
        rho = rho_new
    return x


def vcycle(levels, b, level=0, coarse_rtol=1e-3, coarse_maxit=1000):
    """One V-cycle (Algorithm multigrid_algorithm) on ``levels[level:]``.

    Each level is a dict with ``A`` (apply), ``dinv``, ``lmax``, ``degree``,
    ``mask`` and, except the last, ``restrict``/``prolong`` to the next level.
    The coarsest level is solved by Jacobi-PCG to ``coarse_rtol``, or, when its
    dict has ``cheb`` = (a, b, degree), by that fixed Jacobi-preconditioned
    Chebyshev polynomial."""
    L = levels[level]
    if level == len(levels) - 1:
        if "cheb" in L:   # fixed coarse solve: (a, b, degree) of a Jacobi-preconditioned polynomial
            a, bnd, degree = L["cheb"]
            return chebyshev_solve(L["A"], lambda v: L["dinv"] * v, b, a, bnd, degree)
        x, _, _ = cg_lanczos(L["A"], b, apply_M=lambda v: L["dinv"] * v, rtol=coarse_rtol,
                             maxit=coarse_maxit)
        return x
    x = chebyshev(L["A"], L["dinv"], b, np.zeros_like(b), L["lmax"], L["degree"])
    r = b - L["A"](x)
    rc = L["restrict"](r)
    rc[levels[level + 1]["mask"]] = 0.0
    ec = vcycle(levels, rc, level + 1, coarse_rtol, coarse_maxit)
    e = L["prolong"](ec)
    e[L["mask"]] = 0.0
    x = x + e
    x = chebyshev(L["A"], L["dinv"], b, x, L["lmax"], L["degree"])
    return x


def newton_krylov(space, mat, mask, g_bc, load_steps, make_precond, krylov_rtol=1e-3, newton_rtol=1e-8,
                  newton_atol=1e-13, maxit=30, line_search=True, krylov_maxit=500):
    """Load-stepped inexact Newton-Krylov solve of F(u) = 0 (Sec. III-A).

    Pseudo-time t_k = k / K with the boundary values t_k g on the constrained
    DoFs.  Each step starts with a predictor that carries the boundary increment
    w = t_k g - u (constrained entries only) into the interior through the
    tangent at the current state, J_uu du = -(F_u(u) + J_uc w), u <- u + w + du;
    then Newton iterations J du = -F(u) until ||F|| <= newton_rtol ||F(u_k^0)||
    (u_k^0 the predicted state) or ||F|| <= newton_atol.  Linear systems: FCG(1)
    to krylov_rtol in the preconditioner's natural norm, preconditioned by
    ``make_precond(state)`` (a callable r -> z built at the current state).
    Step length: one secant step on phi(a) = F(u + a du) . du when phi changes
    sign on [0, 1], clamped to [0.1, 1.5]; else the full step.
    Returns u and per-step lists of (Newton iterations, Krylov iterations)."""
    mask = np.asarray(mask, dtype=bool)
    g = np.asarray(g_bc, dtype=np.float64).ravel()
    u = np.zeros(space.n_dof)
    history = []
    for k in range(1, load_steps + 1):
        gk = g * (k / load_steps)
        st = fem.qp_state(space, mat, u)
        M = make_precond(st)
        A = (lambda s_: (lambda v: fem.jacobian_apply(space, s_, v, mask)))(st)
        w = np.zeros_like(u)
        w[mask] = gk[mask] - u[mask]
        Fu = fem.residual(space, mat, u, mask, gk)
        Fu[mask] = 0.0
        Jw = fem.jacobian_apply(space, st, w)
        Jw[mask] = 0.0
        du, kits, _ = fcg(A, -(Fu + Jw), M, rtol=krylov_rtol, maxit=krylov_maxit, norm="natural")
        u = u + w + du
        F = fem.residual(space, mat, u, mask, gk)
        nr0 = nr = np.linalg.norm(F)
        its = 0
        while not (nr <= newton_rtol * nr0) and not (nr <= newton_atol):
            if its >= maxit:
                raise RuntimeError("newton_krylov: iteration limit")
            st = fem.qp_state(space, mat, u)
            M = make_precond(st)
            A = (lambda s_: (lambda v: fem.jacobian_apply(space, s_, v, mask)))(st)
            du, ki, _ = fcg(A, -F, M, rtol=krylov_rtol, maxit=krylov_maxit, norm="natural")
            kits += ki
            Ft = fem.residual(space, mat, u + du, mask, gk)
            alpha = 1.0
            if line_search:
                phi0, phi1 = F @ du, Ft @ du
                if phi0 * phi1 < 0.0:
                    alpha = min(1.5, max(0.1, phi0 / (phi0 - phi1)))
            u = u + alpha * du
            F = Ft if alpha == 1.0 else fem.residual(space, mat, u, mask, gk)
            nr = np.linalg.norm(F)
            its += 1
        history.append((its, kits))
    return u, history

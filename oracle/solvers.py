"""Solver definitions (oracle; test infrastructure only).

FP64, small meshes.  Krylov methods follow their textbook statements:
* CG (Hestenes-Stiefel) with the Lanczos tridiagonal built from the CG
  coefficients (Sec. III-A: condition-number and lambda_max estimates);
* Chebyshev semi-iteration on D^-1 A over [0.1, 1.1] lambda_max
  (Sec. III-B smoother; Saad, Iterative Methods, Alg. 12.1);
* the p-multigrid V-cycle of Algorithm multigrid_algorithm with
  restriction = prolongation^T;
* flexible CG with truncation 1 (Notay 2000) for variable preconditioners;
* Newton with a direct sparse solve (for manufactured solutions) and the
  load-stepped Newton-Krylov driver (Sec. III-A).
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
    The coarsest level is solved by Jacobi-PCG to ``coarse_rtol``."""
    L = levels[level]
    if level == len(levels) - 1:
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

"""1-D quadrature rules and Lagrange tabulations (oracle; test infrastructure only).

The paper writes every element operator through the 1-D tabulations B_I
(shape-function values at quadrature points) and B_xi (their derivatives),
Sec. II-B, Eq. tensorDense.  It does not say which node set the Lagrange
basis uses; we read it as Gauss-Lobatto-Legendre (GLL) nodes, so that the
Q1 vertices are nodes of every Q_p lattice and p-prolongation is nodal
interpolation.  Quadrature is Gauss-Legendre with q points per direction.
"""
import numpy as np


def legendre(n, x):
    """Legendre polynomial P_n and its derivative at x (three-term recurrence)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # P_n' from (x^2-1) P_n' = n (x P_n - P_{n-1}); valid for |x| != 1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (x * p1 - p0) / (x * x - 1.0)
    at_end = np.abs(np.abs(x) - 1.0) < 1e-300
    if np.any(at_end):
        dp = np.where(at_end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gauss_legendre(q):
    """Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_q, tol 1e-15)."""
    if q < 1:
        raise ValueError("q >= 1")
    i = np.arange(q)
    x = -np.cos(np.pi * (i + 0.75) / (q + 0.5))
    for _ in range(100):
        p, dp = legendre(q, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-15:
            break
    _, dp = legendre(q, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def gauss_lobatto(n):
    """Gauss-Lobatto-Legendre nodes and weights on [-1, 1], n >= 2 points.

    Nodes are -1, 1 and the roots of P'_{n-1}; weights 2 / (N (N+1) P_N(x)^2),
    N = n - 1.
    """
    if n < 2:
        raise ValueError("n >= 2")
    N = n - 1
    x = -np.cos(np.pi * np.arange(n) / N)
    interior = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(N, interior)
        # Legendre ODE: (1-x^2) P'' = 2 x P' - N(N+1) P
        d2p = (2.0 * interior * dp - N * (N + 1) * p) / (1.0 - interior ** 2)
        dx = dp / d2p
        interior = interior - dx
        if interior.size == 0 or np.max(np.abs(dx)) < 1e-15:
            break
    x[1:-1] = interior
    x[0], x[-1] = -1.0, 1.0
    p, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * p * p)
    return x, w


def lagrange_tabulate(nodes, pts):
    """Values B[q, k] = L_k(pts[q]) and derivatives D[q, k] = L_k'(pts[q]).

    L_k is the Lagrange polynomial through ``nodes`` that is 1 at nodes[k]
    (product formula; derivative by the product rule).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    n, m = nodes.size, pts.size
    B = np.ones((m, n))
    D = np.zeros((m, n))
    for k in range(n):
        for l in range(n):
            if l == k:
                continue
            B[:, k] *= (pts - nodes[l]) / (nodes[k] - nodes[l])
        for l in range(n):
            if l == k:
                continue
            term = np.full(m, 1.0 / (nodes[k] - nodes[l]))
            for s in range(n):
                if s == k or s == l:
                    continue
                term *= (pts - nodes[s]) / (nodes[k] - nodes[s])
            D[:, k] += term
    return B, D


def tabulate(p, q):
    """B_I (q x (p+1)) and B_xi (q x (p+1)): GLL Lagrange basis of order p at
    q Gauss points, plus the Gauss weights (Sec. II-B, Eq. tensorDense)."""
    xg, wg = gauss_legendre(q)
    xn, _ = gauss_lobatto(p + 1)
    B, D = lagrange_tabulate(xn, xg)
    return B, D, xg, wg

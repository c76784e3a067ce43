"""Pins of the oracle's 1-D rules and tabulations against closed forms."""
import numpy as np
import pytest

from oracle import basis

# Gauss-Legendre nodes/weights in closed form (n <= 4)
GL = {
    1: ([0.0], [2.0]),
    2: ([-1 / np.sqrt(3), 1 / np.sqrt(3)], [1.0, 1.0]),
    3: ([-np.sqrt(3 / 5), 0.0, np.sqrt(3 / 5)], [5 / 9, 8 / 9, 5 / 9]),
    4: (sorted([s * np.sqrt(3 / 7 + t * 2 / 7 * np.sqrt(6 / 5)) for s in (-1, 1) for t in (-1, 1)]),
        None),
}
# Gauss-Lobatto nodes/weights in closed form (n <= 5)
GLL = {
    2: ([-1.0, 1.0], [1.0, 1.0]),
    3: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    4: ([-1.0, -1 / np.sqrt(5), 1 / np.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    5: ([-1.0, -np.sqrt(3 / 7), 0.0, np.sqrt(3 / 7), 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gauss_legendre_closed_form(n):
    x, w = basis.gauss_legendre(n)
    xe, we = GL[n]
    np.testing.assert_allclose(x, xe, atol=1e-15)
    if we is not None:
        np.testing.assert_allclose(w, we, atol=1e-15)
    if n == 4:
        # weights (18 -+ sqrt 30)/36 for the inner/outer pair
        wi = (18 + np.sqrt(30)) / 36
        wo = (18 - np.sqrt(30)) / 36
        np.testing.assert_allclose(w, [wo, wi, wi, wo], atol=1e-15)


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_exactness(n):
    x, w = basis.gauss_legendre(n)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    # degree 2n is not integrated exactly
    assert abs(np.dot(w, x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-8


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_gauss_lobatto_closed_form(n):
    x, w = basis.gauss_lobatto(n)
    xe, we = GLL[n]
    np.testing.assert_allclose(x, xe, atol=1e-15)
    np.testing.assert_allclose(w, we, atol=1e-15)


@pytest.mark.parametrize("n", range(2, 9))
def test_gauss_lobatto_exactness(n):
    x, w = basis.gauss_lobatto(n)
    for k in range(2 * n - 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p,q", [(1, 2), (2, 3), (3, 4), (4, 5), (2, 5), (1, 5)])
def test_lagrange_tabulation(p, q):
    B, D, xg, wg = basis.tabulate(p, q)
    xn, _ = basis.gauss_lobatto(p + 1)
    # partition of unity; derivative of a constant vanishes (B_xi 1 = 0)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-12)
    # reproduces every monomial of degree <= p and its derivative
    for k in range(p + 1):
        np.testing.assert_allclose(B @ xn ** k, xg ** k, atol=1e-13)
        dk = k * xg ** (k - 1) if k > 0 else 0 * xg
        np.testing.assert_allclose(D @ xn ** k, dk, atol=1e-12)
    # Kronecker property at the nodes
    Bn, _ = basis.lagrange_tabulate(xn, xn)
    np.testing.assert_allclose(Bn, np.eye(p + 1), atol=1e-15)


@pytest.mark.parametrize("p,q", [(2, 3), (3, 4), (1, 4), (2, 5)])
def test_collocated_gradient_pseudoinverse(p, q):
    """B_I has full column rank, B_I^+ B_I = I, and (B_xi B_I^+) B_I = B_xi (Sec. II-B)."""
    B, D, _, _ = basis.tabulate(p, q)
    Bp = np.linalg.pinv(B)
    np.testing.assert_allclose(Bp @ B, np.eye(p + 1), atol=1e-13)
    np.testing.assert_allclose((D @ Bp) @ B, D, atol=1e-12)

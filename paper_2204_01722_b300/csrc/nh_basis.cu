// 1-D quadrature rules and Lagrange tabulations for the element basis
// (Sec. II-B, Eq. tensorDense): Gauss-Legendre points, Gauss-Lobatto nodes,
// B_I (values), B_xi (derivatives) and the collocated derivative
// B_xi B_I^+ used to form gradients with 6 instead of 9 contractions.
// Host code; results are passed to kernels by value.
#include <math.h>
#include <string.h>

#include "nh_internal.cuh"

// Legendre P_n(x) and P_n'(x) by the three-term recurrence, |x| < 1.
static void legendre_pd(int n, double x, double* pn, double* dpn) {
  double a = 1.0, b = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; k++) {
    double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *dpn = n * (a - x * b) / (1.0 - x * x);
}

void nh_gauss(int q, double* x, double* w) {
  for (int i = 0; i < q; i++) {
    double r = cos(M_PI * (q - i - 0.25) / (q + 0.5));  // ascending initial guesses
    for (int it = 0; it < 100; it++) {
      double p, dp;
      legendre_pd(q, r, &p, &dp);
      double dr = p / dp;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    double p, dp;
    legendre_pd(q, r, &p, &dp);
    x[i] = r;
    w[i] = 2.0 / ((1.0 - r * r) * dp * dp);
  }
}

void nh_lobatto(int n, double* x) {
  int N = n - 1;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; i++) {
    double r = -cos(M_PI * i / N);
    for (int it = 0; it < 100; it++) {
      double p, dp;
      legendre_pd(N, r, &p, &dp);
      double d2p = (2.0 * r * dp - N * (N + 1.0) * p) / (1.0 - r * r);
      double dr = dp / d2p;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    x[i] = r;
  }
}

// val[j*n + k] = L_k(pts[j]), der[j*n + k] = L_k'(pts[j]) (product form, the
// derivative accumulated by the product rule).
void nh_lagrange(int n, const double* nodes, int m, const double* pts, double* val, double* der) {
  for (int j = 0; j < m; j++) {
    double x = pts[j];
    for (int k = 0; k < n; k++) {
      double v = 1.0, d = 0.0;
      for (int l = 0; l < n; l++) {
        if (l == k) continue;
        double f = 1.0 / (nodes[k] - nodes[l]);
        d = d * (x - nodes[l]) * f + v * f;
        v *= (x - nodes[l]) * f;
      }
      val[j * n + k] = v;
      if (der) der[j * n + k] = d;
    }
  }
}

// Small dense solve A X = Bm (A n x n, Bm n x m) by Gauss-Jordan elimination
// with partial pivoting, in place.
static void dense_solve(int n, int m, double* A, double* Bm) {
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; k++) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
      for (int k = 0; k < m; k++) { double t = Bm[c * m + k]; Bm[c * m + k] = Bm[piv * m + k]; Bm[piv * m + k] = t; }
    }
    for (int r = 0; r < n; r++) {
      if (r == c) continue;
      double f = A[r * n + c] / A[c * n + c];
      for (int k = 0; k < n; k++) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < m; k++) Bm[r * m + k] -= f * Bm[c * m + k];
    }
  }
  for (int r = 0; r < n; r++)
    for (int k = 0; k < m; k++) Bm[r * m + k] /= A[r * n + r];
}

void nh_tabulate(int p, int q, Tab1D* t) {
  memset(t, 0, sizeof(*t));
  int P = p + 1, Q = q;
  t->P = P;
  t->Q = Q;
  double xg[NH_MAXQ], xn[NH_MAXP], val[NH_MAXQ * NH_MAXP], der[NH_MAXQ * NH_MAXP];
  nh_gauss(Q, xg, t->w);
  nh_lobatto(P, xn);
  nh_lagrange(P, xn, Q, xg, val, der);
  for (int i = 0; i < Q; i++)
    for (int k = 0; k < P; k++) {
      t->B[i][k] = val[i * P + k];
      t->G[i][k] = der[i * P + k];
    }
  // B^+ = (B^T B)^-1 B^T  (P x Q); collocated derivative D = G B^+  (Q x Q)
  double BtB[NH_MAXP * NH_MAXP], Bp[NH_MAXP * NH_MAXQ];
  for (int a = 0; a < P; a++) {
    for (int b = 0; b < P; b++) {
      double s = 0;
      for (int i = 0; i < Q; i++) s += t->B[i][a] * t->B[i][b];
      BtB[a * P + b] = s;
    }
    for (int i = 0; i < Q; i++) Bp[a * Q + i] = t->B[i][a];
  }
  dense_solve(P, Q, BtB, Bp);
  for (int i = 0; i < Q; i++)
    for (int j = 0; j < Q; j++) {
      double s = 0;
      for (int k = 0; k < P; k++) s += t->G[i][k] * Bp[k * Q + j];
      t->D[i][j] = s;
    }
}

// Quadrature-data setup at one point (Sec. II-A/II-B, Eq. Kirchhoff-stress): from
// gX = dX/dxi and gU = du/dxi, W = wq det(dX/dxi), H = grad_X u, F = I + H,
// J - 1 from the invariants of H (log J = log1p(J - 1) without cancellation),
// e = (H + H^T + H H^T)/2, tau = 2 mu e + lambda log J I, grad_x xi = grad_X xi F^-1.
// Stores the layout's scalars at qp[i qstride] (store), returns the residual
// flux W tau (grad_x xi)^T in f (resid), and lowers jmin to J (or -1 for an
// inverted geometry).
#pragma once
#include "nh_internal.cuh"

__device__ __forceinline__ double nh_det3(const double (&A)[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// inverse via the adjugate; returns det
__device__ __forceinline__ double nh_inv3(const double (&A)[3][3], double (&Ai)[3][3]) {
  const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  const double id = 1.0 / det;
  Ai[0][0] = c00 * id;
  Ai[1][0] = c01 * id;
  Ai[2][0] = c02 * id;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
  return det;
}

// The same from the geometry factors R = grad_X xi and detx = det(dX/dxi), which
// depend on the mesh only (computed once and kept by the setup kernel).
template <int LAYOUT>
__device__ __forceinline__ void nh_setup_point_geom(const double (&R)[3][3], double detx, const double (&gU)[3][3],
                                                    double wq, double lam, double mu, double* __restrict__ qp,
                                                    int64_t qstride, int store, int resid, double (&f)[3][3],
                                                    double& jmin) {
  const double W = wq * detx;
  double H[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int K = 0; K < 3; K++) H[c][K] = gU[c][0] * R[0][K] + gU[c][1] * R[1][K] + gU[c][2] * R[2][K];
  const double trH = H[0][0] + H[1][1] + H[2][2];
  double trH2 = 0.0;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) trH2 += H[i][j] * H[j][i];
  const double Jm1 = trH + 0.5 * (trH * trH - trH2) + nh_det3(H);
  const double J = 1.0 + Jm1;
  // a NaN J or an inverted geometry counts as inverted
  jmin = fmin(jmin, (J > 0.0 && detx > 0.0) ? J : (J <= 0.0 ? J : -1.0));
  const double logJ = log1p(Jm1);
  double Fm[3][3], Fi[3][3];
#pragma unroll
  for (int i = 0; i < 9; i++) Fm[i / 3][i % 3] = H[i / 3][i % 3] + (i % 4 == 0 ? 1.0 : 0.0);
  nh_inv3(Fm, Fi);
  double tau[3][3];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const double hh = H[i][0] * H[j][0] + H[i][1] * H[j][1] + H[i][2] * H[j][2];
      tau[i][j] = mu * (H[i][j] + H[j][i] + hh) + (i == j ? lam * logJ : 0.0);
    }
  double X[3][3];  // grad_x xi = grad_X xi F^-1
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int k = 0; k < 3; k++) X[d][k] = R[d][0] * Fi[0][k] + R[d][1] * Fi[1][k] + R[d][2] * Fi[2][k];
  if (store) {
    if (LAYOUT == NH_LAYOUT_CURRENT) {
#pragma unroll
      for (int i = 0; i < 9; i++) qp[i * qstride] = X[i / 3][i % 3];
      qp[9 * qstride] = W * tau[0][0];
      qp[10 * qstride] = W * tau[1][1];
      qp[11 * qstride] = W * tau[2][2];
      qp[12 * qstride] = W * tau[1][2];
      qp[13 * qstride] = W * tau[0][2];
      qp[14 * qstride] = W * tau[0][1];
      qp[15 * qstride] = W * lam;
      qp[16 * qstride] = W * (mu - lam * logJ);
    } else if (LAYOUT == NH_LAYOUT_TAPE) {
      double Ci[3][3];
#pragma unroll
      for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Ci[i][j] = Fi[i][0] * Fi[j][0] + Fi[i][1] * Fi[j][1] + Fi[i][2] * Fi[j][2];
      // S = mu I + (lambda log J - mu) C^-1, the residual's second Piola stress
      const int ix[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
#pragma unroll
      for (int i = 0; i < 9; i++) qp[i * qstride] = R[i / 3][i % 3];
#pragma unroll
      for (int i = 0; i < 9; i++) qp[(9 + i) * qstride] = H[i / 3][i % 3];
#pragma unroll
      for (int m = 0; m < 6; m++) {
        const int i = ix[m][0], j = ix[m][1];
        qp[(18 + m) * qstride] = W * ((lam * logJ - mu) * Ci[i][j] + (i == j ? mu : 0.0));
        qp[(24 + m) * qstride] = Ci[i][j];
      }
      qp[30 * qstride] = W * lam;
      qp[31 * qstride] = 2.0 * W * (mu - lam * logJ);
    } else {
      double Ci[3][3];
#pragma unroll
      for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Ci[i][j] = Fi[i][0] * Fi[j][0] + Fi[i][1] * Fi[j][1] + Fi[i][2] * Fi[j][2];
#pragma unroll
      for (int i = 0; i < 9; i++) qp[i * qstride] = R[i / 3][i % 3];
#pragma unroll
      for (int i = 0; i < 9; i++) qp[(9 + i) * qstride] = H[i / 3][i % 3];
      qp[18 * qstride] = Ci[0][0];
      qp[19 * qstride] = Ci[1][1];
      qp[20 * qstride] = Ci[2][2];
      qp[21 * qstride] = Ci[1][2];
      qp[22 * qstride] = Ci[0][2];
      qp[23 * qstride] = Ci[0][1];
      qp[24 * qstride] = W * mu;
      qp[25 * qstride] = W * lam * logJ;
      qp[26 * qstride] = W * lam;
    }
  }
  if (resid) {
    // f1 = W tau (grad_x xi)^T
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int d = 0; d < 3; d++)
        f[c][d] = W * (tau[c][0] * X[d][0] + tau[c][1] * X[d][1] + tau[c][2] * X[d][2]);
  }
}

template <int LAYOUT>
__device__ __forceinline__ void nh_setup_point(const double (&gX)[3][3], const double (&gU)[3][3], double wq,
                                               double lam, double mu, double* __restrict__ qp, int64_t qstride,
                                               int store, int resid, double (&f)[3][3], double& jmin) {
  double R[3][3];  // grad_X xi
  const double detx = nh_inv3(gX, R);
  nh_setup_point_geom<LAYOUT>(R, detx, gU, wq, lam, mu, qp, qstride, store, resid, f, jmin);
}

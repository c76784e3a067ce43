// Pointwise linearised stress (the D of A = E^T B^T D B E), shared by the
// matrix-free kernels and the Q1 stencil assembly.  Internal.
#pragma once
#include "nh_internal.cuh"
#include "nh_ff.cuh"

namespace nhpw {

// Short dot products a0 b0 + a1 b1 + ...: for FP64 and FP32 the plain left-to-right
// expression (contracted to FMAs as written), in float-float a compensated dot
// product (ffd_*: one TwoSum per term, a single renormalisation).
template <typename T>
__device__ __forceinline__ T dot3(T a0, T b0, T a1, T b1, T a2, T b2) {
  return a0 * b0 + a1 * b1 + a2 * b2;
}
template <typename T>
__device__ __forceinline__ T dot4(T a0, T b0, T a1, T b1, T a2, T b2, T a3, T b3) {
  return a0 * b0 + a1 * b1 + a2 * b2 + a3 * b3;
}
template <typename T>
__device__ __forceinline__ T dot6(T a0, T b0, T a1, T b1, T a2, T b2, T a3, T b3, T a4, T b4, T a5, T b5) {
  return a0 * b0 + a1 * b1 + a2 * b2 + a3 * b3 + a4 * b4 + a5 * b5;
}
#ifndef NH_FF_DOT2_PW
#define NH_FF_DOT2_PW 1
#endif
#if NH_FF_DOT2_PW
template <>
__device__ __forceinline__ ff dot3<ff>(ff a0, ff b0, ff a1, ff b1, ff a2, ff b2) {
  ffdot d = ffd_first(a0, b0);
  ffd_add(d, a1, b1);
  ffd_add(d, a2, b2);
  return ffd_done(d);
}
template <>
__device__ __forceinline__ ff dot4<ff>(ff a0, ff b0, ff a1, ff b1, ff a2, ff b2, ff a3, ff b3) {
  ffdot d = ffd_first(a0, b0);
  ffd_add(d, a1, b1);
  ffd_add(d, a2, b2);
  ffd_add(d, a3, b3);
  return ffd_done(d);
}
template <>
__device__ __forceinline__ ff dot6<ff>(ff a0, ff b0, ff a1, ff b1, ff a2, ff b2, ff a3, ff b3, ff a4, ff b4, ff a5,
                                       ff b5) {
  ffdot d = ffd_first(a0, b0);
  ffd_add(d, a1, b1);
  ffd_add(d, a2, b2);
  ffd_add(d, a3, b3);
  ffd_add(d, a4, b4);
  ffd_add(d, a5, b5);
  return ffd_done(d);
}
#endif

// ---------------------------------------------------------------------------
// Pointwise linearised stress (the D of A = E^T B^T D B E).
// g[c][d] = d du_c / d xi_d at one quadrature point; f[c][d] is the reference
// flux tested against d v_c / d xi_d.  q points at this point's scalar 0,
// consecutive scalars are s apart.
// ---------------------------------------------------------------------------

// Current configuration (Eqs. Jacobian, dtau, depsilon): G = g grad_x xi,
// W sigma = G (W tau) + W lambda tr(G) I + W (mu - lambda log J) (G + G^T),
// f = W sigma (grad_x xi)^T.  Stored: grad_x xi (9, row d = xi_d), W tau
// (00, 11, 22, 12, 02, 01), W lambda, W (mu - lambda log J).
// ld(i) returns stored scalar i of the point
template <typename T, typename LD>
__device__ __forceinline__ void pw_current_ld(LD ld, const T (&g)[3][3], T (&f)[3][3]) {
  T X[3][3];
#pragma unroll
  for (int i = 0; i < 9; i++) X[i / 3][i % 3] = ld(i);
  const T t00 = ld(9), t11 = ld(10), t22 = ld(11);
  const T t12 = ld(12), t02 = ld(13), t01 = ld(14);
  const T wl = ld(15), wm = ld(16);
  const T tau[3][3] = {{t00, t01, t02}, {t01, t11, t12}, {t02, t12, t22}};
  T G[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int k = 0; k < 3; k++) G[c][k] = dot3(g[c][0], X[0][k], g[c][1], X[1][k], g[c][2], X[2][k]);
  const T trG = wl * (G[0][0] + G[1][1] + G[2][2]);
  T S[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int k = 0; k < 3; k++)
      S[c][k] = dot4(G[c][0], tau[0][k], G[c][1], tau[1][k], G[c][2], tau[2][k], wm, G[c][k] + G[k][c]);
  S[0][0] += trG;
  S[1][1] += trG;
  S[2][2] += trG;
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int d = 0; d < 3; d++) f[c][d] = dot3(S[c][0], X[d][0], S[c][1], X[d][1], S[c][2], X[d][2]);
}

// Initial configuration (Sec. V-E, "initial tuned" storage): dF = g grad_X xi,
// dE = sym(F^T dF), W S = W mu I + (W lambda log J - W mu) C^-1,
// W dS = W lambda (C^-1 : dE) C^-1 + 2 (W mu - W lambda log J) C^-1 dE C^-1,
// W dP = dF (W S) + F (W dS), f = W dP (grad_X xi)^T.  Stored: grad_X xi (9),
// H = grad_X u (9), C^-1 (00, 11, 22, 12, 02, 01), W mu, W lambda log J, W lambda.
template <typename T, typename LD>
__device__ __forceinline__ void pw_initial_ld(LD ld, const T (&g)[3][3], T (&f)[3][3]) {
  T R[3][3], F[3][3];
#pragma unroll
  for (int i = 0; i < 9; i++) R[i / 3][i % 3] = ld(i);
#pragma unroll
  for (int i = 0; i < 9; i++) F[i / 3][i % 3] = ld(9 + i) + (i % 4 == 0 ? T(1) : T(0));
  const T c00 = ld(18), c11 = ld(19), c22 = ld(20);
  const T c12 = ld(21), c02 = ld(22), c01 = ld(23);
  const T wmu = ld(24), wll = ld(25), wl = ld(26);
  const T Ci[3][3] = {{c00, c01, c02}, {c01, c11, c12}, {c02, c12, c22}};
  T dF[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int k = 0; k < 3; k++) dF[c][k] = dot3(g[c][0], R[0][k], g[c][1], R[1][k], g[c][2], R[2][k]);
  T dE[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++) dE[k][l] = dot3(F[0][k], dF[0][l], F[1][k], dF[1][l], F[2][k], dF[2][l]);
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = k + 1; l < 3; l++) {
      T m = T(0.5) * (dE[k][l] + dE[l][k]);
      dE[k][l] = m;
      dE[l][k] = m;
    }
  T trc = T(0);
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++) trc += Ci[k][l] * dE[k][l];
  T CdE[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++) CdE[k][l] = dot3(Ci[k][0], dE[0][l], Ci[k][1], dE[1][l], Ci[k][2], dE[2][l]);
  const T two_m = T(2) * (wmu - wll);
  T WdS[3][3], WS[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++) {
      T cdec = dot3(CdE[k][0], Ci[0][l], CdE[k][1], Ci[1][l], CdE[k][2], Ci[2][l]);
      WdS[k][l] = wl * trc * Ci[k][l] + two_m * cdec;
      WS[k][l] = (wll - wmu) * Ci[k][l] + (k == l ? wmu : T(0));
    }
  T dP[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int K = 0; K < 3; K++)
      dP[c][K] = dot6(dF[c][0], WS[0][K], dF[c][1], WS[1][K], dF[c][2], WS[2][K], F[c][0], WdS[0][K], F[c][1],
                      WdS[1][K], F[c][2], WdS[2][K]);
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int d = 0; d < 3; d++) f[c][d] = dot3(dP[c][0], R[d][0], dP[c][1], R[d][1], dP[c][2], R[d][2]);
}

// AD-style tape (Sec. V-E, "initial AD" storage): the same dP = dF S + F dS with
// W S stored by the residual evaluation and the tangent reading its tape, so no
// constitutive function is evaluated: W dS = W lambda (C^-1 : dE) C^-1
// + 2 W (mu - lambda log J) C^-1 dE C^-1.  Stored: grad_X xi (9), H (9),
// W S (00, 11, 22, 12, 02, 01), C^-1 (same order), W lambda, 2 W (mu - lambda log J).
template <typename T, typename LD>
__device__ __forceinline__ void pw_tape_ld(LD ld, const T (&g)[3][3], T (&f)[3][3]) {
  T R[3][3], F[3][3];
#pragma unroll
  for (int i = 0; i < 9; i++) R[i / 3][i % 3] = ld(i);
#pragma unroll
  for (int i = 0; i < 9; i++) F[i / 3][i % 3] = ld(9 + i) + (i % 4 == 0 ? T(1) : T(0));
  const T s00 = ld(18), s11 = ld(19), s22 = ld(20), s12 = ld(21), s02 = ld(22), s01 = ld(23);
  const T c00 = ld(24), c11 = ld(25), c22 = ld(26), c12 = ld(27), c02 = ld(28), c01 = ld(29);
  const T wl = ld(30), two_m = ld(31);
  const T WS[3][3] = {{s00, s01, s02}, {s01, s11, s12}, {s02, s12, s22}};
  const T Ci[3][3] = {{c00, c01, c02}, {c01, c11, c12}, {c02, c12, c22}};
  T dF[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int k = 0; k < 3; k++) dF[c][k] = dot3(g[c][0], R[0][k], g[c][1], R[1][k], g[c][2], R[2][k]);
  T dE[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = k; l < 3; l++) {
      const T a = dot3(F[0][k], dF[0][l], F[1][k], dF[1][l], F[2][k], dF[2][l]);
      const T b = dot3(F[0][l], dF[0][k], F[1][l], dF[1][k], F[2][l], dF[2][k]);
      dE[k][l] = T(0.5) * (a + b);
      dE[l][k] = dE[k][l];
    }
  T trc = T(0);
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++) trc += Ci[k][l] * dE[k][l];
  T CdE[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++) CdE[k][l] = dot3(Ci[k][0], dE[0][l], Ci[k][1], dE[1][l], Ci[k][2], dE[2][l]);
  T WdS[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int l = 0; l < 3; l++)
      WdS[k][l] = wl * trc * Ci[k][l] + two_m * dot3(CdE[k][0], Ci[0][l], CdE[k][1], Ci[1][l], CdE[k][2], Ci[2][l]);
  T dP[3][3];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int K = 0; K < 3; K++)
      dP[c][K] = dot6(dF[c][0], WS[0][K], dF[c][1], WS[1][K], dF[c][2], WS[2][K], F[c][0], WdS[0][K], F[c][1],
                      WdS[1][K], F[c][2], WdS[2][K]);
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int d = 0; d < 3; d++) f[c][d] = dot3(dP[c][0], R[d][0], dP[c][1], R[d][1], dP[c][2], R[d][2]);
}

template <int LAYOUT, typename T, typename LD>
__device__ __forceinline__ void pointwise_ld(LD ld, const T (&g)[3][3], T (&f)[3][3]) {
  if (LAYOUT == NH_LAYOUT_CURRENT)
    pw_current_ld<T>(ld, g, f);
  else if (LAYOUT == NH_LAYOUT_INITIAL)
    pw_initial_ld<T>(ld, g, f);
  else
    pw_tape_ld<T>(ld, g, f);
}

// scalars of the point at q, scalar i at q[i s]
template <int LAYOUT, typename T>
__device__ __forceinline__ void pointwise(const T* __restrict__ q, int64_t s, const T (&g)[3][3], T (&f)[3][3]) {
  pointwise_ld<LAYOUT, T>([&](int i) { return q[i * s]; }, g, f);
}

}  // namespace nhpw

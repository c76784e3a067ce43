// Rediscretised coarse levels (Sec. III-B, the alternative to the exact Galerkin
// coarse operators): the nonlinearity is re-evaluated from the fine state on the
// coarse level's own, smaller Gauss rule, which is sufficient for the coarse
// polynomials and lets the coarse applies stream fewer quadrature points.  One
// thread per coarse quadrature point evaluates the fine field's gradient there
// directly from the element's P_f^3 nodes (a degree-p_f field is not determined
// by fewer collocation points, so no collocated derivative is used) and stores
// that point's quadrature data with the fine setup's pointwise code.
#include "nh_setup_point.cuh"

namespace {

template <int PF, int QC>
struct PtTab {
  double B[QC][PF], G[QC][PF], w[QC];
};

__device__ __forceinline__ unsigned long long ordered_bits_pt(double v) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

template <int PF, int QC, int LAYOUT>
__global__ void __launch_bounds__(128)
    k_setup_pts(int64_t ne, const int* __restrict__ emap, const double* __restrict__ coords,
                const double* __restrict__ u, const double* __restrict__ lamv, const double* __restrict__ muv,
                const PtTab<PF, QC> tb, double* __restrict__ qd, int64_t qstride, unsigned long long* __restrict__ minj) {
  constexpr int Q3 = QC * QC * QC, P3 = PF * PF * PF;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double jmin = 1e300;
  if (gid < ne * Q3) {
    const int64_t e = gid / Q3;
    const int q = (int)(gid - e * Q3);
    const int qi = q % QC, qj = (q / QC) % QC, qk = q / (QC * QC);
    double gX[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gU[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < PF; k++)
      for (int j = 0; j < PF; j++) {
        const double byz = tb.B[qj][j] * tb.B[qk][k], gy = tb.G[qj][j] * tb.B[qk][k], gz = tb.B[qj][j] * tb.G[qk][k];
#pragma unroll
        for (int i = 0; i < PF; i++) {
          const int64_t n = __ldg(&emap[e * P3 + (k * PF + j) * PF + i]);
          const double d0 = tb.G[qi][i] * byz, d1 = tb.B[qi][i] * gy, d2 = tb.B[qi][i] * gz;
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const double xc = __ldg(&coords[3 * n + c]), uc = __ldg(&u[3 * n + c]);
            gX[c][0] += xc * d0;
            gX[c][1] += xc * d1;
            gX[c][2] += xc * d2;
            gU[c][0] += uc * d0;
            gU[c][1] += uc * d1;
            gU[c][2] += uc * d2;
          }
        }
      }
    double f[3][3];
    nh_setup_point<LAYOUT>(gX, gU, tb.w[qi] * tb.w[qj] * tb.w[qk], lamv[e], muv[e], qd + e * Q3 + q, qstride, 1, 0,
                           f, jmin);
  }
  __shared__ unsigned long long bmin;
  if (threadIdx.x == 0) bmin = ~0ull;
  __syncthreads();
  atomicMin(&bmin, ordered_bits_pt(jmin));
  __syncthreads();
  if (threadIdx.x == 0) atomicMin(minj, bmin);
}

template <int PF, int QC>
cudaError_t launch_pq(int layout, cudaStream_t s, int64_t ne, const int* emap, const double* coords, const double* u,
                      const double* lam, const double* mu, double* qd, int64_t qstride, unsigned long long* minj) {
  PtTab<PF, QC> tb;
  double xg[NH_MAXQ], w[NH_MAXQ], xn[NH_MAXP], val[NH_MAXQ * NH_MAXP], der[NH_MAXQ * NH_MAXP];
  nh_gauss(QC, xg, w);
  nh_lobatto(PF, xn);
  nh_lagrange(PF, xn, QC, xg, val, der);
  for (int i = 0; i < QC; i++) {
    tb.w[i] = w[i];
    for (int k = 0; k < PF; k++) {
      tb.B[i][k] = val[i * PF + k];
      tb.G[i][k] = der[i * PF + k];
    }
  }
  const int64_t n = ne * QC * QC * QC;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (layout == NH_LAYOUT_CURRENT)
    k_setup_pts<PF, QC, NH_LAYOUT_CURRENT><<<blocks, 128, 0, s>>>(ne, emap, coords, u, lam, mu, tb, qd, qstride, minj);
  else if (layout == NH_LAYOUT_INITIAL)
    k_setup_pts<PF, QC, NH_LAYOUT_INITIAL><<<blocks, 128, 0, s>>>(ne, emap, coords, u, lam, mu, tb, qd, qstride, minj);
  else
    k_setup_pts<PF, QC, NH_LAYOUT_TAPE><<<blocks, 128, 0, s>>>(ne, emap, coords, u, lam, mu, tb, qd, qstride, minj);
  return cudaGetLastError();
}

template <int PF>
cudaError_t launch_p(int QC, int layout, cudaStream_t s, int64_t ne, const int* emap, const double* coords,
                     const double* u, const double* lam, const double* mu, double* qd, int64_t qstride,
                     unsigned long long* minj) {
  switch (QC) {
    case 2: return launch_pq<PF, 2>(layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 3: return launch_pq<PF, 3>(layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 4: return launch_pq<PF, 4>(layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 5: return launch_pq<PF, 5>(layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 6: return launch_pq<PF, 6>(layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t nh_launch_setup_pts(int PF, int QC, int layout, cudaStream_t s, int64_t ne, const int* emap,
                                const double* coords, const double* u, const double* lam, const double* mu, double* qd,
                                int64_t qstride, unsigned long long* minj) {
  switch (PF) {
    case 2: return launch_p<2>(QC, layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 3: return launch_p<3>(QC, layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 4: return launch_p<4>(QC, layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
    case 5: return launch_p<5>(QC, layout, s, ne, emap, coords, u, lam, mu, qd, qstride, minj);
  }
  return cudaErrorInvalidValue;
}

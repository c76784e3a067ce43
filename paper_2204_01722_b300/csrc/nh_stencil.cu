// Assembled Q1 coarse operator on the structured node lattice.
//
// The p-multigrid coarse level is Q1 with the fine quadrature points and the
// fine quadrature data (exact Galerkin, Sec. III-B).  Applied matrix-free it
// would stream the whole fine quadrature data per coarse apply, and the coarse
// Jacobi-CG solve applies it hundreds of times per V-cycle.  Instead the
// element matrices K_e = sum_q G_q^T D_q G_q (the B^T D B of Sec. III-C) are
// built once per quadrature-data setup and summed into a 27-point block
// stencil: for every node, one 3x3 block per lattice neighbour, stored
// [27][9][n_nodes] so that one thread per node reads coalesced rows.
// Valid for the structured box meshes of nh_space_box.
#include "nh_krylov.cuh"
#include "nh_pointwise.cuh"

namespace {

constexpr int kQC = 8;  // quadrature points per chunk of pointwise tangents in shared memory

template <int Q>
struct Q1Tab {
  double B[Q][2], G[Q][2];
};

// One block of 64 threads per element; thread (a, b) accumulates the 3x3 block
// K_ab[c][c'] = sum_q sum_{d,d'} dN_a/dxi_d D[q; c,d; c',d'] dN_b/dxi_d'.
template <int Q, int LAYOUT>
__global__ void __launch_bounds__(64)
    k_assemble(int64_t ne, int nx, int ny, const double* __restrict__ qd, int64_t qstride, const Q1Tab<Q> tb,
               double* __restrict__ A, int64_t nn, int Nx, int Ny) {
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  __shared__ double Dq[kQC][81];
  const int t = threadIdx.x;
  const int a = t & 7, b = t >> 3;
  const int64_t e = blockIdx.x;
  const int ai = a & 1, aj = (a >> 1) & 1, ak = a >> 2;
  const int bi = b & 1, bj = (b >> 1) & 1, bk = b >> 2;
  double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int q0 = 0; q0 < Q3; q0 += kQC) {
    // pointwise tangent of kQC points: task = (point, c', d'), 9 per point
    for (int task = t; task < kQC * 9; task += 64) {
      const int ql = task / 9, cd = task % 9, cp = cd / 3, dp = cd % 3;
      const int q = q0 + ql;
      if (q < Q3) {
        double g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, f[3][3];
        g[cp][dp] = 1.0;
        nhpw::pointwise<LAYOUT, double>(qd + e * Q3 + q, qstride, g, f);
        for (int c = 0; c < 3; c++)
          for (int d = 0; d < 3; d++) Dq[ql][((c * 3 + d) * 3 + cp) * 3 + dp] = f[c][d];
      }
    }
    __syncthreads();
    for (int ql = 0; ql < kQC && q0 + ql < Q3; ql++) {
      const int q = q0 + ql, qi = q % Q, qj = (q / Q) % Q, qk = q / Q2;
      const double ga[3] = {tb.G[qi][ai] * tb.B[qj][aj] * tb.B[qk][ak], tb.B[qi][ai] * tb.G[qj][aj] * tb.B[qk][ak],
                            tb.B[qi][ai] * tb.B[qj][aj] * tb.G[qk][ak]};
      const double gb[3] = {tb.G[qi][bi] * tb.B[qj][bj] * tb.B[qk][bk], tb.B[qi][bi] * tb.G[qj][bj] * tb.B[qk][bk],
                            tb.B[qi][bi] * tb.B[qj][bj] * tb.G[qk][bk]};
      const double* D = Dq[ql];
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int cp = 0; cp < 3; cp++) {
          double s = 0.0;
#pragma unroll
          for (int d = 0; d < 3; d++)
#pragma unroll
            for (int dp = 0; dp < 3; dp++) s += ga[d] * D[((c * 3 + d) * 3 + cp) * 3 + dp] * gb[dp];
          K[c][cp] += s;
        }
    }
    __syncthreads();
  }
  // scatter into the stencil row of node a, neighbour offset b - a
  const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
  const int64_t na = (ex + ai) + Nx * ((ey + aj) + (int64_t)Ny * (ez + ak));
  const int s = (bi - ai + 1) + 3 * (bj - aj + 1) + 9 * (bk - ak + 1);
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int cp = 0; cp < 3; cp++) atomicAdd(&A[((int64_t)s * 9 + c * 3 + cp) * nn + na], K[c][cp]);
}

// y = M A M x + (I - M) x, M = projection onto unconstrained components
__global__ void __launch_bounds__(256)
    k_apply(int Nx, int Ny, int Nz, const uint8_t* __restrict__ bc, const double* __restrict__ A,
            const double* __restrict__ x, double* __restrict__ y) {
  const int64_t nn = (int64_t)Nx * Ny * Nz;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int I = (int)(n % Nx), J = (int)((n / Nx) % Ny), K = (int)(n / ((int64_t)Nx * Ny));
  double acc[3] = {0, 0, 0};
  for (int s = 0; s < 27; s++) {
    const int di = s % 3 - 1, dj = (s / 3) % 3 - 1, dk = s / 9 - 1;
    const int I2 = I + di, J2 = J + dj, K2 = K + dk;
    if (I2 < 0 || I2 >= Nx || J2 < 0 || J2 >= Ny || K2 < 0 || K2 >= Nz) continue;
    const int64_t m = I2 + (int64_t)Nx * (J2 + (int64_t)Ny * K2);
    const unsigned mb = bc[m];
    const double x0 = (mb & 1u) ? 0.0 : x[3 * m], x1 = (mb & 2u) ? 0.0 : x[3 * m + 1],
                 x2 = (mb & 4u) ? 0.0 : x[3 * m + 2];
    const double* As = A + (int64_t)s * 9 * nn + n;
    acc[0] += As[0 * nn] * x0 + As[1 * nn] * x1 + As[2 * nn] * x2;
    acc[1] += As[3 * nn] * x0 + As[4 * nn] * x1 + As[5 * nn] * x2;
    acc[2] += As[6 * nn] * x0 + As[7 * nn] * x1 + As[8 * nn] * x2;
  }
  const unsigned mb = bc[n];
  for (int c = 0; c < 3; c++) y[3 * n + c] = ((mb >> c) & 1u) ? x[3 * n + c] : acc[c];
}

__global__ void k_diag(int64_t nn, const uint8_t* __restrict__ bc, const double* __restrict__ A,
                       double* __restrict__ d) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const unsigned mb = bc[n];
  for (int c = 0; c < 3; c++) d[3 * n + c] = ((mb >> c) & 1u) ? 1.0 : A[((int64_t)13 * 9 + c * 4) * nn + n];
}

template <int Q>
cudaError_t assemble_q(cudaStream_t st, int64_t ne, int nx, int ny, int nz, const double* qd, int64_t qstride,
                       int layout, const Tab1D* tab, double* A) {
  Q1Tab<Q> tb;
  for (int i = 0; i < Q; i++)
    for (int j = 0; j < 2; j++) {
      tb.B[i][j] = tab->B[i][j];
      tb.G[i][j] = tab->G[i][j];
    }
  const int Nx = nx + 1, Ny = ny + 1;
  const int64_t nn = (int64_t)Nx * Ny * (nz + 1);
  if (ne == 0) return cudaSuccess;
  if (layout == NH_LAYOUT_CURRENT)
    k_assemble<Q, NH_LAYOUT_CURRENT><<<(unsigned)ne, 64, 0, st>>>(ne, nx, ny, qd, qstride, tb, A, nn, Nx, Ny);
  else
    k_assemble<Q, NH_LAYOUT_INITIAL><<<(unsigned)ne, 64, 0, st>>>(ne, nx, ny, qd, qstride, tb, A, nn, Nx, Ny);
  return cudaGetLastError();
}

}  // namespace

cudaError_t ks_assemble_q1(int Q, cudaStream_t st, int64_t ne, int nx, int ny, int nz, const uint8_t* bc,
                           const double* qd, int64_t qstride, int layout, const Tab1D* tab, double* A) {
  (void)bc;
  switch (Q) {
    case 2: return assemble_q<2>(st, ne, nx, ny, nz, qd, qstride, layout, tab, A);
    case 3: return assemble_q<3>(st, ne, nx, ny, nz, qd, qstride, layout, tab, A);
    case 4: return assemble_q<4>(st, ne, nx, ny, nz, qd, qstride, layout, tab, A);
    case 5: return assemble_q<5>(st, ne, nx, ny, nz, qd, qstride, layout, tab, A);
    case 6: return assemble_q<6>(st, ne, nx, ny, nz, qd, qstride, layout, tab, A);
  }
  return cudaErrorInvalidValue;
}

cudaError_t ks_apply(cudaStream_t st, int Nx, int Ny, int Nz, const uint8_t* bc, const double* A, const double* x,
                     double* y) {
  const int64_t nn = (int64_t)Nx * Ny * Nz;
  if (nn == 0) return cudaSuccess;
  k_apply<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Nx, Ny, Nz, bc, A, x, y);
  return cudaGetLastError();
}

cudaError_t ks_diag(cudaStream_t st, int64_t nn, const uint8_t* bc, const double* A, double* d) {
  if (nn == 0) return cudaSuccess;
  k_diag<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(nn, bc, A, d);
  return cudaGetLastError();
}

// Geometric multigrid for the assembled Q1 coarsest level: a structured stand-in
// for the algebraic multigrid coarse solve of Sec. III-B.  The vertex lattice is
// coarsened by 2 per direction; P is trilinear interpolation with constrained
// components neither interpolated to nor restricted from; coarse stencils are the
// Galerkin products A_c = P^T A P; smoothing is damped Jacobi; the coarsest
// lattice is solved exactly with a dense inverse.  All stencils use the layout
// [27][9][n_nodes] of the assembled Q1 operator, with zero entries for
// neighbours outside the lattice and for constrained columns.
#include "nh_krylov.cuh"

namespace {

constexpr int kT = 256;

__device__ __forceinline__ void node_ijk(int64_t n, int Nx, int Ny, int& I, int& J, int& K) {
  I = (int)(n % Nx);
  J = (int)((n / Nx) % Ny);
  K = (int)(n / ((int64_t)Nx * Ny));
}

// row (n, c) of the stencil times v, neighbour indices clamped into the lattice
// (their stored entries are zero)
__device__ __forceinline__ double hrow(int Nx, int Ny, int Nz, int64_t nn, int64_t n, int c,
                                       const double* __restrict__ A, const double* __restrict__ v) {
  int I, J, K;
  node_ijk(n, Nx, Ny, I, J, K);
  double acc = 0.0;
#pragma unroll
  for (int s = 0; s < 27; s++) {
    const int I2 = min(max(I + s % 3 - 1, 0), Nx - 1), J2 = min(max(J + (s / 3) % 3 - 1, 0), Ny - 1),
              K2 = min(max(K + s / 9 - 1, 0), Nz - 1);
    const int64_t m = I2 + (int64_t)Nx * (J2 + (int64_t)Ny * K2);
    const double* As = A + ((int64_t)s * 9 + 3 * c) * nn + n;
    acc += As[0] * v[3 * m] + As[nn] * v[3 * m + 1] + As[2 * nn] * v[3 * m + 2];
  }
  return acc;
}

// 1-D trilinear weight of fine index f for coarse index C (f = 2 C +- 1: 1/2)
__device__ __forceinline__ double w1(int f, int C) {
  const int d = f - 2 * C;
  return d == 0 ? 1.0 : (d == 1 || d == -1) ? 0.5 : 0.0;
}

__global__ void k_coarse_bc(int Nfx, int Nfy, int Ncx, int Ncy, int64_t nnc, const uint8_t* __restrict__ bcf,
                            uint8_t* __restrict__ bcc) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nnc) return;
  int x, y, z;
  node_ijk(I, Ncx, Ncy, x, y, z);
  bcc[I] = bcf[2 * x + (int64_t)Nfx * (2 * y + (int64_t)Nfy * 2 * z)];
}

// A_c[sc][c][c'][I] = sum_i sum_sf w(i, I) A_f[sf][c][c'][i] w(j, J), j = i + off(sf), J = I + off(sc),
// with constrained (fine or coarse) components excluded on both sides
__global__ void __launch_bounds__(kT) k_rap(int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz,
                                            const uint8_t* __restrict__ bcf, const uint8_t* __restrict__ bcc,
                                            const double* __restrict__ Af, double* __restrict__ Ac) {
  const int64_t nnf = (int64_t)Nfx * Nfy * Nfz, nnc = (int64_t)Ncx * Ncy * Ncz;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 27 * nnc) return;
  const int sc = (int)(tid / nnc);
  const int64_t I = tid - sc * nnc;
  int Ix, Iy, Iz;
  node_ijk(I, Ncx, Ncy, Ix, Iy, Iz);
  const int Jx = Ix + sc % 3 - 1, Jy = Iy + (sc / 3) % 3 - 1, Jz = Iz + sc / 9 - 1;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (Jx >= 0 && Jx < Ncx && Jy >= 0 && Jy < Ncy && Jz >= 0 && Jz < Ncz) {
    const unsigned mI = bcc[I], mJ = bcc[Jx + (int64_t)Ncx * (Jy + (int64_t)Ncy * Jz)];
    // per direction and fine offset a = i - 2 I: the stencil offsets s = j - i
    // with j inside the lattice and in the support of J (|j - 2 J| <= 1), in
    // increasing order -- the terms the full 27 x 27 walk would keep, in its order
    const int Ic[3] = {Ix, Iy, Iz}, Jc[3] = {Jx, Jy, Jz}, Nf[3] = {Nfx, Nfy, Nfz};
    unsigned vm[3];  // direction d: bit 3 (a + 1) + sd + 1 set when offset sd is kept for i = 2 I + a
#pragma unroll
    for (int d = 0; d < 3; d++) {
      unsigned m = 0;
#pragma unroll
      for (int a = -1; a <= 1; a++) {
        const int i = 2 * Ic[d] + a;
#pragma unroll
        for (int sd = -1; sd <= 1; sd++) {
          const int j = i + sd;
          if (i >= 0 && i < Nf[d] && j >= 0 && j < Nf[d] && j - 2 * Jc[d] >= -1 && j - 2 * Jc[d] <= 1)
            m |= 1u << (3 * (a + 1) + sd + 1);
        }
      }
      vm[d] = m;
    }
    const unsigned vmx = vm[0], vmy = vm[1], vmz = vm[2];
#pragma unroll 1
    for (int az = -1; az <= 1; az++)
#pragma unroll 1
      for (int ay = -1; ay <= 1; ay++)
#pragma unroll 1
        for (int ax = -1; ax <= 1; ax++) {
          const int ix = 2 * Ix + ax, iy = 2 * Iy + ay, iz = 2 * Iz + az;
          if (ix < 0 || ix >= Nfx || iy < 0 || iy >= Nfy || iz < 0 || iz >= Nfz) continue;
          const double wi = w1(ix, Ix) * w1(iy, Iy) * w1(iz, Iz);
          const int64_t ii = ix + (int64_t)Nfx * (iy + (int64_t)Nfy * iz);
          const unsigned mi = bcf[ii] | mI;
          const unsigned bx = vmx >> (3 * (ax + 1)), by = vmy >> (3 * (ay + 1)), bz = vmz >> (3 * (az + 1));
#pragma unroll 1
          for (int sz = -1; sz <= 1; sz++) {
            if (!((bz >> (sz + 1)) & 1u)) continue;
#pragma unroll 1
            for (int sy = -1; sy <= 1; sy++) {
              if (!((by >> (sy + 1)) & 1u)) continue;
#pragma unroll
              for (int sx = -1; sx <= 1; sx++) {
                if (!((bx >> (sx + 1)) & 1u)) continue;
                const int sf = (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
                const int jx = ix + sx, jy = iy + sy, jz = iz + sz;
                const double wj = w1(jx, Jx) * w1(jy, Jy) * w1(jz, Jz);
                const unsigned mj = bcf[jx + (int64_t)Nfx * (jy + (int64_t)Nfy * jz)] | mJ;
                const double* a = Af + (int64_t)sf * 9 * nnf + ii;
                const double w = wi * wj;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                  if ((mi >> c) & 1u) continue;
#pragma unroll
                  for (int cp = 0; cp < 3; cp++)
                    if (!((mj >> cp) & 1u)) acc[3 * c + cp] += w * a[(int64_t)(3 * c + cp) * nnf];
                }
              }
            }
          }
        }
  }
#pragma unroll
  for (int k = 0; k < 9; k++) Ac[((int64_t)sc * 9 + k) * nnc + I] = acc[k];
}

// damped Jacobi sweep on the correction: x_out = x_in + omega D^-1 (b - A x_in), x_in = 0 if zero_in;
// constrained components stay zero
__global__ void __launch_bounds__(kT) k_hjacobi(int Nx, int Ny, int Nz, const uint8_t* __restrict__ bc,
                                                const double* __restrict__ A, const double* __restrict__ dinv,
                                                const double* __restrict__ b, const double* __restrict__ xin,
                                                double* __restrict__ xout, double omega, int zero_in) {
  const int64_t nn = (int64_t)Nx * Ny * Nz;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nn) return;
  const int c = (int)(t / nn);
  const int64_t n = t - c * nn, i = 3 * n + c;
  if ((bc[n] >> c) & 1u) {
    xout[i] = 0.0;
    return;
  }
  const double x0 = zero_in ? 0.0 : xin[i];
  const double ax = zero_in ? 0.0 : hrow(Nx, Ny, Nz, nn, n, c, A, xin);
  xout[i] = x0 + omega * dinv[i] * (b[i] - ax);
}

__global__ void __launch_bounds__(kT) k_hresid(int Nx, int Ny, int Nz, const uint8_t* __restrict__ bc,
                                               const double* __restrict__ A, const double* __restrict__ b,
                                               const double* __restrict__ x, double* __restrict__ r) {
  const int64_t nn = (int64_t)Nx * Ny * Nz;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nn) return;
  const int c = (int)(t / nn);
  const int64_t n = t - c * nn, i = 3 * n + c;
  r[i] = ((bc[n] >> c) & 1u) ? 0.0 : b[i] - hrow(Nx, Ny, Nz, nn, n, c, A, x);
}

// b_c = P^T r_f
__global__ void k_hrestrict(int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* __restrict__ bcf,
                            const uint8_t* __restrict__ bcc, const double* __restrict__ rf, double* __restrict__ bcv) {
  const int64_t nnc = (int64_t)Ncx * Ncy * Ncz;
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nnc) return;
  int Ix, Iy, Iz;
  node_ijk(I, Ncx, Ncy, Ix, Iy, Iz);
  const unsigned mI = bcc[I];
  double s[3] = {0.0, 0.0, 0.0};
  for (int dz = -1; dz <= 1; dz++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dx = -1; dx <= 1; dx++) {
        const int ix = 2 * Ix + dx, iy = 2 * Iy + dy, iz = 2 * Iz + dz;
        if (ix < 0 || ix >= Nfx || iy < 0 || iy >= Nfy || iz < 0 || iz >= Nfz) continue;
        const double w = w1(ix, Ix) * w1(iy, Iy) * w1(iz, Iz);
        const int64_t ii = ix + (int64_t)Nfx * (iy + (int64_t)Nfy * iz);
        const unsigned mi = bcf[ii];
#pragma unroll
        for (int c = 0; c < 3; c++)
          if (!((mi >> c) & 1u)) s[c] += w * rf[3 * ii + c];
      }
#pragma unroll
  for (int c = 0; c < 3; c++) bcv[3 * I + c] = ((mI >> c) & 1u) ? 0.0 : s[c];
}

// x_f += P x_c
__global__ void k_hprolong_add(int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* __restrict__ bcf,
                               const uint8_t* __restrict__ bcc, const double* __restrict__ xc,
                               double* __restrict__ xf) {
  const int64_t nnf = (int64_t)Nfx * Nfy * Nfz;
  const int64_t ii = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ii >= nnf) return;
  int ix, iy, iz;
  node_ijk(ii, Nfx, Nfy, ix, iy, iz);
  const unsigned mi = bcf[ii];
  double s[3] = {0.0, 0.0, 0.0};
  for (int cz = iz >> 1; cz <= (iz + 1) >> 1 && cz < Ncz; cz++)
    for (int cy = iy >> 1; cy <= (iy + 1) >> 1 && cy < Ncy; cy++)
      for (int cx = ix >> 1; cx <= (ix + 1) >> 1 && cx < Ncx; cx++) {
        const double w = w1(ix, cx) * w1(iy, cy) * w1(iz, cz);
        const int64_t J = cx + (int64_t)Ncx * (cy + (int64_t)Ncy * cz);
        const unsigned mJ = bcc[J];
#pragma unroll
        for (int c = 0; c < 3; c++)
          if (!((mJ >> c) & 1u)) s[c] += w * xc[3 * J + c];
      }
#pragma unroll
  for (int c = 0; c < 3; c++)
    if (!((mi >> c) & 1u)) xf[3 * ii + c] += s[c];
}

// x = M b, M dense [n][n] (one warp per row)
__global__ void k_dense_mv(int n, const double* __restrict__ M, const double* __restrict__ b, double* __restrict__ x) {
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += M[(int64_t)row * n + j] * b[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = s;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

cudaError_t hm_coarse_bc(cudaStream_t st, int Nfx, int Nfy, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                         uint8_t* bcc) {
  const int64_t nnc = (int64_t)Ncx * Ncy * Ncz;
  k_coarse_bc<<<blocks_for(nnc), kT, 0, st>>>(Nfx, Nfy, Ncx, Ncy, nnc, bcf, bcc);
  return cudaGetLastError();
}
cudaError_t hm_rap(cudaStream_t st, int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                   const uint8_t* bcc, const double* Af, double* Ac) {
  const int64_t nnc = (int64_t)Ncx * Ncy * Ncz;
  k_rap<<<blocks_for(27 * nnc), kT, 0, st>>>(Nfx, Nfy, Nfz, Ncx, Ncy, Ncz, bcf, bcc, Af, Ac);
  return cudaGetLastError();
}
cudaError_t hm_jacobi(cudaStream_t st, int Nx, int Ny, int Nz, const uint8_t* bc, const double* A, const double* dinv,
                      const double* b, const double* xin, double* xout, double omega, int zero_in) {
  k_hjacobi<<<blocks_for(3 * (int64_t)Nx * Ny * Nz), kT, 0, st>>>(Nx, Ny, Nz, bc, A, dinv, b, xin, xout, omega,
                                                                   zero_in);
  return cudaGetLastError();
}
cudaError_t hm_resid(cudaStream_t st, int Nx, int Ny, int Nz, const uint8_t* bc, const double* A, const double* b,
                     const double* x, double* r) {
  k_hresid<<<blocks_for(3 * (int64_t)Nx * Ny * Nz), kT, 0, st>>>(Nx, Ny, Nz, bc, A, b, x, r);
  return cudaGetLastError();
}
cudaError_t hm_restrict(cudaStream_t st, int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                        const uint8_t* bcc, const double* rf, double* bcv) {
  k_hrestrict<<<blocks_for((int64_t)Ncx * Ncy * Ncz), kT, 0, st>>>(Nfx, Nfy, Nfz, Ncx, Ncy, Ncz, bcf, bcc, rf, bcv);
  return cudaGetLastError();
}
cudaError_t hm_prolong_add(cudaStream_t st, int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                           const uint8_t* bcc, const double* xc, double* xf) {
  k_hprolong_add<<<blocks_for((int64_t)Nfx * Nfy * Nfz), kT, 0, st>>>(Nfx, Nfy, Nfz, Ncx, Ncy, Ncz, bcf, bcc, xc, xf);
  return cudaGetLastError();
}
cudaError_t hm_dense_mv(cudaStream_t st, int n, const double* M, const double* b, double* x) {
  k_dense_mv<<<(unsigned)(((int64_t)n * 32 + kT - 1) / kT), kT, 0, st>>>(n, M, b, x);
  return cudaGetLastError();
}

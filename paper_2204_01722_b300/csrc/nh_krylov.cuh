// Launchers of the Krylov / smoother vector kernels (nh_krylov.cu) and of the
// assembled Q1 block stencil (nh_stencil.cu).  Internal.
#pragma once
#include "nh_internal.cuh"

template <typename T>
cudaError_t kv_axpby(cudaStream_t st, int64_t n, double a, const T* x, double b, T* y);
template <typename T>
cudaError_t kv_axpy_dev(cudaStream_t st, int64_t n, const T* x, T* y, const double* sc, int num, int den, double s);
template <typename T>
cudaError_t kv_cg_update(cudaStream_t st, int64_t n, const T* p, const T* q, T* x, T* r, const double* sc, int num,
                         int den);
template <typename T>
cudaError_t kv_xpby_dev(cudaStream_t st, int64_t n, const T* z, T* p, const double* sc, int num, int den, double s);
template <typename T>
cudaError_t kv_mul(cudaStream_t st, int64_t n, const T* d, const T* x, T* y);
template <typename T>
cudaError_t kv_recip(cudaStream_t st, int64_t n, T* d);
template <typename TI, typename TO>
cudaError_t kv_convert(cudaStream_t st, int64_t n, const TI* x, TO* y);
template <typename T>
cudaError_t kv_mask_zero(cudaStream_t st, int64_t nn, const uint8_t* bc, T* v);
cudaError_t kv_mask_keep(cudaStream_t st, int64_t nn, const uint8_t* bc, double* v);
cudaError_t kv_lift(cudaStream_t st, int64_t nn, const uint8_t* bc, double* v, const double* g, double s);
template <typename T>
cudaError_t kv_cheb(cudaStream_t st, int64_t n, double c1, double c2, const T* dinv, const T* r, T* d, T* x);
cudaError_t kv_uniform(cudaStream_t st, int64_t n, uint64_t seed, double* v);
template <typename TA, typename TB>
cudaError_t kv_dot(cudaStream_t st, int64_t n, const TA* x, const TB* y, double* part, double* out);
// out[j] = W_j . v for the k rows W_j = W + j ldw (length n), each summed in a
// fixed order; part: k * kv_multidot_parts() doubles
cudaError_t kv_multidot(cudaStream_t st, int k, int64_t n, const double* W, int64_t ldw, const double* v,
                        double* part, double* out);
int kv_multidot_parts();
// y += alpha sum_j c[j] W_j, c a device vector of k <= 256 entries
cudaError_t kv_gemv_rows(cudaStream_t st, int64_t n, int k, const double* W, int64_t ldw, const double* c,
                         double alpha, double* y);

// Assembled Q1 operator on a structured node lattice: 27 neighbour 3x3 blocks per
// node, stored [27][9][n_nodes].
// f32: sum the element blocks in float-float arithmetic on the FP32 pipes (current layout;
// the stencil stays FP64)
cudaError_t ks_assemble_q1(int Q, cudaStream_t st, int64_t ne, int nx, int ny, int nz, const uint8_t* bc,
                           const double* qd, int64_t qstride, int layout, const Tab1D* tab, double* A, int f32 = 0);
cudaError_t ks_apply(cudaStream_t st, int Nx, int Ny, int Nz, const uint8_t* bc, const double* A, const double* x,
                     double* y);
cudaError_t ks_diag(cudaStream_t st, int64_t nn, const uint8_t* bc, const double* A, double* d);
// general meshes: element 3x3 blocks of the Q1 operator at the fine points into
// COO slots [ne][8][8][9]; symbolic phase; slot sums; block-row apply and diagonal
cudaError_t ks_element_blocks_q1(int Q, cudaStream_t st, int64_t ne, const double* qd, int64_t qstride, int layout,
                                 const Tab1D* tab, double* coo);
void ks_coo_symbolic(int64_t ne, int64_t nn, const int* emap, std::vector<int64_t>& rowptr, std::vector<int>& col,
                     std::vector<int64_t>& jstart, std::vector<int64_t>& perm);
cudaError_t ks_coo_sum(cudaStream_t st, int64_t nnzb, const int64_t* jstart, const int64_t* perm, const double* coo,
                       double* val);
cudaError_t ks_bsr_apply(cudaStream_t st, int64_t nn, const int64_t* rowptr, const int* col, const double* val,
                         const uint8_t* bc, const double* x, double* y);
cudaError_t ks_bsr_diag(cudaStream_t st, int64_t nn, const int64_t* rowptr, const int* col, const double* val,
                        const uint8_t* bc, double* d);

// Jacobi-preconditioned CG on the assembled Q1 stencil in one cooperative
// launch (all blocks co-resident, bounded grid barriers, convergence tested on
// the device).  Solves A x = b from x = 0 (warm = 0) or from the given x
// (warm = 1, tolerance relative to ref = sqrt(b . D^-1 b)); stops when
// sqrt(r . z) <= rtol sqrt(r0 . z0) (tested every 4 iterations) or after maxit
// iterations.  Work vectors
// r, z, p, q of 3 n_nodes doubles; part: 2 * ks_pcg_max_blocks() doubles;
// bar: 2 unsigned; out[0] = iterations, out[1] = 1 if a residual was not finite.
struct KsPcg {
  int Nx, Ny, Nz;
  const uint8_t* bc;
  const double *A, *dinv, *b;
  double *x, *r, *z, *p, *q;
  double* part;
  unsigned* bar;
  double* out;
  double rtol, ref;
  int maxit, warm;
  int* err;
};
int ks_pcg_max_blocks();
// failure-detection test: a cooperative launch whose grid barrier one block skips
cudaError_t ks_wait_timeout_grid(cudaStream_t st, unsigned* bar, int* err);

// Geometric multigrid on the Q1 vertex lattice (nh_hmg.cu): coarse Dirichlet bits
// (node 2I of the finer lattice), Galerkin coarse stencil P^T A P, damped Jacobi
// sweep, residual, restriction P^T, prolongation x_f += P x_c, dense x = M b.
cudaError_t hm_coarse_bc(cudaStream_t st, int Nfx, int Nfy, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                         uint8_t* bcc);
cudaError_t hm_rap(cudaStream_t st, int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                   const uint8_t* bcc, const double* Af, double* Ac);
cudaError_t hm_jacobi(cudaStream_t st, int Nx, int Ny, int Nz, const uint8_t* bc, const double* A, const double* dinv,
                      const double* b, const double* xin, double* xout, double omega, int zero_in);
cudaError_t hm_resid(cudaStream_t st, int Nx, int Ny, int Nz, const uint8_t* bc, const double* A, const double* b,
                     const double* x, double* r);
cudaError_t hm_restrict(cudaStream_t st, int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                        const uint8_t* bcc, const double* rf, double* bcv);
cudaError_t hm_prolong_add(cudaStream_t st, int Nfx, int Nfy, int Nfz, int Ncx, int Ncy, int Ncz, const uint8_t* bcf,
                           const uint8_t* bcc, const double* xc, double* xf);
cudaError_t hm_dense_mv(cudaStream_t st, int n, const double* M, const double* b, double* x);
cudaError_t ks_pcg(cudaStream_t st, const KsPcg& a);

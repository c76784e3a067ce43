// Internal declarations of the nh library: handles, 1-D basis tables and the
// per-(P,Q) kernel launchers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nh.h"

#define NH_MAXP 5   // nodes per direction (p <= 4)
#define NH_MAXQ 6   // Gauss points per direction

// elements per block of the fused element kernels (about 128 threads, Q*Q per element)
__host__ __device__ constexpr int nh_layout_scalars(int layout) {
  return layout == NH_LAYOUT_CURRENT ? 17 : layout == NH_LAYOUT_INITIAL ? 27 : 32;
}
__host__ __device__ constexpr int nh_epb(int Q) { return (128 / (Q * Q)) > 0 ? 128 / (Q * Q) : 1; }
// Blocked FP32 quadrature data: per batch of EPB elements, Q z-planes of
// NP = EPB Q^2 points, each plane padded to a multiple of 4 floats (16 bytes, for
// the bulk copies).  Within a plane, point p (element-major, then y, x) keeps its
// first 4 (S/4) scalars as S/4 contiguous 16-byte chunks at [p][S/4][4], chunk k
// in slot (k + nh_f32_rot(S, p)) mod S/4 -- a per-point rotation that puts the 8
// lanes of one 16-byte shared load on distinct banks -- and its last S mod 4
// scalars at [NP][S mod 4] after all points' chunks.
// Direct form (nh_f32_direct(q)): the FP32 apply loads its quadrature data from
// global memory straight into registers; a plane is then scalar-major,
// [S][NPP] with NPP = NP rounded up to 32 points, so that each warp load of one
// scalar reads 128 contiguous bytes.  Taken for the q whose bit is set in
// NH_F32_DIRECT_QMASK, or for every q with NH_F32_DIRECT = 1.  Measured at full
// size against the plane ring: q = 3 +4.5%, q = 5 equal (with the vector gather
// of node lines in both), q = 4 -3%; so q = 3 only.
#ifndef NH_F32_DIRECT
#define NH_F32_DIRECT 0
#endif
#ifndef NH_F32_DIRECT_QMASK
#define NH_F32_DIRECT_QMASK (1 << 3)
#endif
__host__ __device__ constexpr bool nh_f32_direct(int Q) { return NH_F32_DIRECT || ((NH_F32_DIRECT_QMASK >> Q) & 1); }
__host__ __device__ constexpr int nh_f32_npp(int Q) { return (nh_epb(Q) * Q * Q + 31) / 32 * 32; }
__host__ __device__ constexpr long long nh_f32_plane_floats(int Q, int S) {
  return nh_f32_direct(Q) ? (long long)S * nh_f32_npp(Q) : ((long long)S * nh_epb(Q) * Q * Q + 3) / 4 * 4;
}
__host__ __device__ constexpr long long nh_f32_batch_floats(int Q, int S) { return (long long)Q * nh_f32_plane_floats(Q, S); }
__host__ __device__ constexpr int nh_f32_rot(int S, int p) { return S / 4 == 4 ? ((p & 7) >> 1) : ((p & 7) >> 2); }

// ---- 1-D tables ---------------------------------------------------------------
// Host-side tabulations in double; kernels receive them by value as kernel
// parameters (constant bank), converted to the kernel's scalar type.
struct Tab1D {
  int P, Q;
  double B[NH_MAXQ][NH_MAXP];    // GLL Lagrange basis at Gauss points (B_I)
  double G[NH_MAXQ][NH_MAXP];    // its derivative (B_xi)
  double D[NH_MAXQ][NH_MAXQ];    // collocated derivative B_xi B_I^+ (Sec. II-B)
  double w[NH_MAXQ];             // Gauss weights
};

// 1-D rules and Lagrange tabulation (nh_basis.cu)
void nh_gauss(int q, double* x, double* w);
void nh_lobatto(int n, double* x);
// Q_p element restriction and node coordinates of a conforming hexahedral mesh;
// returns an error message, empty on success (nh_mesh.cu).
std::string nh_hex_numbering(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int p,
                             std::vector<int>& emap, std::vector<double>& coords, int64_t& n_nodes);
// true when two spaces discretise the same mesh (box dimensions and vertices, or hex connectivity)
bool nh_same_mesh(nh_space a, nh_space b);
// Z-order of the elements by centroid: perm[k] = element placed k-th (nh_mesh.cu)
void nh_hex_morton(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int64_t* perm);
void nh_lagrange(int n, const double* nodes, int m, const double* pts, double* val, double* der);
void nh_tabulate(int p, int q, Tab1D* t);

template <int P, int Q, typename T>
struct KTab {
  T B[Q][P];
  T D[Q][Q];
};

template <int P, int Q, typename T>
inline KTab<P, Q, T> make_ktab(const Tab1D& t) {
  KTab<P, Q, T> k;
  for (int i = 0; i < Q; i++)
    for (int j = 0; j < P; j++) k.B[i][j] = (T)t.B[i][j];
  for (int i = 0; i < Q; i++)
    for (int j = 0; j < Q; j++) k.D[i][j] = (T)t.D[i][j];
  return k;
}

// ---- handles -------------------------------------------------------------------
struct nh_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 148;
  std::string err;
  int64_t launches = 0;
  // scratch for reductions (library owned)
  double* red = nullptr;               // partial sums + result slot
  size_t red_len = 0;
  double* red_host = nullptr;          // pinned
  unsigned long long* minj = nullptr;  // ordered-bits min of det F
  int* dev_err = nullptr;              // set by a kernel whose bounded wait expired
  // kernel timing (nh_profile_*)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;   // 2 per recorded launch
  size_t ev_used = 0;
  // host-buffer apply pipeline: upload and download streams, per-chunk events
  cudaStream_t s_in = nullptr, s_out = nullptr, s_k2 = nullptr;  // host apply: upload, download, second kernel stream
  std::vector<cudaEvent_t> ev_chunk;  // 2 per chunk (uploaded, computed)
};

struct nh_space_s {
  nh_ctx ctx = nullptr;
  int nx = 0, ny = 0, nz = 0, p = 0, q = 0, P = 0, Q = 0;
  int64_t ne = 0, n_nodes = 0, n_dof = 0;
  int Nx = 0, Ny = 0, Nz = 0;     // node lattice dims
  Tab1D tab;
  int* emap = nullptr;            // [ne][P^3] element restriction
  double* coords = nullptr;       // [n_nodes][3] device
  std::vector<double> coords_host;
  std::vector<double> verts_host; // [(nx+1)(ny+1)(nz+1)][3], empty for the unit cube; hex: [nv][3]
  bool hex = false;               // built by nh_space_hex (unstructured); nx = ny = nz = 0
  std::vector<int64_t> hex8_host; // hex: [ne][8] vertex ids
  std::vector<int> emap_host;     // hex: [ne][P^3] copy of emap (coarse Dirichlet masks)
  std::vector<int64_t> hex_need;  // hex: 1 + largest node id of elements [0, e] (du prefix they read)
  std::vector<int64_t> hex_fin;   // hex: smallest node id of elements [e, ne) (y below it is final)
  uint64_t mesh_hash = 0;         // FNV-1a of the mesh (dimensions or connectivity, and vertices)
  uint8_t* bc = nullptr;          // [n_nodes] bit c set = component c constrained (device)
  unsigned* emapb = nullptr;      // [ne][P^3] node id | constrained bits << 29 (FP32 apply)
  double* inv_mult = nullptr;     // [n_nodes] 1 / multiplicity
  float* inv_mult_f = nullptr;
  int64_t n_constrained = 0;
};

struct nh_op_s {
  nh_space space = nullptr;       // space this operator acts on
  nh_op parent = nullptr;         // fine operator whose qdata is shared (coarse levels)
  int layout = 0;
  int S = 17;                     // scalars per quadrature point
  double nu = 0.3;
  double* lam = nullptr;          // [ne] device
  double* mu = nullptr;
  double* qd = nullptr;           // [S][ne*Q^3] FP64 quadrature data (fine op only)
  float* qd_f = nullptr;          // FP32 copy, blocked per element batch (nh_f32_batch_floats)
  float* qd_ff = nullptr;         // float-float pairs (h, l), same indexing as qd (NH_F64X)
  double* u_state = nullptr;      // copy of the u of the last nh_qdata_setup (rediscretised levels)
  double* geom = nullptr;         // [10][ne*Q^3] grad_X xi and det(dX/dxi) per point (fine op only)
  bool geom_valid = false;
  int scatter = 0;                // E^T of the applies: 0 = atomic scatter-add, 1 = eight-colour passes
  bool qd_ff_valid = false;
  bool have_qd = false;
  bool qd_f_valid = false;
  // device staging for nh_jacobian_apply_host
  void* hbuf_in = nullptr;
  void* hbuf_out = nullptr;
  size_t hbuf_bytes = 0;
};

// ---- error helpers -------------------------------------------------------------
nh_status nh_fail(nh_ctx ctx, nh_status st, const std::string& msg);
nh_status nh_cuda_check(nh_ctx ctx, cudaError_t e, const char* what);
#define NH_CUDA(ctx, call)                                        \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return nh_cuda_check(ctx, _e, #call);  \
  } while (0)

// ---- kernel launchers (nh_operator.cu, one object per P) -------------------------
struct OpArgs {
  int64_t ne;
  const int* emap;
  const unsigned* emapb;  // element map with the Dirichlet bits packed in (node id < 2^29)
  const uint8_t* bc;
  const void* qd;      // quadrature data of the prec type
  int64_t qstride;     // ne * Q^3
  const void* in;      // du (apply) / u (setup, residual)
  void* out;           // y / r / diag
  const double* coords;
  const double* gbc;
  const double* lam;
  const double* mu;
  double* qd_out;      // setup: FP64 quadrature data to write (nullable)
  unsigned long long* minj;
  int layout;
  int prec;            // nh_prec of in/out vectors (apply, diagonal)
  int store;           // setup: write quadrature data
  int resid;           // setup: compute residual
  int lift;            // apply: keep constrained inputs, leave constrained rows zero
  int nx;              // elements along x of the (box) space
  int ny, nz;          // elements along y, z (box)
  int colour;          // apply: -1 = atomic scatter; 0..7 = the parity class of the eight-colour scatter
  int* err;            // device error flag for bounded waits
  const Tab1D* tab;
  double* geom;        // setup: geometry factors kept per point (nullable)
  int geom_mode;       // setup: 1 = compute and keep them in geom, 2 = read them
};

// Return cudaErrorInvalidValue if (P, Q) is outside the compiled set.
cudaError_t nh_launch_apply(int P, int Q, nh_prec prec, const OpArgs& a, cudaStream_t s);
cudaError_t nh_launch_setup(int P, int Q, const OpArgs& a, cudaStream_t s);
cudaError_t nh_launch_diag(int P, int Q, const OpArgs& a, cudaStream_t s);

#define NH_DECLARE_P(PP)                                                                  \
  cudaError_t nh_launch_apply_P##PP(int Q, nh_prec prec, const OpArgs& a, cudaStream_t s); \
  cudaError_t nh_launch_setup_P##PP(int Q, const OpArgs& a, cudaStream_t s);              \
  cudaError_t nh_launch_diag_P##PP(int Q, const OpArgs& a, cudaStream_t s);
NH_DECLARE_P(2)
NH_DECLARE_P(3)
NH_DECLARE_P(4)
NH_DECLARE_P(5)

// y = J_full x on unconstrained rows, 0 on constrained rows, constrained inputs kept
// (lifting of a Dirichlet increment); FP64 (nh_api.cu)
nh_status nh_jacobian_apply_lift(nh_op op, const double* x, double* y);

// transfer with the ABI's checks (nh_api.cu); dir 0 = prolong, 1 = restrict
nh_status nh_transfer_internal(nh_space c, nh_space f, nh_prec prec, int dir, const void* in, void* out);

// transfer (nh_transfer.cu)
cudaError_t nh_launch_transfer(int Pc, int Pf, nh_prec prec, int restrict_dir, int64_t ne,
                               const int* emap_c, const int* emap_f, const double* inv_mult,
                               const float* inv_mult_f, const void* in, void* out,
                               const double* ctof /* [Pf][Pc] */, cudaStream_t s);

// vector kernels (nh_vector.cu)
cudaError_t nh_launch_dot_partials(int64_t n, const double* x, const double* y, double* partials,
                                   int nblocks, cudaStream_t s);
cudaError_t nh_launch_sum_partials(const double* partials, int nblocks, double* out, cudaStream_t s);
cudaError_t nh_launch_f64_to_f32(int64_t n, const double* x, float* y, cudaStream_t s);
// FP64 -> float-float pairs (h, l) elementwise
cudaError_t nh_launch_setup_pts(int PF, int QC, int layout, cudaStream_t s, int64_t ne, const int* emap,
                                const double* coords, const double* u, const double* lam, const double* mu, double* qd,
                                int64_t qstride, unsigned long long* minj);
cudaError_t nh_launch_wait_timeout_mbar(cudaStream_t s, int* err);
cudaError_t nh_launch_pack_emap(cudaStream_t s, int64_t n, const int* emap, const uint8_t* bc, unsigned* out);
cudaError_t nh_launch_f64_to_ff(int64_t n, const double* x, float* y2, cudaStream_t s);
// FP64 SoA quadrature data [S][ne Q^3] -> blocked FP32 [batch][S][EPB][Q^3]
cudaError_t nh_launch_f32_blocked(int Q, int S, int64_t ne, const double* qd, float* qdf, cudaStream_t s);

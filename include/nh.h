/*
 * nh.h -- C ABI of the matrix-free Neo-Hookean operator library for B300 (sm_103a).
 *
 * The library applies the operators of compressible Neo-Hookean
 * hyperelasticity on continuous Q_p hexahedral spaces in the decomposition
 * A = P^T E^T B^T D B E P of arXiv 2204.01722 (Sec. II-C, Eq.
 * libceed_representation): element restriction E, tensor-product basis B,
 * pointwise quadrature function D.  On one GPU the parallel restriction P is
 * the identity, so T-vectors and L-vectors coincide.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Vectors are caller-owned DEVICE pointers unless a name ends in _host.
 *   The library never frees them.  Layout: node-major interleaved
 *   [n_nodes][3] (x, y, z displacement components), nodes numbered
 *   lexicographically over the (p nx + 1)(p ny + 1)(p nz + 1) lattice with x
 *   fastest.  Vectors cover every DoF, constrained ones included.
 * - NH_F64 entry points take double vectors, NH_F32 entry points take float
 *   vectors.  Device pointers must be 16-byte aligned (torch allocations are).
 * - Every call is stream-ordered on the context stream and does not block
 *   the host, except those returning host scalars (documented per call).
 * - Argument errors return at once (NH_ERR_ARG, NH_ERR_UNSUPPORTED) and
 *   launch nothing.  Asynchronous device errors are returned by the next
 *   call that synchronises, or by nh_sync.  nh_last_error gives the text.
 * - Handles (ctx, space, op) are owned by the caller through create/destroy;
 *   the library owns every internal device buffer (maps, qdata, scratch).
 * - Dirichlet convention: the Jacobian acts as the identity on constrained
 *   DoFs and drops constrained columns; the residual returns u - g there.
 * - Not thread-safe per context: calls on one context must be serialised.
 */
#ifndef NH_H
#define NH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nh_ctx_s* nh_ctx;
typedef struct nh_space_s* nh_space;
typedef struct nh_op_s* nh_op;

typedef enum {
  NH_OK = 0,
  NH_ERR_ARG = 1,            /* invalid argument (null handle, bad size, misaligned pointer) */
  NH_ERR_CUDA = 2,           /* a CUDA runtime call failed; see nh_last_error */
  NH_ERR_OOM = 3,            /* device allocation failed */
  NH_ERR_INVERTED = 4,       /* det F <= 0 (or not finite) at some quadrature point */
  NH_ERR_NOT_CONVERGED = 5,  /* a solver hit its iteration limit; the report is filled */
  NH_ERR_NAN = 6,            /* a NaN/Inf appeared in a solver scalar */
  NH_ERR_TIMEOUT = 7,        /* a bounded device wait expired */
  NH_ERR_STATE = 8,          /* call out of order (e.g. apply before nh_qdata_setup) */
  NH_ERR_UNSUPPORTED = 9     /* (p, q) or layout outside the compiled set */
} nh_status;

/* NH_F64X: FP64 vectors in and out, arithmetic in float-float (pairs of FP32
 * with about 48 significant bits) on the FP32 pipes, which B300 runs at 64 times
 * its FP64 FMA rate; results agree with NH_F64 to ~1e-13.  The quadrature data
 * are converted to float pairs on first use.  Accepted by nh_jacobian_apply and
 * nh_jacobian_apply_host only. */
typedef enum { NH_F64 = 0, NH_F32 = 1, NH_F64X = 2 } nh_prec;

/* Stored quadrature data.  NH_LAYOUT_CURRENT is the paper's 17 scalars per
 * point (Sec. III-B and Table different-storage "current"): grad_x xi (9),
 * W tau (6), W lambda, W (mu - lambda log J).  NH_LAYOUT_INITIAL stores the
 * initial-configuration data of Table different-storage "initial tuned" with
 * the material folded in (27 scalars): grad_X xi (9), H = grad_X u (9),
 * C^-1 (6), W mu, W lambda log J, W lambda; its Jacobian is
 * dP = dF S + F dS (Sec. V-E).  NH_LAYOUT_TAPE is the AD-style storage of
 * Table different-storage "initial AD": the residual's by-products kept for a
 * split forward-mode tangent that performs no constitutive evaluation (32
 * scalars): grad_X xi (9), H (9), W S (6), and the tangent's tape C^-1 (6),
 * W lambda, 2 W (mu - lambda log J); the same Jacobian as NH_LAYOUT_INITIAL. */
typedef enum { NH_LAYOUT_CURRENT = 0, NH_LAYOUT_INITIAL = 1, NH_LAYOUT_TAPE = 2 } nh_layout;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on (borrowed, not destroyed), or NULL to create a private
 * non-blocking stream.  Errors: NH_ERR_ARG (null out), NH_ERR_CUDA, NH_ERR_OOM. */
nh_status nh_create(nh_ctx* out, int device, void* cuda_stream);
nh_status nh_destroy(nh_ctx ctx);
/* Text of the last error on this context (storage owned by the context). */
const char* nh_last_error(nh_ctx ctx);
/* Block until the context stream is idle; returns any latched device error. */
nh_status nh_sync(nh_ctx ctx);
/* Failure-detection test hook (no counterpart in the paper): launches a kernel
 * whose bounded wait cannot complete -- kind 0: an mbarrier that no copy
 * arrives on (the wait of the FP32 apply's staged loads); kind 1: a grid
 * barrier that one block of a cooperative launch skips (the coarse PCG's
 * barrier) -- with a short poll limit.  The wait gives up, sets the device error
 * flag and the kernel returns; the next nh_sync returns NH_ERR_TIMEOUT and clears
 * the flag, and the context stays usable.  Errors: NH_ERR_ARG (kind). */
nh_status nh_debug_wait_timeout(nh_ctx ctx, int kind);
/* Number of kernels this context has launched since creation. */
int64_t nh_launch_count(nh_ctx ctx);

/* ---- spaces: mesh + element restriction + basis (Sec. II-B) ------------ */

/* Structured box of nx*ny*nz hexahedra with a trilinear geometry.
 * vertex_xyz: HOST array [(nx+1)(ny+1)(nz+1)][3], x fastest, or NULL for the
 * unit cube.  p: polynomial order (1..4); q: Gauss points per direction,
 * p+1 <= q <= 6.  Lagrange nodes are Gauss-Lobatto (GLL).  Outputs the node
 * and DoF counts.  Copies the mesh to the device; builds the element
 * restriction E as an int32 map [n_elem][(p+1)^3] and the node coordinates
 * (trilinear image of the GLL lattice).  Synchronises.
 * Errors: NH_ERR_ARG, NH_ERR_UNSUPPORTED (also when the node count reaches
 * 2^29: the FP32 apply packs the Dirichlet bits into the top three bits of
 * a second copy of E), NH_ERR_OOM. */
nh_status nh_space_box(nh_ctx ctx, int nx, int ny, int nz, const double* vertex_xyz,
                       int p, int q, nh_space* out, int64_t* n_nodes, int64_t* n_dof);
/* Unstructured conforming hexahedral mesh with a trilinear geometry (Sec. II-B:
 * the element restriction E of a general mesh; the paper's Schwarz-P and
 * extruded meshes are of this kind).  xyz: HOST [nv][3] vertex coordinates;
 * hex8: HOST [ne][8] vertex ids, vertex v of an element at the corner
 * (v & 1, (v >> 1) & 1, v >> 2) of the reference cube (tensor order; VTK's
 * hexahedron order 0 1 2 3 4 5 6 7 is 0 1 3 2 4 5 7 6 here).  p, q as for
 * nh_space_box.  Node numbering: vertices, edge, face and element interiors
 * identified by their global vertex ids (edges numbered from the smaller id,
 * faces in a frame anchored at their smallest corner id), ids handed out in
 * order of first touch over the elements.  Validates: ids in range and distinct
 * per element, a positive Jacobian at every corner, no face shared by more than
 * two elements, and equal coordinates for every shared node (conformity).
 * Spaces of lower order on the same xyz/hex8 are the p-multigrid levels.
 * Synchronises.  Errors: NH_ERR_ARG (with the reason in nh_last_error),
 * NH_ERR_UNSUPPORTED (orders, or 2^29 nodes), NH_ERR_OOM. */
nh_status nh_space_hex(nh_ctx ctx, int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int p, int q,
                       nh_space* out, int64_t* n_nodes, int64_t* n_dof);
/* Host only, no device or context needed: the node numbering and coordinates
 * nh_space_hex builds for (xyz, hex8, p), for inspection and mesh tooling.
 * Writes *n_nodes; with emap (HOST [ne][(p+1)^3] int32) and coords (HOST
 * [n_nodes][3]) non-NULL also the element map and the node coordinates (call
 * first with both NULL to size them).  On failure err (if non-NULL) receives
 * the reason, up to err_len bytes.  Errors: NH_ERR_ARG (invalid mesh),
 * NH_ERR_UNSUPPORTED (p outside 1..4, or 2^29 nodes). */
nh_status nh_hex_mesh_numbering(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int p,
                                int64_t* n_nodes, int* emap, double* coords, char* err, int64_t err_len);
/* Host only: the 3x3 block-row pattern of the Q1 COO assembly (the symbolic
 * phase of nh_op_assemble_q1) for an element map emap [ne][8] over n_nodes
 * nodes.  Writes *nnzb; with rowptr (HOST [n_nodes + 1] int64) and col (HOST
 * [nnzb] int32) non-NULL also the pattern, columns sorted per row.
 * Errors: NH_ERR_ARG (ids outside [0, n_nodes)). */
nh_status nh_q1_block_pattern(int64_t ne, int64_t n_nodes, const int* emap, int64_t* nnzb, int64_t* rowptr, int* col);
/* Host only: an element order for locality.  perm (HOST [ne]) receives the
 * elements sorted along a Z-order (Morton) curve through their centroids
 * (21 bits per axis of the bounding box): perm[k] is the element to place k-th.
 * Building the space from hex8 rows in that order (and per-element data in the
 * same order) makes neighbouring elements, and through the first-touch
 * numbering their nodes, neighbours in memory.  Errors: NH_ERR_ARG. */
nh_status nh_hex_morton_order(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int64_t* perm);
/* Node coordinates, HOST out [n_nodes][3]. */
nh_status nh_space_coords(nh_space s, double* xyz_host);
/* Dirichlet DoFs: HOST array [n_dof], nonzero = constrained.  Copied; synchronises. */
nh_status nh_space_set_dirichlet(nh_space s, const uint8_t* dof_mask_host);
nh_status nh_space_destroy(nh_space s);

/* ---- operators (Sec. II-A, II-B, III-B) -------------------------------- */

/* Neo-Hookean operator on `fine`.  Young's modulus per element from the HOST
 * array E_per_elem [n_elem], or the constant E when it is NULL; Poisson
 * ratio nu in (-1, 0.5).  layout: nh_layout.  Allocates the FP64 quadrature
 * data (S * n_elem * q^3 doubles).  Errors: NH_ERR_ARG, NH_ERR_UNSUPPORTED,
 * NH_ERR_OOM. */
nh_status nh_op_create(nh_space fine, double nu, const double* E_per_elem, double E,
                       int layout, nh_op* out);
/* Galerkin coarse operator on `coarse` (same mesh, lower p, same q) that
 * shares the fine operator's quadrature data: coarse basis tabulated at the
 * fine quadrature points, an exact Galerkin coarse operator (Sec. III-B).
 * The fine operator must outlive it. */
nh_status nh_op_level(nh_op fine, nh_space coarse, nh_op* out);
nh_status nh_op_destroy(nh_op op);
/* Scalars per quadrature point and bytes of stored quadrature data for prec. */
nh_status nh_op_info(nh_op op, nh_prec prec, int* scalars_per_qp, int64_t* qdata_bytes);

/* Quadrature data from the displacement u (device, double [n_dof]): F, J,
 * log J (from the invariants of H, so log1p does not cancel), tau, grad_x xi,
 * W (Eq. Kirchhoff-stress, Sec. III-B), always in FP64; an FP32 copy is made
 * on first FP32 use.  Writes min det F over all points to *min_J (HOST;
 * this call synchronises).  Returns NH_ERR_INVERTED if min det F <= 0 or is
 * not finite (the stored data are then invalid).  The first call (or the first
 * nh_residual) also keeps the mesh's geometry factors grad_X xi and
 * det(dX/dxi) per point on the operator (80 bytes per point, FP64); later calls
 * read them instead of recomputing them from the coordinates, with the same
 * values.  Without memory for them every call recomputes.
 * Errors: NH_ERR_ARG, NH_ERR_STATE (coarse op). */
nh_status nh_qdata_setup(nh_op op, const double* u, double* min_J);

/* Rediscretised coarse operator (Sec. III-B: the alternative to the exact
 * Galerkin levels, re-evaluating the nonlinearity on a smaller set of
 * quadrature points): an operator on `coarse` (same mesh and layout, p_c <= p_f,
 * its own q, typically p_c + 1) owning its quadrature data [S][n_elem q_c^3]
 * and a copy of the fine per-element material.  Synchronises.
 * Errors: NH_ERR_ARG (not the fine operator, different mesh), NH_ERR_OOM. */
nh_status nh_op_rediscretize(nh_op fine, nh_space coarse, nh_op* out);
/* Quadrature data of a rediscretised operator from the fine state: the fine
 * displacement u_fine (device L-vector of the fine space, 16-byte aligned) and
 * geometry are evaluated at the coarse Gauss points with the fine basis, then
 * F, J, log J, tau and grad_x xi (or the initial layout) as in nh_qdata_setup.
 * min_J (HOST out, nullable) = min det F over the coarse points.  Synchronises.
 * Errors: NH_ERR_ARG, NH_ERR_INVERTED (min det F <= 0). */
nh_status nh_qdata_setup_rediscretized(nh_op op, nh_op fine, const double* u_fine, double* min_J);

/* Residual r = F(u) (Eq. residual-discrete-ref with f_1 = tau, f_0 = 0):
 * sum_e E^T B_xi^T W tau (grad_x xi)^T; constrained rows r = u - g_bc.
 * g_bc may be NULL (zero).  FP64 device vectors; does not touch the stored
 * quadrature data (it reads or keeps the geometry factors as nh_qdata_setup).
 * Errors: NH_ERR_ARG, NH_ERR_STATE (coarse op). */
nh_status nh_residual(nh_op op, const double* u, const double* g_bc, double* r);

/* Jacobian action y = J du (Eq. Jacobian-discrete-ref with Eqs. dtau and
 * depsilon): fused gather E, sum-factorised collocated gradient, pointwise
 * linearised stress from stored quadrature data, transposed contractions
 * and scatter-add E^T.  du and y: device [n_dof] of prec type, must not
 * alias.  Errors: NH_ERR_ARG, NH_ERR_STATE (no quadrature data yet). */
nh_status nh_jacobian_apply(nh_op op, nh_prec prec, const void* du, void* y);
/* Same, with HOST du_host and y_host (pinned memory recommended): copies in,
 * applies, copies out through library-owned device buffers; synchronises.  The
 * apply runs in up to 8 chunks of z-layers of the box: a chunk's du node layers
 * are uploaded on one copy stream while the previous chunk computes, and node
 * layers that no later chunk touches are downloaded on another. */
nh_status nh_jacobian_apply_host(nh_op op, nh_prec prec, const void* du_host, void* y_host);

/* Diagonal of the assembled Jacobian for Jacobi smoothing (Sec. III-B):
 * diag[a,c] = sum_e sum_q sum_{d,d'} B_xi,d[q,a] D[q; c,d; c,d'] B_xi,d'[q,a];
 * 1 on constrained DoFs.  Device out [n_dof] of prec type, computed in that
 * precision's arithmetic (NH_F32: FP32, from the FP64 quadrature data). */
nh_status nh_jacobian_diagonal(nh_op op, nh_prec prec, void* diag);
/* Assembled operator on a Q1 (p = 1) space as 3x3 block rows (Sec. III-D: the
 * split-phase COO assembly that hands the coarse level to a sparse solver).
 * Symbolic phase on the host: COO entry (e, a, b) couples the element's nodes a
 * (row) and b (column); rows bucketed, columns sorted and made unique, every
 * entry listed under its block slot.  Numeric phase on the device: one block of
 * 64 threads per element computes its 8 x 8 blocks sum_q G_a^T D_q G_b from the
 * operator's quadrature data (a coarse level: the fine data at the fine points,
 * exact Galerkin), then one thread per slot entry sums the slot's COO entries
 * in a fixed order (no atomics, reproducible).  Call with rowptr = NULL to get
 * the block count in *nnzb; then with HOST arrays rowptr [n_nodes + 1] (int64),
 * col [nnzb] (node ids, sorted per row) and val [nnzb][3][3] (row-major block,
 * row component first).  Dirichlet convention applied: constrained rows are
 * identity rows, constrained columns zero.  The p-multigrid uses the same
 * assembly (kept on the device) for the Q1 level of nh_space_hex meshes.
 * Synchronises.  Errors: NH_ERR_UNSUPPORTED (p != 1), NH_ERR_STATE (no
 * quadrature data), NH_ERR_ARG, NH_ERR_OOM. */
nh_status nh_op_assemble_q1(nh_op op, int64_t* nnzb, int64_t* rowptr, int* col, double* val);

/* ---- p-multigrid transfer (Eq. mg_prolong) ----------------------------- */

/* uf = P uc, P = sum_e E_f^T Lambda(m_f^-1) B_ctof E_c, m_f = node multiplicity.
 * coarse and fine: same mesh, p_c < p_f.  Device vectors of prec type. */
nh_status nh_prolong(nh_space coarse, nh_space fine, nh_prec prec, const void* uc, void* uf);
/* rc = P^T rf (restriction = prolongation transposed, Sec. III-B). */
nh_status nh_restrict(nh_space fine, nh_space coarse, nh_prec prec, const void* rf, void* rc);

/* Scatter E^T of this operator's Jacobian applies (Sec. IV discusses the
 * atomic writes among the operator overheads).  mode 0 (default): one launch,
 * atomic scatter-add.  mode 1: eight launches, one per parity class of the box
 * mesh's elements -- FP64 and float-float: elements classed by the parities of
 * (ex, ey, ez); FP32: batches of the kernel's consecutive elements along x
 * classed by the parities of (batch x, ey, ez) -- with plain read-modify-writes
 * of y: no two elements (batches) of a class share a node, and within an FP32
 * batch the rows are summed in shared memory or the elements take turns.
 * Summation order is then fixed.  mode 1 needs a box mesh whose x-element count
 * is a multiple of the FP32 kernel's elements per block (14, 8, 5 for q = 3, 4,
 * 5), else NH_ERR_UNSUPPORTED.  Errors: NH_ERR_ARG. */
nh_status nh_op_set_scatter(nh_op op, int mode);

/* ---- kernel timing ----------------------------------------------------- */

/* When on, every Jacobian-apply kernel launch on this context is bracketed by
 * CUDA events on the context stream (up to 65536 launches are kept). */
nh_status nh_profile_enable(nh_ctx ctx, int on);
/* Total device time (ms) and number of Jacobian-apply kernels recorded since
 * the last read; clears the record.  Synchronises. */
nh_status nh_profile_read(nh_ctx ctx, double* total_ms, int64_t* launches);

/* Measured FMA throughput of this GPU (not part of the method): a kernel in
 * which every thread runs 8 independent fused multiply-add chains for `iters`
 * steps on 8 resident 256-thread blocks per SM, timed with CUDA events on the
 * context stream after one warm-up launch.  prec NH_F64 (DFMA) or NH_F32
 * (FFMA); *tflops = 2 x FMAs / time, *ms (optional) = the timed launch.  It is
 * the denominator of the FP64 and float-float applies' ALU rooflines.
 * Allocates and frees a small output buffer; synchronises.
 * Errors: NH_ERR_ARG (iters < 1, other prec), NH_ERR_CUDA. */
nh_status nh_fma_peak(nh_ctx ctx, nh_prec prec, int64_t iters, double* tflops, double* ms);

/* ---- vector kernels --------------------------------------------------- */

/* Deterministic FP64 dot product of two device double vectors of length n
 * (the Krylov inner products of Sec. III-A): per-block partial sums in
 * library scratch, then one fixed-order pass.  Result to *result_host (HOST;
 * synchronises). */
nh_status nh_dot(nh_ctx ctx, int64_t n, const double* x, const double* y, double* result_host);

/* ---- p-multigrid and the Newton-Krylov solve (Sec. III-A, III-B) -------- */

typedef struct nh_mg_s* nh_mg;

typedef struct {
  int n_levels;            /* levels including the fine one (2..8) */
  int level_p[8];          /* polynomial order per level, fine first, e.g. {4, 2, 1} */
  int cheb_degree;         /* Chebyshev smoother degree (paper: 2; default 3) */
  double cheb_lo, cheb_hi; /* target interval [lo, hi] * lambda_max (0.1, 1.1) */
  int lanczos_iters;       /* CG/Lanczos steps for lambda_max on a rough seed (10) */
  double coarse_rtol;      /* coarsest-level Jacobi-PCG relative tolerance, natural norm (1e-3) */
  int coarse_maxit;        /* (2000) */
  int coarse_assembled;    /* 1: a p = 1 coarsest level is assembled: a 27-point block stencil on
                              nh_space_box meshes, COO-assembled 3x3 block rows (nh_op_assemble_q1)
                              on nh_space_hex meshes; 0: applied matrix-free */
  int mixed;               /* 1: FP32 applies, smoothers and transfers on levels with p > 1 */
  uint64_t seed;           /* seed of the rough Lanczos start vector (splitmix64, uniform(-1, 1)) */
  int load_steps;          /* pseudo-time steps t_k = k / load_steps (1) */
  double newton_rtol;      /* stop when ||F(u)|| <= rtol ||F(u_k^0)||, u_k^0 = lifted start (1e-8) */
  double newton_atol;      /* or ||F(u)|| <= atol (1e-13) */
  int newton_maxit;        /* per load step (30) */
  double krylov_rtol;      /* FCG relative tolerance on sqrt(r^T M r) (1e-3) */
  int krylov_maxit;        /* (500) */
  int line_search;         /* 1: one secant step on F(u + a du)^T du = 0 (critical point) */
  int verbose;             /* 1: one line per Newton step on stderr */
  int learned_accept;      /* outer learned stage test: 0 = ||r - J z1||_2 < ||r||_2 (z1 as is);
                              1 = energy decrease with the optimal step a = z1.r / z1.J z1, i.e. z1.r > 0;
                              learned_mode 4 without a network: 1 = exact coarse space (see there) */
  int learned_mode;        /* where a network set by nh_mg_set_learned acts:
                              1 = outer FCG stage (predicts the fine error at the vertices);
                              2 = coarse warm start (predicts y ~ A_c^-1 r_c; the coarsest PCG, or the
                                  fixed polynomial with coarse_fixed, starts from a y, a = y.r_c / y.A_c y
                                  the step that minimises the A-norm error along y, when a > 0 and that
                                  start at least halves the residual's natural norm, else from zero);
                              3 = coarse post-correction: after the plain coarsest solve x1 (best with
                                  coarse_fixed), predicts the error A_c^-1 r1 it leaves from the scaled
                                  residual D_c^-1 r1, r1 = r_c - A_c x1, and adds a y,
                                  a = y.r1 / y.A_c y, when y.r1 > 0 and
                                  y.A_c y > 0 (the coarse A_c-norm error then strictly decreases);
                              4 = learned coarse space, built at every nh_mg_setup: for learned_vectors
                                  seeded probes r the network predicts the error A_c^-1 r1 that the plain
                                  coarsest solve x1 leaves (r1 = r - A_c x1); these predictions,
                                  A_c-orthonormalised, form W, and the coarsest solve becomes the two-level
                                  balancing map x = W W^T b + (I - W W^T A_c) Q (I - A_c W W^T) b around
                                  the plain coarsest solve Q: linear, symmetric positive definite, fixed
                                  between setups.  With no network set, W is built from the probes' x1
                                  (the same construction without the learned part), or, with
                                  learned_accept = 1, from the exact errors A_c^-1 r1 (coarse PCG to
                                  1e-9 per probe: the space a perfect network would give) */
  int fp64_kind;           /* arithmetic of the FP64-accurate matrix-free applies (outer FCG, Lanczos,
                              FP64 smoothers): 0 = native FP64 (NH_F64), 1 = float-float (NH_F64X) */
  int coarse_rediscretize; /* 1: matrix-free coarse levels get their own Gauss rule q = p_l + 1 and
                              quadrature data re-evaluated from the fine state (nh_op_rediscretize);
                              0: exact Galerkin levels on the fine points (default).  An assembled
                              Q1 coarsest level is always built from the fine data. */
  int nonlinear;           /* 0: Newton-Krylov (FCG + V-cycle); 1: L-BFGS with one V-cycle of the load
                              step's tangent (set up after the predictor) as the initial inverse Hessian
                              (Sec. III-A); same line search, predictor and tolerances; at most
                              4 newton_maxit iterations per load step */
  int lbfgs_m;             /* L-BFGS history pairs (5), 1..32 */
  int coarse_solver;       /* assembled Q1 coarsest level: 0 = Jacobi-PCG (one cooperative kernel);
                              1 = PCG with a geometric multigrid V-cycle on the vertex lattice (Galerkin
                              P^T A P stencils, damped Jacobi, exact solve on 3^3 nodes), used when the
                              lattice halves evenly down to 3 nodes per direction and the coarsest
                              stencil is positive definite, else Jacobi-PCG; box meshes only
                              (NH_ERR_UNSUPPORTED from nh_mg_create on nh_space_hex meshes) */
  int coarse_fixed;        /* 0 (default): the coarsest solve is the PCG chosen by coarse_solver, stopped
                              at coarse_rtol, so its work and result depend on the residual and the
                              V-cycle is not a fixed operator.  k > 0: a fixed linear coarse solve
                              instead -- k steps of Chebyshev semi-iteration (Saad, Alg. 12.1) on the
                              coarsest level, preconditioned by its Jacobi diagonal (coarse_solver 0)
                              or by one geometric V-cycle (coarse_solver 1), over [l_min, cheb_hi l_max]
                              of the preconditioned operator, the extreme Ritz values of 20 (or
                              2 lanczos_iters, at most 60) preconditioned Lanczos steps at setup.  The
                              V-cycle is then a fixed symmetric positive definite operator (FCG(1)
                              reduces to PCG), and the coarse solve has no reductions and no host
                              synchronisation.  coarse_its counts k per coarse solve */
  int learned_vectors;     /* learned_mode 4: probes for the coarse space (32), 0..256 */
} nh_mg_opts;

typedef struct {
  int status;              /* nh_status of the solve */
  int load_steps, newton_its, krylov_its, vcycles, coarse_its;
  double rel_residual;     /* ||F(u)|| / ||F(u_k^0)|| at the end of the last load step */
  double abs_residual;
  double seconds;          /* wall time of the call */
  double t_setup, t_krylov, t_residual; /* qdata + multigrid setup, FCG, residuals + line search */
  int learned_accepted, learned_rejected;
} nh_solve_report;

/* Defaults: 3 levels {p, 2, 1} from the fine order (2 levels for p = 2), the
 * values in parentheses above. */
nh_status nh_mg_default_opts(nh_op fine, nh_mg_opts* out);
/* Build the hierarchy: coarse spaces on the same mesh with the fine q, their
 * Dirichlet DoFs taken face by face from the fine space (a face component is
 * constrained on the coarse level when it is constrained at every fine node of
 * that face), Galerkin coarse operators sharing the fine quadrature data
 * (nh_op_level), vectors in each level's precision. */
nh_status nh_mg_create(nh_op fine, const nh_mg_opts* opts, nh_mg* out);
/* From the fine operator's current quadrature data: diagonals, the assembled
 * coarse stencil, and lambda_max of D^-1 A on every level (FP64). Synchronises. */
nh_status nh_mg_setup(nh_mg mg);
/* Space, operator and lambda_max of level `level` (0 = fine); any out may be NULL. */
nh_status nh_mg_level_info(nh_mg mg, int level, nh_space* space, nh_op* op, double* lambda_max);
/* z = M r: one V-cycle (Algorithm multigrid_algorithm) with Chebyshev/Jacobi
 * pre- and post-smoothing, restriction = prolongation^T and a Jacobi-PCG
 * coarsest solve.  r, z: device double [n_dof] of the fine space. */
nh_status nh_mg_vcycle(nh_mg mg, const double* r, double* z);
nh_status nh_mg_destroy(nh_mg mg);
/* Flexible CG (Notay's FCG with truncation 1) on J x = b with the V-cycle as
 * preconditioner; x is the initial guess and the result.  norm: 0 = natural
 * norm sqrt(r^T M r), 1 = ||r||_2.  Returns NH_ERR_NOT_CONVERGED (report
 * filled) if maxit is reached. */
nh_status nh_linear_solve(nh_mg mg, const double* b, double* x, double rtol, int maxit, int norm,
                          nh_solve_report* report);
/* Load-stepped Newton-Krylov solve (Sec. III-A): for t_k = k / load_steps the
 * constrained DoFs of u are set to t_k g_bc, then Newton steps J du = -F(u)
 * solved by FCG + V-cycle to krylov_rtol, with the secant line search, until
 * the residual criterion holds.  u: device double [n_dof], initial guess in,
 * solution out.  g_bc: device double [n_dof], boundary values at t = 1.
 * Errors: NH_ERR_INVERTED, NH_ERR_NOT_CONVERGED, NH_ERR_NAN (report filled). */
nh_status nh_solve(nh_mg mg, const double* g_bc, double* u, nh_solve_report* report);

/* ---- learned coarse correction (not in the paper) ----------------------- */

typedef struct nh_net_s* nh_net;

/* A 3-D convolution U-Net on the Q1 vertex grid (N^3 nodes, N odd): input
 * 4 channels (restricted residual x, y, z scaled by its RMS, and log10 of the
 * node-averaged Young's modulus), output 3 channels (error estimate in the same
 * scaling).  `levels` resolutions N, (N-1)/2+1, ...; channels[l] in
 * {8, 16, 32, 48, 64}; 3x3x3 convolutions with zero padding, stride-2
 * vertex-centred downsampling, linear upsampling, additive skips, ReLU.
 * bf16 = 1: activations and weights in BF16, FP32 accumulation (0: FP32).
 * Weights He-normal from a splitmix64 stream of `seed`, biases zero.
 * Parameter layout: layers in network order, each W [Cout][Cin][27] (tap
 * kx + 3 (ky + 3 kz)) then b [Cout].  Fields are channel-major [C][N^3], x fastest. */
nh_status nh_net_create(nh_ctx ctx, int N, int levels, const int* channels, int bf16, uint64_t seed, nh_net* out);
nh_status nh_net_destroy(nh_net net);
/* BF16 networks: convolutions as implicit GEMMs on the tensor cores (on = 1,
 * the default) or on the CUDA cores (on = 0, FP32 FMAs on the BF16 values).
 * Tensor cores: forward mma.sync m16n8k16 (BF16 operands, FP32 accumulation;
 * the same FP32 sums as the CUDA-core path in another order, rounded to BF16);
 * input and weight gradients mma.sync m16n8k8 TF32 (the FP32 gradient fields
 * rounded to TF32, BF16 activations and weights exact; FP32 accumulation).
 * No effect on FP32 networks. */
nh_status nh_net_set_tensor_cores(nh_net net, int on);
nh_status nh_net_param_count(nh_net net, int64_t* count);
/* FP32 master parameters to / from HOST memory (set resets the Adam state). */
nh_status nh_net_get_params(nh_net net, float* host);
nh_status nh_net_set_params(nh_net net, const float* host);
/* out [3][N^3] = net(in [4][N^3]); device float pointers. */
nh_status nh_net_forward(nh_net net, const float* in, float* out);
/* Gradient of the relative squared error ||net(in) - target||^2 / ||target||^2
 * with respect to the parameters, to device float dparams [count]; the loss to
 * *loss (HOST, may be NULL; synchronises when given). */
nh_status nh_net_gradient(nh_net net, const float* in, const float* target, float* dparams, double* loss);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the mean loss of `batch`
 * samples in [batch][4][N^3] / [batch][3][N^3]. */
nh_status nh_net_train_step(nh_net net, int batch, const float* in, const float* target, float lr, double* loss);
/* Insert the network as an extra flexible-CG preconditioner stage of nh_solve /
 * nh_linear_solve (NULL removes it): z1 = a P net(R r) (R, P through the p levels
 * down to the Q1 level; a = 1, or the energy-optimal step, see learned_accept),
 * accepted by the opts' test, then z = z1 + V-cycle(r - J z1); otherwise
 * z = V-cycle(r).  Needs a hierarchy
 * ending at p = 1 whose vertex grid matches the network's N. */
nh_status nh_mg_set_learned(nh_mg mg, nh_net net);
/* Training pairs from the linear system J x = b at the current quadrature data.
 * learned_mode 1: solves to ||r|| <= 1e-10 ||b|| for x*, then runs FCG +
 * V-cycle to krylov_rtol from zero and, before every preconditioner
 * application, stores the network input for the residual r_k and the target
 * (x* - x_k injected at the vertex nodes, in the input's scaling).
 * learned_mode 2: runs FCG + V-cycle to krylov_rtol; at every coarsest solve
 * stores the input for the coarse right-hand side r_c and the target
 * A_c^-1 r_c (coarse PCG to 1e-9, in the input's scaling).
 * learned_mode 3 and 4: runs FCG + V-cycle to krylov_rtol; at every coarsest
 * solve stores the input for the residual r1 = r_c - A_c x1 left by the plain
 * coarsest solve x1 (the network sees D_c^-1 r1, scaled to unit RMS, and
 * log10 E) and the target A_c^-1 r1 (PCG to 1e-9) scaled to unit RMS: these
 * modes use only the prediction's direction.  The V-cycle continues with x1.
 * feats: device float
 * [max_pairs][4][N^3], targets [max_pairs][3][N^3]; *n_pairs = pairs written. */
nh_status nh_mg_collect(nh_mg mg, const double* b, int max_pairs, float* feats, float* targets, int* n_pairs);

/* ---- allocation-free variant ------------------------------------------ */

/* Largest n accepted by nh_dot_noalloc (2^28 elements). */
#define NH_DOT_NOALLOC_MAX_N ((int64_t)1 << 28)

/* Deterministic FP64 dot product that allocates nothing.  The paper has no
 * counterpart: this is a service for callers that cannot let a library call
 * cudaMalloc -- applications whose device memory is owned by their own pool
 * allocator (an allocation behind its back breaks the pool's budget or fails),
 * and latency-critical loops where cudaMalloc/cudaFree would synchronise the
 * device.  It needs no nh_ctx (nh_create itself allocates).
 * x, y: device double [n]; result: device double [1], caller-owned; all three
 * 8-byte aligned.  Runs on the current CUDA device, stream-ordered on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream); does not block
 * the host.  Summation order depends only on n (one partial sum per 8192
 * elements, then a fixed-order sum), so repeated calls give identical results.
 * Scratch: a fixed 256 KiB array in the library's device image, held by every
 * GPU that loads the library until the process exits; n > NH_DOT_NOALLOC_MAX_N
 * returns NH_ERR_UNSUPPORTED.  The scratch address is per CUDA context: the
 * first call in each context (the device's primary context, a fresh one after
 * cudaDeviceReset, or a driver-API context of the caller's) looks it up with
 * that context current and caches it under the context's id, so make that first
 * call before any stream capture; a process that meets more than 64 contexts
 * looks the address up on every call from then on.  All calls share the one
 * scratch array, which keeps the last call's partial sums (no slot needs
 * clearing: each call writes every slot it reads); calls that can overlap on
 * the GPU (two streams, two host threads) race and must be serialised by the
 * caller.
 * Errors: NH_ERR_ARG (n < 0, null or misaligned pointer), NH_ERR_UNSUPPORTED,
 * NH_ERR_CUDA (symbol lookup or one of this call's two launches failed; an error
 * left pending by earlier, unrelated work is neither reported nor cleared). */
nh_status nh_dot_noalloc(void* cuda_stream, int64_t n, const double* x, const double* y, double* result);

#ifdef __cplusplus
}
#endif
#endif /* NH_H */

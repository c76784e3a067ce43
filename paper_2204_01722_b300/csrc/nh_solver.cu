// p-multigrid preconditioner and the load-stepped Newton-Krylov solve
// (Sec. III-A, Sec. III-B, Algorithm multigrid_algorithm), orchestrated from the
// host; every vector operation is a kernel on the context stream.
//
// * Levels share the fine quadrature data (Galerkin coarse operators, Sec. III-B).
//   A p = 1 coarsest level is assembled into a 27-point block stencil once per
//   setup (nh_stencil.cu); other levels are matrix-free.
// * Smoother: Chebyshev semi-iteration on D^-1 A over [lo, hi] lambda_max
//   (Saad, Iterative Methods, Alg. 12.1), lambda_max from a few CG/Lanczos steps
//   on a rough seed.
// * Coarsest solve: Jacobi-PCG to a relative tolerance in the natural norm.
// * Outer Krylov: flexible CG with truncation 1 (Notay 2000), since a
//   preconditioner with an inner tolerance is not a fixed linear operator.
// * Mixed precision: levels with p > 1 keep FP32 vectors, FP32 quadrature data,
//   FP32 smoothers and transfers; the outer residual, dot products, eigenvalue
//   estimates, the coarsest solve and the Newton residual stay FP64.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "nh_krylov.cuh"
#include "nh_net.cuh"

namespace {

// device scalar slots
// (the coarsest PCG runs inside the V-cycle, i.e. inside an FCG step: the two
// must not share slots)
enum {
  S_RZ0 = 0, S_RZ1 = 1, S_PQ = 2,                   // PCG / Lanczos
  S_FPQ = 8, S_FPR = 9, S_FZQ = 10, S_FRR = 11,      // FCG
  S_TMP = 12,
  S_PCG = 14,             // cooperative coarse PCG: iterations, non-finite flag
  S_HIST = 16,            // Lanczos history: rz[k] at S_HIST + k, pq[k] at S_HIST + 64 + k
  S_LEN = S_HIST + 128
};

struct Level {
  nh_space space = nullptr;
  nh_op op = nullptr;
  bool own = false;        // space/op created by the hierarchy
  int p = 1;
  nh_prec prec = NH_F64;
  int64_t n = 0, nn = 0;
  // level-precision vectors
  void *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *t = nullptr, *dinv = nullptr;
  void* ct = nullptr;      // coarse-sized temporary in this level's precision (precision change)
  // FP64 work vectors (Lanczos, coarsest PCG)
  double *w[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* dinv64 = nullptr;
  double lmax = 0.0;
  double cmin = 0.0, cmax = 0.0;  // coarsest level, fixed solve: Chebyshev interval of M A
  bool stencil = false;
  bool redisc = false;     // rediscretised: own Gauss rule and quadrature data from the fine state
  double* A = nullptr;     // [27][9][nn]
  // assembled Q1 level of an unstructured mesh: 3x3 block rows (split-phase COO assembly)
  bool bsr = false;
  int64_t nnzb = 0;
  int64_t *rowptr = nullptr, *jstart = nullptr, *perm = nullptr;
  int* col = nullptr;
  double *coo = nullptr, *val = nullptr;
};

// one lattice of the geometric multigrid on the assembled Q1 level
struct HLevel {
  int Nx = 0, Ny = 0, Nz = 0;
  int64_t nn = 0;
  uint8_t* bc = nullptr;
  double *A = nullptr, *dinv = nullptr, *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
  bool own = false;  // level 0 borrows the p-multigrid's stencil, bits and diagonal
};

}  // namespace

struct nh_mg_s {
  nh_ctx ctx = nullptr;
  nh_op fine = nullptr;
  nh_mg_opts o;
  std::vector<Level> L;
  double* sc = nullptr;    // device scalars
  double* part = nullptr;  // dot partials
  double* hsc = nullptr;   // pinned host mirror
  std::vector<HLevel> H;           // geometric multigrid on the assembled Q1 level (coarse_solver 1)
  bool hmg_ok = false;             // its current setup succeeded (else the coarse solve is Jacobi-PCG)
  double* Hinv = nullptr;          // dense inverse on the coarsest lattice
  int Hn = 0;
  double* pcg_part = nullptr;      // coarse cooperative PCG: block partials
  unsigned* pcg_bar = nullptr;     // its grid barrier words
  // FCG / Newton work (fine, FP64)
  double *fr = nullptr, *fz = nullptr, *fp = nullptr, *fq = nullptr;  // FCG work
  double *fx = nullptr, *fu = nullptr, *fg = nullptr, *fb = nullptr, *ft = nullptr, *fs = nullptr;  // Newton
  double* fsave = nullptr;  // state at the start of a load increment
  std::vector<double*> lbs, lby;  // L-BFGS history: steps s_i and residual changes y_i (allocated on first use)
  double* lbr = nullptr;          // L-BFGS: residual at the previous iterate
  bool setup_done = false;
  nh_prec p64 = NH_F64;    // arithmetic of the FP64-accurate matrix-free applies
  int vcycles = 0, coarse_its = 0;
  // learned stage
  nh_net net = nullptr;
  float *feat = nullptr, *nout = nullptr, *logE = nullptr;
  double *lz1 = nullptr, *lw = nullptr, *lxs = nullptr, *lx = nullptr, *lt = nullptr;
  double *lc1 = nullptr, *lc2 = nullptr;  // coarse-sized: post-correction prediction, exact correction
  // coarse space of learned_mode 4: Wk A_c-orthonormal coarse vectors W_j = W + j n_c
  double *W = nullptr, *Wc = nullptr, *Wpart = nullptr;
  int Wk = 0, Wcap = 0;
  int acc = 0, rej = 0;
  struct Collect* coll = nullptr;  // coarse-pair collection in progress
};

namespace {

size_t wsize(nh_prec p) { return p == NH_F64 ? 8 : 4; }

#define CK(call)                                          \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return nh_cuda_check(mg->ctx, _e, #call); \
  } while (0)
#define ST(call)                         \
  do {                                   \
    nh_status _s = (call);               \
    if (_s != NH_OK) return _s;          \
  } while (0)

nh_status dalloc(nh_mg mg, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nh_fail(mg->ctx, NH_ERR_OOM, "nh_mg: device allocation failed");
  }
  return NH_OK;
}

// read device scalar slots [i0, i0 + k) to the host (synchronises)
nh_status read_sc(nh_mg mg, int i0, int k, double* out) {
  CK(cudaMemcpyAsync(mg->hsc, mg->sc + i0, sizeof(double) * k, cudaMemcpyDeviceToHost, mg->ctx->stream));
  CK(cudaStreamSynchronize(mg->ctx->stream));
  memcpy(out, mg->hsc, sizeof(double) * k);
  return NH_OK;
}

template <typename TA, typename TB>
nh_status dot(nh_mg mg, int64_t n, const TA* x, const TB* y, int slot) {
  CK((kv_dot<TA, TB>(mg->ctx->stream, n, x, y, mg->part, mg->sc + slot)));
  mg->ctx->launches += 2;
  return NH_OK;
}

nh_status dot_host(nh_mg mg, int64_t n, const double* x, const double* y, double* out) {
  ST(dot(mg, n, x, y, S_TMP));
  return read_sc(mg, S_TMP, 1, out);
}

// y = A_l x in precision prec (the stencil is FP64 only)
nh_status level_apply(nh_mg mg, Level& l, nh_prec prec, const void* x, void* y) {
  if (l.stencil && prec == NH_F64) {
    CK(ks_apply(mg->ctx->stream, l.space->Nx, l.space->Ny, l.space->Nz, l.space->bc, l.A, (const double*)x,
                (double*)y));
    mg->ctx->launches++;
    return NH_OK;
  }
  if (l.bsr && prec == NH_F64) {
    CK(ks_bsr_apply(mg->ctx->stream, l.nn, l.rowptr, l.col, l.val, l.space->bc, (const double*)x, (double*)y));
    mg->ctx->launches++;
    return NH_OK;
  }
  return nh_jacobian_apply(l.op, prec == NH_F64 ? mg->p64 : prec, x, y);
}

// --- smallest building blocks, templated on the level precision ----------------
template <typename T>
nh_status cheb(nh_mg mg, Level& l, T* x, const T* b, bool zero_init) {
  cudaStream_t st = mg->ctx->stream;
  const double a = mg->o.cheb_lo * l.lmax, bb = mg->o.cheb_hi * l.lmax;
  const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  T* r = (T*)l.r;
  T* d = (T*)l.d;
  T* t = (T*)l.t;
  const T* dinv = (const T*)l.dinv;
  const nh_prec pr = l.prec;
  if (zero_init) {
    CK(cudaMemcpyAsync(r, b, sizeof(T) * l.n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(x, 0, sizeof(T) * l.n, st));
  } else {
    ST(level_apply(mg, l, pr, x, r));
    CK(kv_axpby<T>(st, l.n, 1.0, b, -1.0, r));  // r = b - A x
    mg->ctx->launches++;
  }
  CK(cudaMemsetAsync(d, 0, sizeof(T) * l.n, st));
  // d = dinv r / theta ; x += d
  CK(kv_cheb<T>(st, l.n, 0.0, 1.0 / theta, dinv, r, d, x));
  mg->ctx->launches++;
  for (int k = 1; k < mg->o.cheb_degree; k++) {
    ST(level_apply(mg, l, pr, d, t));
    CK(kv_axpby<T>(st, l.n, -1.0, t, 1.0, r));  // r -= A d
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    CK(kv_cheb<T>(st, l.n, rho_new * rho, 2.0 * rho_new / delta, dinv, r, d, x));
    mg->ctx->launches += 2;
    rho = rho_new;
  }
  return NH_OK;
}

// Jacobi-PCG in FP64 on level l: A x = b, x = 0 start.  With hist, runs exactly
// `maxit` steps and leaves rz_k, pq_k in the history slots (Lanczos).
// Returns iterations in *its.
nh_status pcg64(nh_mg mg, Level& l, const double* b, double* x, double rtol, int maxit, bool hist, int* its,
                bool warm = false, double ref = 0.0) {
  cudaStream_t st = mg->ctx->stream;
  const int64_t n = l.n;
  double *r = l.w[0], *z = l.w[1], *p = l.w[2], *q = l.w[3];
  const double* dinv = l.dinv64;
  if (l.stencil && !hist) {  // assembled coarsest level: the whole solve in one cooperative launch
    KsPcg a;
    a.Nx = l.space->Nx;
    a.Ny = l.space->Ny;
    a.Nz = l.space->Nz;
    a.bc = l.space->bc;
    a.A = l.A;
    a.dinv = dinv;
    a.b = b;
    a.x = x;
    a.r = r;
    a.z = z;
    a.p = p;
    a.q = q;
    a.part = mg->pcg_part;
    a.bar = mg->pcg_bar;
    a.out = mg->sc + S_PCG;
    a.rtol = rtol;
    a.ref = ref;
    a.maxit = maxit;
    a.warm = warm ? 1 : 0;
    a.err = mg->ctx->dev_err;
    CK(ks_pcg(st, a));
    mg->ctx->launches += 2;
    double res[2] = {0.0, 0.0};
    ST(read_sc(mg, S_PCG, 2, res));
    ST(nh_sync(mg->ctx));
    if (res[1] != 0.0) return nh_fail(mg->ctx, NH_ERR_NAN, "coarse PCG: non-finite residual");
    *its = (int)res[0];
    return NH_OK;
  }
  if (warm) {  // r = b - A x for the given start x
    ST(level_apply(mg, l, NH_F64, x, r));
    CK(kv_axpby<double>(st, n, 1.0, b, -1.0, r));
    mg->ctx->launches++;
  } else {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  }
  CK(kv_mul<double>(st, n, dinv, r, z));
  CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  mg->ctx->launches++;
  int cur = S_RZ0;
  ST(dot(mg, n, r, z, hist ? S_HIST : cur));
  double rz0 = 0.0;
  if (!hist) {
    ST(read_sc(mg, cur, 1, &rz0));
    if (warm) {
      // tolerance relative to the right-hand side's natural norm (ref^2 = b.D^-1 b)
      if (sqrt(fabs(rz0)) <= rtol * ref) {
        *its = 0;
        return NH_OK;
      }
      rz0 = ref * ref;
    }
    if (!(rz0 > 0.0)) {
      *its = 0;
      return NH_OK;
    }
  }
  const int check = 4;
  int k = 0;
  for (; k < maxit; k++) {
    const int rz_slot = hist ? S_HIST + k : cur;
    const int pq_slot = hist ? S_HIST + 64 + k : S_PQ;
    const int nx_slot = hist ? S_HIST + k + 1 : (cur == S_RZ0 ? S_RZ1 : S_RZ0);
    ST(level_apply(mg, l, NH_F64, p, q));
    ST(dot(mg, n, p, q, pq_slot));
    CK(kv_cg_update<double>(st, n, p, q, x, r, mg->sc, rz_slot, pq_slot));
    CK(kv_mul<double>(st, n, dinv, r, z));
    mg->ctx->launches += 2;
    ST(dot(mg, n, r, z, nx_slot));
    CK(kv_xpby_dev<double>(st, n, z, p, mg->sc, nx_slot, rz_slot, 1.0));
    mg->ctx->launches++;
    if (!hist) {
      cur = nx_slot;
      if ((k + 1) % check == 0 || k + 1 == maxit) {
        double rz = 0.0;
        ST(read_sc(mg, cur, 1, &rz));
        if (!isfinite(rz)) return nh_fail(mg->ctx, NH_ERR_NAN, "coarse PCG: non-finite residual");
        if (sqrt(fabs(rz)) <= rtol * sqrt(rz0)) {
          k++;
          break;
        }
      }
    }
  }
  *its = k;
  return NH_OK;
}

// largest eigenvalue of a symmetric tridiagonal matrix (Sturm bisection)
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; i++) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < n; i++) {
      d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) c++;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, fabs(hi)); it++) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) < n) lo = mid; else hi = mid;
  }
  return hi;
}

nh_status lanczos(nh_mg mg, Level& l) {
  cudaStream_t st = mg->ctx->stream;
  const int k = std::max(1, std::min(mg->o.lanczos_iters, 60));
  double* seed = l.w[4];
  CK(kv_uniform(st, l.n, mg->o.seed, seed));
  CK(kv_mask_zero<double>(st, l.nn, l.space->bc, seed));
  mg->ctx->launches += 2;
  // x goes to l.x only when the level is FP64; use w-scratch otherwise: reuse seed as x after copy
  double* x = (l.prec == NH_F64) ? (double*)l.x : nullptr;
  std::vector<double> hx;
  if (!x) {
    // FP32 level: x of the Lanczos run is not needed; borrow the fine FCG buffer sized for level 0
    x = mg->fx;
  }
  int its = 0;
  ST(pcg64(mg, l, seed, x, 0.0, k, true, &its));
  std::vector<double> h(2 * 64 + 1);
  ST(read_sc(mg, S_HIST, 128, h.data()));
  std::vector<double> al(k), be(k > 1 ? k - 1 : 0);
  int m = k;
  for (int i = 0; i < k; i++) {
    const double rz = h[i], pq = h[64 + i];
    if (!(pq > 0.0) || !(rz > 0.0)) {
      m = i;
      break;
    }
    const double alpha = rz / pq;
    const double beta_prev = i > 0 ? h[i] / h[i - 1] : 0.0;
    const double alpha_prev = i > 0 ? h[i - 1] / h[64 + i - 1] : 1.0;
    al[i] = 1.0 / alpha + (i > 0 ? beta_prev / alpha_prev : 0.0);
    if (i + 1 < k) {
      const double beta = h[i + 1] / h[i];
      be[i] = sqrt(fabs(beta)) / alpha;
    }
  }
  if (m == 0) return nh_fail(mg->ctx, NH_ERR_NAN, "Lanczos: no positive curvature on the seed vector");
  al.resize(m);
  be.resize(m > 1 ? m - 1 : 0);
  l.lmax = tridiag_max_eig(al, be);
  if (!(l.lmax > 0.0) || !isfinite(l.lmax)) return nh_fail(mg->ctx, NH_ERR_NAN, "Lanczos: lambda_max <= 0");
  return NH_OK;
}

template <typename T>
nh_status vcycle_t(nh_mg mg, int lv);

// x_lv = V-cycle(b_lv), dispatch on the level precision
nh_status coarse_solve(nh_mg mg, Level& l);
nh_status build_coarse_space(nh_mg mg);

nh_status vcycle(nh_mg mg, int lv) {
  Level& l = mg->L[lv];
  if (lv == (int)mg->L.size() - 1) return coarse_solve(mg, l);
  return l.prec == NH_F64 ? vcycle_t<double>(mg, lv) : vcycle_t<float>(mg, lv);
}

template <typename T>
nh_status vcycle_t(nh_mg mg, int lv) {
  cudaStream_t st = mg->ctx->stream;
  Level& l = mg->L[lv];
  Level& c = mg->L[lv + 1];
  T* x = (T*)l.x;
  T* b = (T*)l.b;
  T* r = (T*)l.r;
  ST(cheb<T>(mg, l, x, b, true));
  // r = b - A x
  ST(level_apply(mg, l, l.prec, x, r));
  CK(kv_axpby<T>(st, l.n, 1.0, b, -1.0, r));
  mg->ctx->launches++;
  // restrict in this level's precision, convert if the coarse level differs
  if (c.prec == l.prec) {
    ST(nh_transfer_internal(c.space, l.space, l.prec, 1, r, c.b));
  } else {
    ST(nh_transfer_internal(c.space, l.space, l.prec, 1, r, l.ct));
    if (l.prec == NH_F32)
      CK((kv_convert<float, double>(st, c.n, (const float*)l.ct, (double*)c.b)));
    else
      CK((kv_convert<double, float>(st, c.n, (const double*)l.ct, (float*)c.b)));
    mg->ctx->launches++;
  }
  if (c.prec == NH_F64)
    CK(kv_mask_zero<double>(st, c.nn, c.space->bc, (double*)c.b));
  else
    CK(kv_mask_zero<float>(st, c.nn, c.space->bc, (float*)c.b));
  mg->ctx->launches++;
  ST(vcycle(mg, lv + 1));
  // prolong the correction
  const void* xc = c.x;
  if (c.prec != l.prec) {
    if (l.prec == NH_F32)
      CK((kv_convert<double, float>(st, c.n, (const double*)c.x, (float*)l.ct)));
    else
      CK((kv_convert<float, double>(st, c.n, (const float*)c.x, (double*)l.ct)));
    mg->ctx->launches++;
    xc = l.ct;
  }
  ST(nh_transfer_internal(c.space, l.space, l.prec, 0, xc, l.t));
  CK(kv_mask_zero<T>(st, l.nn, l.space->bc, (T*)l.t));
  CK(kv_axpby<T>(st, l.n, 1.0, (const T*)l.t, 1.0, x));
  mg->ctx->launches += 2;
  ST(cheb<T>(mg, l, x, b, false));
  return NH_OK;
}

// the coarse Dirichlet mask by faces: a face component is constrained on the
// coarse space if it is constrained at every fine node of that face
// Unstructured mesh: a coarse node lies on one entity of an element (vertex, or the
// interior of an edge, face or the element); it is constrained in component c
// when every fine node on the same entity of that element is.  For masks made of
// whole boundary faces this is the box rule above, entity by entity.
nh_status coarse_mask_hex(nh_space f, nh_space c, const std::vector<uint8_t>& fb, std::vector<uint8_t>& out) {
  const int pf = f->p, pc = c->p, Pf = pf + 1, Pc = pc + 1;
  out.assign((size_t)c->n_dof, 0);
  for (int64_t e = 0; e < c->ne; e++)
    for (int k = 0; k < Pc; k++)
      for (int j = 0; j < Pc; j++)
        for (int i = 0; i < Pc; i++) {
          const int L[3] = {i, j, k};
          int lo[3], hi[3];  // fine lattice range of the same entity
          for (int d = 0; d < 3; d++) {
            if (L[d] == 0) lo[d] = hi[d] = 0;
            else if (L[d] == pc) lo[d] = hi[d] = pf;
            else { lo[d] = 1; hi[d] = pf - 1; }
          }
          unsigned m = 7u;
          for (int kk = lo[2]; kk <= hi[2]; kk++)
            for (int jj = lo[1]; jj <= hi[1]; jj++)
              for (int ii = lo[0]; ii <= hi[0]; ii++)
                m &= fb[f->emap_host[(size_t)e * Pf * Pf * Pf + (kk * Pf + jj) * Pf + ii]];
          const int64_t n = c->emap_host[(size_t)e * Pc * Pc * Pc + (k * Pc + j) * Pc + i];
          for (int cc = 0; cc < 3; cc++) out[3 * n + cc] = (m >> cc) & 1u;
        }
  return NH_OK;
}

nh_status coarse_mask(nh_mg mg, nh_space f, nh_space c, std::vector<uint8_t>& out) {
  std::vector<uint8_t> fb((size_t)f->n_nodes);
  CK(cudaMemcpy(fb.data(), f->bc, f->n_nodes, cudaMemcpyDeviceToHost));
  if (f->hex) return coarse_mask_hex(f, c, fb, out);
  const int dims_f[3] = {f->Nx, f->Ny, f->Nz}, dims_c[3] = {c->Nx, c->Ny, c->Nz};
  unsigned face[6];  // (axis, side) -> component bits constrained everywhere on that face
  for (int ax = 0; ax < 3; ax++)
    for (int sd = 0; sd < 2; sd++) {
      unsigned acc = 7u;
      const int fixed = sd ? dims_f[ax] - 1 : 0;
      const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
      for (int i = 0; i < dims_f[a1]; i++)
        for (int j = 0; j < dims_f[a2]; j++) {
          int idx[3];
          idx[ax] = fixed;
          idx[a1] = i;
          idx[a2] = j;
          acc &= fb[idx[0] + (int64_t)dims_f[0] * (idx[1] + (int64_t)dims_f[1] * idx[2])];
        }
      face[ax * 2 + sd] = acc;
    }
  out.assign((size_t)c->n_dof, 0);
  for (int64_t n = 0; n < c->n_nodes; n++) {
    const int I[3] = {(int)(n % dims_c[0]), (int)((n / dims_c[0]) % dims_c[1]), (int)(n / ((int64_t)dims_c[0] * dims_c[1]))};
    unsigned m = 0;
    for (int ax = 0; ax < 3; ax++) {
      if (I[ax] == 0) m |= face[ax * 2];
      if (I[ax] == dims_c[ax] - 1) m |= face[ax * 2 + 1];
    }
    for (int cc = 0; cc < 3; cc++) out[3 * n + cc] = (m >> cc) & 1u;
  }
  return NH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" nh_status nh_mg_default_opts(nh_op fine, nh_mg_opts* o) {
  if (!fine || !o) return NH_ERR_ARG;
  memset(o, 0, sizeof(*o));
  const int p = fine->space->p;
  if (p >= 3) {
    o->n_levels = 3;
    o->level_p[0] = p;
    o->level_p[1] = 2;
    o->level_p[2] = 1;
  } else if (p == 2) {
    o->n_levels = 2;
    o->level_p[0] = 2;
    o->level_p[1] = 1;
  } else {
    o->n_levels = 1;
    o->level_p[0] = 1;
  }
  o->cheb_degree = 3;
  o->cheb_lo = 0.1;
  o->cheb_hi = 1.1;
  o->lanczos_iters = 10;
  o->coarse_rtol = 1e-3;
  o->coarse_maxit = 2000;
  o->coarse_assembled = 1;
  o->mixed = 0;
  o->seed = 12345;
  o->load_steps = 1;
  o->newton_rtol = 1e-8;
  o->newton_atol = 1e-13;
  o->newton_maxit = 30;
  o->krylov_rtol = 1e-3;
  o->krylov_maxit = 500;
  o->line_search = 1;
  o->verbose = 0;
  o->learned_accept = 0;
  o->learned_mode = 2;
  o->fp64_kind = 0;
  o->coarse_rediscretize = 0;
  o->nonlinear = 0;
  o->lbfgs_m = 5;
  o->coarse_solver = 0;
  o->coarse_fixed = 0;
  o->learned_vectors = 32;
  return NH_OK;
}

extern "C" nh_status nh_mg_destroy(nh_mg mg) {
  if (!mg) return NH_ERR_ARG;
  cudaStreamSynchronize(mg->ctx->stream);
  for (Level& l : mg->L) {
    for (void* p : {l.x, l.b, l.r, l.d, l.t, l.dinv, l.ct}) cudaFree(p);
    for (void* p : {(void*)l.rowptr, (void*)l.col, (void*)l.jstart, (void*)l.perm, (void*)l.coo, (void*)l.val})
      cudaFree(p);
    for (double* p : l.w) cudaFree(p);
    if (l.dinv64 != (double*)l.dinv) cudaFree(l.dinv64);
    cudaFree(l.A);
    if (l.own) {
      nh_op_destroy(l.op);
      nh_space_destroy(l.space);
    }
  }
  cudaFree(mg->sc);
  cudaFree(mg->part);
  cudaFree(mg->pcg_part);
  cudaFree(mg->pcg_bar);
  for (HLevel& h : mg->H) {
    if (h.own) {
      cudaFree(h.bc);
      cudaFree(h.A);
      cudaFree(h.dinv);
    }
    for (double* p : {h.x, h.b, h.r, h.t}) cudaFree(p);
  }
  cudaFree(mg->Hinv);
  cudaFreeHost(mg->hsc);
  for (double* p : mg->lbs) cudaFree(p);
  for (double* p : mg->lby) cudaFree(p);
  cudaFree(mg->lbr);
  for (double* p : {mg->fr, mg->fz, mg->fp, mg->fq, mg->fx, mg->fu, mg->fg, mg->fb, mg->ft, mg->fs, mg->fsave})
    cudaFree(p);
  for (void* p : {(void*)mg->lc1, (void*)mg->lc2, (void*)mg->W, (void*)mg->Wc, (void*)mg->Wpart}) cudaFree(p);
  for (void* p : {(void*)mg->feat, (void*)mg->nout, (void*)mg->logE, (void*)mg->lz1, (void*)mg->lw, (void*)mg->lxs,
                  (void*)mg->lx, (void*)mg->lt})
    cudaFree(p);
  delete mg;
  return NH_OK;
}

extern "C" nh_status nh_mg_create(nh_op fine, const nh_mg_opts* opts, nh_mg* out) {
  if (!fine || !out) return NH_ERR_ARG;
  *out = nullptr;
  if (fine->parent) return nh_fail(fine->space->ctx, NH_ERR_ARG, "nh_mg_create: needs the fine operator");
  nh_mg mg = new nh_mg_s();
  mg->ctx = fine->space->ctx;
  mg->fine = fine;
  if (opts)
    mg->o = *opts;
  else
    nh_mg_default_opts(fine, &mg->o);
  const nh_mg_opts& o = mg->o;
  nh_space fs = fine->space;
  auto bad = [&](const char* m) {
    nh_fail(mg->ctx, NH_ERR_ARG, m);
    delete mg;
    return NH_ERR_ARG;
  };
  if (o.n_levels < 1 || o.n_levels > 8) return bad("nh_mg_create: 1 <= n_levels <= 8");
  if (o.level_p[0] != fs->p) return bad("nh_mg_create: level_p[0] must be the fine order");
  for (int i = 1; i < o.n_levels; i++)
    if (o.level_p[i] < 1 || o.level_p[i] >= o.level_p[i - 1]) return bad("nh_mg_create: orders must decrease to >= 1");
  if (o.cheb_degree < 1 || !(o.cheb_hi > o.cheb_lo) || !(o.cheb_lo > 0)) return bad("nh_mg_create: bad Chebyshev options");
  if (o.fp64_kind != 0 && o.fp64_kind != 1) return bad("nh_mg_create: fp64_kind must be 0 or 1");
  if (o.coarse_rediscretize != 0 && o.coarse_rediscretize != 1)
    return bad("nh_mg_create: coarse_rediscretize must be 0 or 1");
  if (o.nonlinear != 0 && o.nonlinear != 1) return bad("nh_mg_create: nonlinear must be 0 (Newton) or 1 (L-BFGS)");
  if (o.nonlinear == 1 && (o.lbfgs_m < 1 || o.lbfgs_m > 32)) return bad("nh_mg_create: need 1 <= lbfgs_m <= 32");
  if (o.coarse_fixed < 0 || o.coarse_fixed > 100000) return bad("nh_mg_create: need 0 <= coarse_fixed <= 100000");
  if (o.learned_mode < 1 || o.learned_mode > 4) return bad("nh_mg_create: learned_mode must be 1 to 4");
  if (o.learned_vectors < 0 || o.learned_vectors > 256) return bad("nh_mg_create: need 0 <= learned_vectors <= 256");
  if (o.coarse_solver != 0 && o.coarse_solver != 1) return bad("nh_mg_create: coarse_solver must be 0 or 1");
  if (fs->hex && o.coarse_solver) {
    delete mg;
    return nh_fail(fine->space->ctx, NH_ERR_UNSUPPORTED,
                   "nh_mg_create: the geometric coarse multigrid needs a box mesh (coarse_solver = 0 on nh_space_hex "
                   "meshes)");
  }
  mg->p64 = o.fp64_kind ? NH_F64X : NH_F64;
  cudaSetDevice(mg->ctx->device);
  nh_status s;
  mg->L.resize(o.n_levels);
  for (int i = 0; i < o.n_levels; i++) {
    Level& l = mg->L[i];
    l.p = o.level_p[i];
    if (i == 0) {
      l.space = fs;
      l.op = fine;
    } else {
      const bool assembled = (i == o.n_levels - 1) && l.p == 1 && o.coarse_assembled;
      l.redisc = o.coarse_rediscretize && !assembled;
      int64_t nn, nd;
      if (fs->hex)
        s = nh_space_hex(mg->ctx, (int64_t)fs->verts_host.size() / 3, fs->verts_host.data(), fs->ne,
                         fs->hex8_host.data(), l.p, l.redisc ? l.p + 1 : fs->q, &l.space, &nn, &nd);
      else
        s = nh_space_box(mg->ctx, fs->nx, fs->ny, fs->nz, fs->verts_host.empty() ? nullptr : fs->verts_host.data(),
                         l.p, l.redisc ? l.p + 1 : fs->q, &l.space, &nn, &nd);
      if (s != NH_OK) { nh_mg_destroy(mg); return s; }
      l.own = true;
      std::vector<uint8_t> m;
      if ((s = coarse_mask(mg, fs, l.space, m)) != NH_OK) { nh_mg_destroy(mg); return s; }
      if ((s = nh_space_set_dirichlet(l.space, m.data())) != NH_OK) { nh_mg_destroy(mg); return s; }
      s = l.redisc ? nh_op_rediscretize(fine, l.space, &l.op) : nh_op_level(fine, l.space, &l.op);
      if (s != NH_OK) { nh_mg_destroy(mg); return s; }
    }
    l.n = l.space->n_dof;
    l.nn = l.space->n_nodes;
    l.prec = (o.mixed && l.p > 1) ? NH_F32 : NH_F64;
    const bool asm_level = (i == o.n_levels - 1) && l.p == 1 && o.coarse_assembled && o.n_levels > 1;
    l.stencil = asm_level && !fs->hex;
    l.bsr = asm_level && fs->hex;
    if (l.bsr) {  // symbolic phase on the host, once per hierarchy
      std::vector<int64_t> rp, js, pm;
      std::vector<int> cl;
      ks_coo_symbolic(l.space->ne, l.nn, l.space->emap_host.data(), rp, cl, js, pm);
      l.nnzb = (int64_t)cl.size();
      if ((s = dalloc(mg, (void**)&l.rowptr, sizeof(int64_t) * rp.size())) != NH_OK ||
          (s = dalloc(mg, (void**)&l.col, sizeof(int) * cl.size())) != NH_OK ||
          (s = dalloc(mg, (void**)&l.jstart, sizeof(int64_t) * js.size())) != NH_OK ||
          (s = dalloc(mg, (void**)&l.perm, sizeof(int64_t) * pm.size())) != NH_OK ||
          (s = dalloc(mg, (void**)&l.coo, sizeof(double) * 9 * pm.size())) != NH_OK ||
          (s = dalloc(mg, (void**)&l.val, sizeof(double) * 9 * cl.size())) != NH_OK) {
        nh_mg_destroy(mg);
        return s;
      }
      cudaError_t ce = cudaMemcpy(l.rowptr, rp.data(), sizeof(int64_t) * rp.size(), cudaMemcpyHostToDevice);
      if (!ce) ce = cudaMemcpy(l.col, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice);
      if (!ce) ce = cudaMemcpy(l.jstart, js.data(), sizeof(int64_t) * js.size(), cudaMemcpyHostToDevice);
      if (!ce) ce = cudaMemcpy(l.perm, pm.data(), sizeof(int64_t) * pm.size(), cudaMemcpyHostToDevice);
      if (ce) {
        nh_mg_destroy(mg);
        return nh_cuda_check(fine->space->ctx, ce, "nh_mg_create: block-row pattern upload");
      }
    }
    const size_t wb = wsize(l.prec) * l.n;
    for (void** v : {&l.x, &l.b, &l.r, &l.d, &l.t, &l.dinv})
      if ((s = dalloc(mg, v, wb)) != NH_OK) { nh_mg_destroy(mg); return s; }
    for (int k = 0; k < 5; k++)
      if ((s = dalloc(mg, (void**)&l.w[k], 8 * l.n)) != NH_OK) { nh_mg_destroy(mg); return s; }
    if (l.prec == NH_F64) {
      l.dinv64 = (double*)l.dinv;
    } else if ((s = dalloc(mg, (void**)&l.dinv64, 8 * l.n)) != NH_OK) {
      nh_mg_destroy(mg);
      return s;
    }
    if (l.stencil && (s = dalloc(mg, (void**)&l.A, sizeof(double) * 243 * l.nn)) != NH_OK) {
      nh_mg_destroy(mg);
      return s;
    }
  }
  for (int i = 0; i + 1 < o.n_levels; i++) {
    Level& l = mg->L[i];
    if (mg->L[i + 1].prec != l.prec && (s = dalloc(mg, &l.ct, wsize(l.prec) * mg->L[i + 1].n)) != NH_OK) {
      nh_mg_destroy(mg);
      return s;
    }
  }
  const size_t fb = 8 * (size_t)fs->n_dof;
  if ((s = dalloc(mg, (void**)&mg->sc, sizeof(double) * S_LEN)) != NH_OK ||
      (s = dalloc(mg, (void**)&mg->part, sizeof(double) * 148 * 8 + 64)) != NH_OK ||
      (s = dalloc(mg, (void**)&mg->pcg_part, sizeof(double) * (2 * (size_t)ks_pcg_max_blocks() + 2))) != NH_OK ||
      (s = dalloc(mg, (void**)&mg->pcg_bar, 64)) != NH_OK) {
    nh_mg_destroy(mg);
    return s;
  }
  for (double** v : {&mg->fr, &mg->fz, &mg->fp, &mg->fq, &mg->fx, &mg->fu, &mg->fg, &mg->fb, &mg->ft, &mg->fs, &mg->fsave})
    if ((s = dalloc(mg, (void**)v, fb)) != NH_OK) { nh_mg_destroy(mg); return s; }
  if (cudaMallocHost(&mg->hsc, sizeof(double) * S_LEN) != cudaSuccess) {
    cudaGetLastError();
    nh_mg_destroy(mg);
    return NH_ERR_OOM;
  }
  cudaMemset(mg->sc, 0, sizeof(double) * S_LEN);
  // geometric multigrid for an assembled Q1 coarsest level: halve the lattice while
  // every direction has an even number of cells, down to 3 nodes per direction
  Level& lc = mg->L.back();
  if (o.coarse_solver == 1 && lc.stencil) {
    HLevel h0;
    h0.Nx = lc.space->Nx;
    h0.Ny = lc.space->Ny;
    h0.Nz = lc.space->Nz;
    h0.nn = lc.nn;
    h0.bc = lc.space->bc;
    h0.A = lc.A;
    h0.dinv = lc.dinv64;
    mg->H.push_back(h0);
    auto even = [](int N) { return N >= 5 && (N - 1) % 2 == 0; };
    while (even(mg->H.back().Nx) && even(mg->H.back().Ny) && even(mg->H.back().Nz)) {
      const HLevel& f = mg->H.back();
      HLevel c;
      c.Nx = (f.Nx - 1) / 2 + 1;
      c.Ny = (f.Ny - 1) / 2 + 1;
      c.Nz = (f.Nz - 1) / 2 + 1;
      c.nn = (int64_t)c.Nx * c.Ny * c.Nz;
      c.own = true;
      mg->H.push_back(c);
      HLevel& cc = mg->H.back();
      if ((s = dalloc(mg, (void**)&cc.bc, cc.nn)) != NH_OK || (s = dalloc(mg, (void**)&cc.A, 8 * 243 * cc.nn)) != NH_OK ||
          (s = dalloc(mg, (void**)&cc.dinv, 8 * 3 * cc.nn)) != NH_OK) {
        nh_mg_destroy(mg);
        return s;
      }
    }
    for (HLevel& h : mg->H)
      for (double** v : {&h.x, &h.b, &h.r, &h.t})
        if ((s = dalloc(mg, (void**)v, 8 * 3 * h.nn)) != NH_OK) { nh_mg_destroy(mg); return s; }
    if (mg->H.size() < 2 || mg->H.back().nn > 216) {
      // no usable hierarchy (odd cell counts or a large coarsest lattice): Jacobi-PCG
      for (HLevel& h : mg->H) {
        if (h.own) {
          cudaFree(h.bc);
          cudaFree(h.A);
          cudaFree(h.dinv);
        }
        for (double* p : {h.x, h.b, h.r, h.t}) cudaFree(p);
      }
      mg->H.clear();
    } else {
      mg->Hn = (int)(3 * mg->H.back().nn);
      if ((s = dalloc(mg, (void**)&mg->Hinv, 8 * (size_t)mg->Hn * mg->Hn)) != NH_OK) { nh_mg_destroy(mg); return s; }
    }
  }
  *out = mg;
  return NH_OK;
}

// ---- geometric multigrid on the assembled Q1 level ------------------------------
// Galerkin stencils down the lattice hierarchy, Jacobi diagonals, and the dense
// inverse of the coarsest stencil (constrained rows identity; Cholesky on the host).
static nh_status hmg_setup(nh_mg mg) {
  cudaStream_t st = mg->ctx->stream;
  for (size_t l = 1; l < mg->H.size(); l++) {
    HLevel &f = mg->H[l - 1], &c = mg->H[l];
    CK(hm_coarse_bc(st, f.Nx, f.Ny, c.Nx, c.Ny, c.Nz, f.bc, c.bc));
    CK(hm_rap(st, f.Nx, f.Ny, f.Nz, c.Nx, c.Ny, c.Nz, f.bc, c.bc, f.A, c.A));
    CK(ks_diag(st, c.nn, c.bc, c.A, c.dinv));
    CK(kv_recip<double>(st, 3 * c.nn, c.dinv));
    mg->ctx->launches += 4;
  }
  const HLevel& L = mg->H.back();
  const int n = mg->Hn;
  std::vector<double> A((size_t)243 * L.nn), D((size_t)n * n, 0.0);
  std::vector<uint8_t> bc((size_t)L.nn);
  CK(cudaMemcpyAsync(A.data(), L.A, 8 * A.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(bc.data(), L.bc, bc.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int64_t I = 0; I < L.nn; I++) {
    const int x = (int)(I % L.Nx), y = (int)((I / L.Nx) % L.Ny), z = (int)(I / ((int64_t)L.Nx * L.Ny));
    for (int c = 0; c < 3; c++) {
      const int64_t row = 3 * I + c;
      if ((bc[I] >> c) & 1u) {
        D[row * n + row] = 1.0;
        continue;
      }
      for (int s = 0; s < 27; s++) {
        const int x2 = x + s % 3 - 1, y2 = y + (s / 3) % 3 - 1, z2 = z + s / 9 - 1;
        if (x2 < 0 || x2 >= L.Nx || y2 < 0 || y2 >= L.Ny || z2 < 0 || z2 >= L.Nz) continue;
        const int64_t J = x2 + (int64_t)L.Nx * (y2 + (int64_t)L.Ny * z2);
        for (int cp = 0; cp < 3; cp++)
          if (!((bc[J] >> cp) & 1u)) D[row * n + 3 * J + cp] += A[((size_t)s * 9 + 3 * c + cp) * L.nn + I];
      }
    }
  }
  // Cholesky D = C C^T, then the inverse column by column
  std::vector<double> C((size_t)n * n, 0.0), Inv((size_t)n * n, 0.0);
  for (int j = 0; j < n; j++) {
    double d = D[(size_t)j * n + j];
    for (int k = 0; k < j; k++) d -= C[(size_t)j * n + k] * C[(size_t)j * n + k];
    if (!(d > 0.0)) {  // indefinite tangent (e.g. past a limit point): no SPD V-cycle this time
      mg->hmg_ok = false;
      return NH_OK;
    }
    const double cjj = sqrt(d);
    C[(size_t)j * n + j] = cjj;
    for (int i = j + 1; i < n; i++) {
      double v = 0.5 * (D[(size_t)i * n + j] + D[(size_t)j * n + i]);
      for (int k = 0; k < j; k++) v -= C[(size_t)i * n + k] * C[(size_t)j * n + k];
      C[(size_t)i * n + j] = v / cjj;
    }
  }
  std::vector<double> w(n);
  for (int e = 0; e < n; e++) {
    for (int i = 0; i < n; i++) {  // C w = e_e
      double v = (i == e) ? 1.0 : 0.0;
      for (int k = 0; k < i; k++) v -= C[(size_t)i * n + k] * w[k];
      w[i] = v / C[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {  // C^T x = w
      double v = w[i];
      for (int k = i + 1; k < n; k++) v -= C[(size_t)k * n + i] * Inv[(size_t)k * n + e];
      Inv[(size_t)i * n + e] = v / C[(size_t)i * n + i];
    }
  }
  CK(cudaMemcpyAsync(mg->Hinv, Inv.data(), 8 * Inv.size(), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  mg->hmg_ok = true;
  return NH_OK;
}

namespace {
constexpr double kHOmega = 0.6;  // Jacobi damping
constexpr int kHSweeps = 2;      // pre- and post-smoothing sweeps

// x = M_l b: one symmetric V-cycle from lattice l (x, b of that lattice's size)
nh_status hvcycle(nh_mg mg, size_t l, const double* b, double* x) {
  cudaStream_t st = mg->ctx->stream;
  HLevel& h = mg->H[l];
  if (l + 1 == mg->H.size()) {
    CK(hm_dense_mv(st, mg->Hn, mg->Hinv, b, x));
    mg->ctx->launches++;
    return NH_OK;
  }
  HLevel& c = mg->H[l + 1];
  const size_t bytes = 8 * 3 * (size_t)h.nn;
  CK(hm_jacobi(st, h.Nx, h.Ny, h.Nz, h.bc, h.A, h.dinv, b, x, x, kHOmega, 1));
  for (int s = 1; s < kHSweeps; s++) {
    CK(hm_jacobi(st, h.Nx, h.Ny, h.Nz, h.bc, h.A, h.dinv, b, x, h.t, kHOmega, 0));
    CK(cudaMemcpyAsync(x, h.t, bytes, cudaMemcpyDeviceToDevice, st));
  }
  CK(hm_resid(st, h.Nx, h.Ny, h.Nz, h.bc, h.A, b, x, h.r));
  CK(hm_restrict(st, h.Nx, h.Ny, h.Nz, c.Nx, c.Ny, c.Nz, h.bc, c.bc, h.r, c.b));
  mg->ctx->launches += 1 + kHSweeps + 1;
  ST(hvcycle(mg, l + 1, c.b, c.x));
  CK(hm_prolong_add(st, h.Nx, h.Ny, h.Nz, c.Nx, c.Ny, c.Nz, h.bc, c.bc, c.x, x));
  for (int s = 0; s < kHSweeps; s++) {
    CK(hm_jacobi(st, h.Nx, h.Ny, h.Nz, h.bc, h.A, h.dinv, b, x, h.t, kHOmega, 0));
    CK(cudaMemcpyAsync(x, h.t, bytes, cudaMemcpyDeviceToDevice, st));
  }
  mg->ctx->launches += 1 + kHSweeps;
  return NH_OK;
}

// PCG on the assembled Q1 level with the geometric V-cycle as preconditioner
// (symmetric: same damped Jacobi sweeps before and after, P^T restriction,
// exact coarsest solve); stops on sqrt(r.z) <= rtol sqrt(r0.z0).
nh_status hmg_pcg(nh_mg mg, Level& l, const double* b, double* x, double rtol, int maxit, int* its) {
  cudaStream_t st = mg->ctx->stream;
  const int64_t n = l.n;
  double *r = l.w[0], *z = l.w[1], *p = l.w[2], *q = l.w[3];
  CK(cudaMemsetAsync(x, 0, 8 * n, st));
  CK(cudaMemcpyAsync(r, b, 8 * n, cudaMemcpyDeviceToDevice, st));
  ST(hvcycle(mg, 0, r, z));
  double rz = 0.0;
  ST(dot_host(mg, n, r, z, &rz));
  const double rz0 = rz;
  int k = 0;
  if (rz0 > 0.0) {
    CK(cudaMemcpyAsync(p, z, 8 * n, cudaMemcpyDeviceToDevice, st));
    while (k < maxit) {
      ST(level_apply(mg, l, NH_F64, p, q));
      double pq = 0.0;
      ST(dot_host(mg, n, p, q, &pq));
      const double a = rz / pq;
      CK(kv_axpby<double>(st, n, a, p, 1.0, x));
      CK(kv_axpby<double>(st, n, -a, q, 1.0, r));
      mg->ctx->launches += 2;
      ST(hvcycle(mg, 0, r, z));
      double rzn = 0.0;
      ST(dot_host(mg, n, r, z, &rzn));
      k++;
      if (!isfinite(rzn)) return nh_fail(mg->ctx, NH_ERR_NAN, "coarse multigrid PCG: non-finite residual");
      if (sqrt(fabs(rzn)) <= rtol * sqrt(rz0)) break;
      CK(kv_axpby<double>(st, n, 1.0, z, rzn / rz, p));
      mg->ctx->launches++;
      rz = rzn;
    }
  }
  *its = k;
  return NH_OK;
}

// z = M r, the preconditioner of the fixed coarse solve: one geometric V-cycle
// when that hierarchy is set up, else the Jacobi diagonal.
nh_status coarse_prec(nh_mg mg, Level& l, const double* r, double* z) {
  if (mg->hmg_ok && &l == &mg->L.back()) return hvcycle(mg, 0, r, z);
  CK(kv_mul<double>(mg->ctx->stream, l.n, l.dinv64, r, z));
  mg->ctx->launches++;
  return NH_OK;
}

// Interval of the fixed coarse solve: extreme Ritz values of M A from m steps of
// M-preconditioned CG on a seeded rough vector (the Lanczos tridiagonal of the
// CG coefficients, as for the smoothers' lambda_max).  The upper end gets the
// smoothers' margin cheb_hi: Chebyshev semi-iteration must not see eigenvalues
// above its interval; below it (the Ritz value overestimates lambda_min) it only
// damps less.
nh_status coarse_bounds(nh_mg mg, Level& l) {
  cudaStream_t st = mg->ctx->stream;
  const int m = std::min(60, std::max(20, 2 * mg->o.lanczos_iters));
  double *r = l.w[0], *z = l.w[1], *p = l.w[2], *q = l.w[3], *seed = l.w[4];
  CK(kv_uniform(st, l.n, mg->o.seed, seed));
  CK(kv_mask_zero<double>(st, l.nn, l.space->bc, seed));
  mg->ctx->launches += 2;
  CK(cudaMemcpyAsync(r, seed, 8 * l.n, cudaMemcpyDeviceToDevice, st));
  ST(coarse_prec(mg, l, r, z));
  CK(cudaMemcpyAsync(p, z, 8 * l.n, cudaMemcpyDeviceToDevice, st));
  double rz = 0.0;
  ST(dot_host(mg, l.n, r, z, &rz));
  std::vector<double> al, be;
  double alpha_prev = 1.0, beta_prev = 0.0;
  for (int k = 0; k < m && rz > 0.0 && isfinite(rz); k++) {
    ST(level_apply(mg, l, NH_F64, p, q));
    double pq = 0.0;
    ST(dot_host(mg, l.n, p, q, &pq));
    if (!(pq > 0.0) || !isfinite(pq)) break;
    const double alpha = rz / pq;
    al.push_back(1.0 / alpha + (k > 0 ? beta_prev / alpha_prev : 0.0));
    CK(kv_axpby<double>(st, l.n, -alpha, q, 1.0, r));
    mg->ctx->launches++;
    ST(coarse_prec(mg, l, r, z));
    double rzn = 0.0;
    ST(dot_host(mg, l.n, r, z, &rzn));
    const double beta = rzn / rz;
    be.push_back(sqrt(fabs(beta)) / alpha);
    CK(kv_axpby<double>(st, l.n, 1.0, z, beta, p));  // p = z + beta p
    mg->ctx->launches++;
    alpha_prev = alpha;
    beta_prev = beta;
    rz = rzn;
  }
  if (al.empty()) return nh_fail(mg->ctx, NH_ERR_NAN, "coarse Lanczos: no positive curvature on the seed vector");
  be.resize(al.size() - 1);
  const double lmax = tridiag_max_eig(al, be);
  std::vector<double> neg(al.size());
  for (size_t i = 0; i < al.size(); i++) neg[i] = -al[i];
  const double lmin = -tridiag_max_eig(neg, be);
  if (!(lmax > 0.0) || !isfinite(lmax)) return nh_fail(mg->ctx, NH_ERR_NAN, "coarse Lanczos: lambda_max <= 0");
  l.cmax = mg->o.cheb_hi * lmax;
  l.cmin = (lmin > 0.0 && isfinite(lmin)) ? std::min(lmin, 0.5 * l.cmax) : 1e-3 * l.cmax;
  return NH_OK;
}

// Fixed coarse solve: x = q(M A) M b after `degree` steps of Chebyshev
// semi-iteration preconditioned by M over [cmin, cmax] (Saad, Iterative
// Methods, Alg. 12.1), from x = 0, or from the given x (warm).  A fixed
// polynomial: the map b -> x is linear, symmetric and positive definite, and
// it needs no reduction and no host synchronisation.
nh_status coarse_cheb(nh_mg mg, Level& l, const double* b, double* x, bool warm) {
  cudaStream_t st = mg->ctx->stream;
  const int64_t n = l.n;
  double *r = l.w[0], *d = l.w[1], *z = l.w[2], *t = l.w[3];
  const double theta = 0.5 * (l.cmax + l.cmin), delta = 0.5 * (l.cmax - l.cmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  const bool jac = !(mg->hmg_ok && &l == &mg->L.back());
  if (warm) {
    ST(level_apply(mg, l, NH_F64, x, t));
    CK(cudaMemcpyAsync(r, b, 8 * n, cudaMemcpyDeviceToDevice, st));
    CK(kv_axpby<double>(st, n, -1.0, t, 1.0, r));  // r = b - A x
    mg->ctx->launches++;
  } else {
    CK(cudaMemcpyAsync(r, b, 8 * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(x, 0, 8 * n, st));
  }
  const int deg = std::max(1, mg->o.coarse_fixed);
  for (int k = 0; k < deg; k++) {
    double c1 = 0.0, c2 = 1.0 / theta;
    if (k > 0) {
      ST(level_apply(mg, l, NH_F64, d, t));
      CK(kv_axpby<double>(st, n, -1.0, t, 1.0, r));  // r -= A d
      mg->ctx->launches++;
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c1 = rho_new * rho;
      c2 = 2.0 * rho_new / delta;
      rho = rho_new;
    }
    if (jac) {
      CK(kv_cheb<double>(st, n, c1, c2, l.dinv64, r, d, x));  // d = c1 d + c2 D^-1 r; x += d
      mg->ctx->launches++;
    } else {
      ST(coarse_prec(mg, l, r, z));
      CK(kv_axpby<double>(st, n, c2, z, c1, d));  // d = c1 d + c2 M r
      CK(kv_axpby<double>(st, n, 1.0, d, 1.0, x));
      mg->ctx->launches += 2;
    }
  }
  return NH_OK;
}
}  // namespace

static nh_status learned_buffers(nh_mg mg);

extern "C" nh_status nh_mg_setup(nh_mg mg) {
  if (!mg) return NH_ERR_ARG;
  nh_op root = mg->fine;
  if (!root->have_qd) return nh_fail(mg->ctx, NH_ERR_STATE, "nh_mg_setup: call nh_qdata_setup first");
  cudaStream_t st = mg->ctx->stream;
  CK(cudaSetDevice(mg->ctx->device));
  const bool timing = mg->o.verbose >= 2;
  auto mark = [&](const char* what, int lv, double& t0) -> nh_status {
    if (!timing) return NH_OK;
    CK(cudaStreamSynchronize(st));
    const double t1 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    fprintf(stderr, "nh_mg_setup level %d %-9s %8.3f ms\n", lv, what, 1e3 * (t1 - t0));
    t0 = t1;
    return NH_OK;
  };
  double t0 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  int lv = 0;
  for (Level& l : mg->L) {
    if (l.bsr) {
      const int Qf = root->space->Q;
      const int64_t Q3 = (int64_t)Qf * Qf * Qf;
      CK(ks_element_blocks_q1(Qf, st, l.space->ne, root->qd, root->space->ne * Q3, root->layout, &l.space->tab, l.coo));
      CK(ks_coo_sum(st, l.nnzb, l.jstart, l.perm, l.coo, l.val));
      CK(ks_bsr_diag(st, l.nn, l.rowptr, l.col, l.val, l.space->bc, l.dinv64));
      mg->ctx->launches += 3;
      ST(mark("coo", lv, t0));
    } else if (l.stencil) {
      CK(cudaMemsetAsync(l.A, 0, sizeof(double) * 243 * l.nn, st));
      const int64_t Q3 = (int64_t)root->space->Q * root->space->Q * root->space->Q;
      // mixed precision: the element blocks are summed in float-float on the FP32 pipes
      CK(ks_assemble_q1(root->space->Q, st, l.space->ne, l.space->nx, l.space->ny, l.space->nz, l.space->bc, root->qd,
                        root->space->ne * Q3, root->layout, &l.space->tab, l.A, mg->o.mixed ? 1 : 0));
      CK(ks_diag(st, l.nn, l.space->bc, l.A, l.dinv64));
      mg->ctx->launches += 2;
      ST(mark("stencil", lv, t0));
    } else {
      if (l.redisc) {
        ST(nh_qdata_setup_rediscretized(l.op, root, root->u_state, nullptr));
        ST(mark("qdata", lv, t0));
      }
      if (l.prec == NH_F32) {  // FP32 smoother level: the diagonal in FP32 arithmetic
        ST(nh_jacobian_diagonal(l.op, NH_F32, l.dinv));
        CK((kv_convert<float, double>(st, l.n, (const float*)l.dinv, l.dinv64)));
        mg->ctx->launches++;
      } else {
        ST(nh_jacobian_diagonal(l.op, NH_F64, l.dinv64));
      }
      ST(mark("diagonal", lv, t0));
    }
    CK(kv_recip<double>(st, l.n, l.dinv64));
    mg->ctx->launches++;
    if (l.prec == NH_F32) {
      CK((kv_convert<double, float>(st, l.n, l.dinv64, (float*)l.dinv)));
      mg->ctx->launches++;
    }
    if (&l != &mg->L.back()) {
      ST(lanczos(mg, l));
      ST(mark("lanczos", lv, t0));
    }
    lv++;
  }
  if (!mg->H.empty()) {
    ST(hmg_setup(mg));
    ST(mark("h-mg", lv, t0));
  }
  if (mg->o.coarse_fixed > 0) {
    ST(coarse_bounds(mg, mg->L.back()));
    ST(mark("c-bounds", lv, t0));
  }
  mg->Wk = 0;
  if (mg->o.learned_mode == 4 && mg->o.learned_vectors > 0 && mg->L.size() >= 2 && mg->L.back().p == 1 &&
      !mg->L[0].space->hex) {
    ST(learned_buffers(mg));
    ST(build_coarse_space(mg));
    ST(mark("c-space", lv, t0));
  }
  CK(cudaStreamSynchronize(st));
  mg->setup_done = true;
  return NH_OK;
}

extern "C" nh_status nh_mg_level_info(nh_mg mg, int level, nh_space* space, nh_op* op, double* lmax) {
  if (!mg || level < 0 || level >= (int)mg->L.size()) return NH_ERR_ARG;
  if (space) *space = mg->L[level].space;
  if (op) *op = mg->L[level].op;
  if (lmax) *lmax = mg->L[level].lmax;
  return NH_OK;
}

static nh_status vcycle_fp64(nh_mg mg, const double* r, double* z) {
  cudaStream_t st = mg->ctx->stream;
  Level& l = mg->L[0];
  if (mg->L.size() == 1) {
    int its = mg->o.coarse_fixed;
    if (mg->o.coarse_fixed > 0)
      ST(coarse_cheb(mg, l, r, z, false));
    else
      ST(pcg64(mg, l, r, z, mg->o.coarse_rtol, mg->o.coarse_maxit, false, &its));
    mg->coarse_its += its;
    mg->vcycles++;
    return NH_OK;
  }
  if (l.prec == NH_F64) {
    CK(cudaMemcpyAsync(l.b, r, 8 * l.n, cudaMemcpyDeviceToDevice, st));
  } else {
    CK((kv_convert<double, float>(st, l.n, r, (float*)l.b)));
    mg->ctx->launches++;
  }
  ST(vcycle(mg, 0));
  if (l.prec == NH_F64) {
    CK(cudaMemcpyAsync(z, l.x, 8 * l.n, cudaMemcpyDeviceToDevice, st));
  } else {
    CK((kv_convert<float, double>(st, l.n, (const float*)l.x, z)));
    mg->ctx->launches++;
  }
  mg->vcycles++;
  return NH_OK;
}

extern "C" nh_status nh_mg_vcycle(nh_mg mg, const double* r, double* z) {
  if (!mg || !r || !z) return NH_ERR_ARG;
  if (!mg->setup_done) return nh_fail(mg->ctx, NH_ERR_STATE, "nh_mg_vcycle: call nh_mg_setup first");
  CK(cudaSetDevice(mg->ctx->device));
  return vcycle_fp64(mg, r, z);
}

// ---- learned stage ---------------------------------------------------------------
struct Collect {
  const double* xs;  // converged solution (outer mode)
  float* feats;
  float* tgts;
  int max, n;
};

namespace {

// network input for a coarse right-hand side bc: scaled by its RMS (0 if bc = 0)
nh_status coarse_features(nh_mg mg, const double* bc, float* feat, double* scale) {
  Level& c = mg->L.back();
  double rr = 0.0;
  ST(dot_host(mg, c.n, bc, bc, &rr));
  *scale = sqrt(rr / (double)c.n);
  if (!(*scale > 0.0) || !isfinite(*scale)) {
    *scale = 0.0;
    return NH_OK;
  }
  CK(kn_features(mg->ctx->stream, c.nn, bc, 1.0 / *scale, mg->logE, feat));
  mg->ctx->launches++;
  return NH_OK;
}

// the coarsest solve without any learned stage: the fixed polynomial, or the PCG
// chosen by coarse_solver to coarse_rtol
nh_status coarse_plain(nh_mg mg, Level& l, const double* b, double* x, int* its) {
  if (mg->o.coarse_fixed > 0) {
    ST(coarse_cheb(mg, l, b, x, false));
    *its = mg->o.coarse_fixed;
  } else if (mg->hmg_ok && &l == &mg->L.back()) {
    ST(hmg_pcg(mg, l, b, x, mg->o.coarse_rtol, mg->o.coarse_maxit, its));
  } else {
    ST(pcg64(mg, l, b, x, mg->o.coarse_rtol, mg->o.coarse_maxit, false, its));
  }
  return NH_OK;
}

// learned post-correction (learned_mode 3): after the plain coarse solve x1,
// the network predicts the error e1 = A_c^-1 r1 left by it from the residual
// r1 = b - A_c x1, and x = x1 + a y with the step a = y.r1 / y.A_c y that
// minimises the A_c-norm error along the prediction y.  Whenever y.r1 > 0 the
// coarse error strictly decreases in the A_c-norm; otherwise x = x1 (rejected).
nh_status coarse_post_correct(nh_mg mg, Level& l, const double* b, double* x) {
  cudaStream_t st = mg->ctx->stream;
  double *r1 = l.w[4], *y = mg->lc1, *ay = l.w[0];
  ST(level_apply(mg, l, NH_F64, x, r1));
  CK(kv_axpby<double>(st, l.n, 1.0, b, -1.0, r1));  // r1 = b - A x1
  CK(kv_mul<double>(st, l.n, l.dinv64, r1, y));     // network input: D^-1 r1
  mg->ctx->launches += 2;
  double scale = 0.0;
  ST(coarse_features(mg, y, mg->feat, &scale));
  if (scale == 0.0) return NH_OK;
  ST(nh_net_forward_internal(mg->net, mg->feat, mg->nout));
  CK(kn_from_net(st, l.nn, mg->nout, scale, y));
  CK(kv_mask_zero<double>(st, l.nn, l.space->bc, y));
  mg->ctx->launches += 2;
  ST(level_apply(mg, l, NH_F64, y, ay));
  double yr = 0.0, yay = 0.0;
  ST(dot_host(mg, l.n, y, r1, &yr));
  ST(dot_host(mg, l.n, y, ay, &yay));
  if (isfinite(yr) && isfinite(yay) && yr > 0.0 && yay > 0.0) {
    CK(kv_axpby<double>(st, l.n, yr / yay, y, 1.0, x));
    mg->ctx->launches++;
    mg->acc++;
  } else {
    mg->rej++;
  }
  return NH_OK;
}

// learned_mode 4: a coarse space built once per setup.  For probe j (a seeded
// uniform(-1, 1) coarse vector r, constrained entries zeroed) the plain coarse
// solve gives x1 and leaves r1 = r - A_c x1; the network predicts the error
// e1 = A_c^-1 r1 that remains, y_j = N(r1).  The y_j are A_c-orthonormalised
// (classical Gram-Schmidt, twice), dropping any whose A_c-norm falls below
// 1e-8 of its norm before the projection.  Without a network, y_j = x1 (the
// plain solve's own output: the non-learned coarse space of the same size), or,
// with learned_accept = 1, the exact error A_c^-1 r1 (the space a perfect
// network would span; a diagnostic, each vector costs a coarse PCG to 1e-9).
nh_status build_coarse_space(nh_mg mg) {
  Level& l = mg->L.back();
  cudaStream_t st = mg->ctx->stream;
  const int k = mg->o.learned_vectors;
  mg->Wk = 0;
  if (k <= 0) return NH_OK;
  if (mg->Wcap < k) {
    for (void* p : {(void*)mg->W, (void*)mg->Wc, (void*)mg->Wpart}) cudaFree(p);
    mg->W = mg->Wc = mg->Wpart = nullptr;
    mg->Wcap = 0;
    ST(dalloc(mg, (void**)&mg->W, 8 * (size_t)k * l.n));
    ST(dalloc(mg, (void**)&mg->Wc, 8 * 2 * (size_t)k));
    ST(dalloc(mg, (void**)&mg->Wpart, 8 * (size_t)k * kv_multidot_parts()));
    mg->Wcap = k;
  }
  double *r = l.w[4], *x1 = mg->lc1, *y = mg->lc2, *ay = l.w[0];
  for (int j = 0; j < k; j++) {
    CK(kv_uniform(st, l.n, mg->o.seed + 7919ull * (uint64_t)(j + 1), r));
    CK(kv_mask_zero<double>(st, l.nn, l.space->bc, r));
    mg->ctx->launches += 2;
    int its = 0;
    ST(coarse_plain(mg, l, r, x1, &its));
    if (!mg->net && mg->o.learned_accept == 1) {
      // diagnostic: the exact errors the plain solve leaves, A_c^-1 r1 (PCG to 1e-9),
      // i.e. the coarse space a perfect network would give
      ST(level_apply(mg, l, NH_F64, x1, ay));
      CK(kv_axpby<double>(st, l.n, -1.0, ay, 1.0, r));  // r1 = r - A x1
      mg->ctx->launches++;
      int its2 = 0;
      ST(pcg64(mg, l, r, y, 1e-9, 20000, false, &its2));
    } else if (mg->net) {
      ST(level_apply(mg, l, NH_F64, x1, ay));
      CK(kv_axpby<double>(st, l.n, -1.0, ay, 1.0, r));  // r1 = r - A x1
      CK(kv_mul<double>(st, l.n, l.dinv64, r, y));      // network input: D^-1 r1
      mg->ctx->launches += 2;
      double scale = 0.0;
      ST(coarse_features(mg, y, mg->feat, &scale));
      if (scale == 0.0) continue;
      ST(nh_net_forward_internal(mg->net, mg->feat, mg->nout));
      CK(kn_from_net(st, l.nn, mg->nout, scale, y));
      CK(kv_mask_zero<double>(st, l.nn, l.space->bc, y));
      mg->ctx->launches += 2;
    } else {
      CK(cudaMemcpyAsync(y, x1, 8 * l.n, cudaMemcpyDeviceToDevice, st));
    }
    ST(level_apply(mg, l, NH_F64, y, ay));
    double e0 = 0.0;
    ST(dot_host(mg, l.n, y, ay, &e0));
    if (!(e0 > 0.0) || !isfinite(e0)) continue;
    for (int pass = 0; pass < 2 && mg->Wk > 0; pass++) {
      CK(kv_multidot(st, mg->Wk, l.n, mg->W, l.n, ay, mg->Wpart, mg->Wc));  // c = W^T A y
      CK(kv_gemv_rows(st, l.n, mg->Wk, mg->W, l.n, mg->Wc, -1.0, y));      // y -= W c
      mg->ctx->launches += 3;
      ST(level_apply(mg, l, NH_F64, y, ay));
    }
    double e = 0.0;
    ST(dot_host(mg, l.n, y, ay, &e));
    if (!(e > 1e-8 * e0) || !isfinite(e)) continue;
    CK(kv_axpby<double>(st, l.n, 1.0 / sqrt(e), y, 0.0, mg->W + (int64_t)mg->Wk * l.n));
    mg->ctx->launches++;
    mg->Wk++;
  }
  return NH_OK;
}

// Two-level coarse solve with the coarse space W (W^T A_c W = I) around the
// plain coarse solve Q (balancing form):
//   x = W W^T b + (I - W W^T A_c) Q (I - A_c W W^T) b,
// symmetric positive definite for Q SPD, linear, and with no host synchronisation.
nh_status coarse_two_level(nh_mg mg, Level& l, const double* b, double* x, int* its) {
  cudaStream_t st = mg->ctx->stream;
  const int k = mg->Wk;
  double *v = l.w[4], *x1 = mg->lc1, *t = mg->lc2;
  CK(kv_multidot(st, k, l.n, mg->W, l.n, b, mg->Wpart, mg->Wc));  // c = W^T b
  CK(cudaMemsetAsync(x, 0, 8 * l.n, st));
  CK(kv_gemv_rows(st, l.n, k, mg->W, l.n, mg->Wc, 1.0, x));      // x = y0 = W c
  mg->ctx->launches += 3;
  ST(level_apply(mg, l, NH_F64, x, t));
  CK(cudaMemcpyAsync(v, b, 8 * l.n, cudaMemcpyDeviceToDevice, st));
  CK(kv_axpby<double>(st, l.n, -1.0, t, 1.0, v));                // v = b - A y0
  mg->ctx->launches++;
  ST(coarse_plain(mg, l, v, x1, its));
  ST(level_apply(mg, l, NH_F64, x1, t));
  CK(kv_multidot(st, k, l.n, mg->W, l.n, t, mg->Wpart, mg->Wc + k));  // c2 = W^T A x1
  CK(kv_axpby<double>(st, l.n, 1.0, x1, 1.0, x));
  CK(kv_gemv_rows(st, l.n, k, mg->W, l.n, mg->Wc + k, -1.0, x));   // x = y0 + x1 - W c2
  mg->ctx->launches += 4;
  return NH_OK;
}

// coarsest solve (the coarsest level is always FP64), with the learned warm start
// (learned_mode 2) or post-correction (learned_mode 3), and pair recording in
// collection mode
nh_status coarse_solve(nh_mg mg, Level& l) {
  cudaStream_t st = mg->ctx->stream;
  const double* b = (const double*)l.b;
  double* x = (double*)l.x;
  int its = 0;
  if (mg->coll && mg->coll->n < mg->coll->max && mg->o.learned_mode == 3) {
    // collection for the post-correction: the residual r1 the plain solve leaves
    // and its exact correction A^-1 r1 (PCG to 1e-9); the V-cycle goes on with x1
    ST(coarse_plain(mg, l, b, x, &its));
    mg->coarse_its += its;
    double *r1 = l.w[4], *e1 = mg->lc2;
    ST(level_apply(mg, l, NH_F64, x, r1));
    CK(kv_axpby<double>(st, l.n, 1.0, b, -1.0, r1));
    CK(kv_mul<double>(st, l.n, l.dinv64, r1, e1));  // network input: D^-1 r1
    mg->ctx->launches += 2;
    double scale = 0.0;
    float* f = mg->coll->feats + (int64_t)mg->coll->n * 4 * l.nn;
    ST(coarse_features(mg, e1, f, &scale));
    if (scale > 0.0) {
      // target: the exact correction, scaled to unit RMS (only its direction is used)
      int its2 = 0;
      ST(pcg64(mg, l, r1, e1, 1e-9, 20000, false, &its2));
      double ee = 0.0;
      ST(dot_host(mg, l.n, e1, e1, &ee));
      const double rms = sqrt(ee / (double)l.n);
      if (rms > 0.0 && isfinite(rms)) {
        CK(kn_to_channels(st, l.nn, e1, 1.0 / rms, mg->coll->tgts + (int64_t)mg->coll->n * 3 * l.nn));
        mg->ctx->launches++;
        mg->coll->n++;
      }
    }
    return NH_OK;
  }
  if (mg->coll && mg->coll->n < mg->coll->max) {
    // collection: tight solve, store (scaled b, scaled A^-1 b)
    ST(pcg64(mg, l, b, x, 1e-9, 20000, false, &its));
    double scale = 0.0;
    float* f = mg->coll->feats + (int64_t)mg->coll->n * 4 * l.nn;
    ST(coarse_features(mg, b, f, &scale));
    if (scale > 0.0) {
      CK(kn_to_channels(st, l.nn, x, 1.0 / scale, mg->coll->tgts + (int64_t)mg->coll->n * 3 * l.nn));
      mg->ctx->launches++;
      mg->coll->n++;
    }
    mg->coarse_its += its;
    return NH_OK;
  }
  if (mg->net && mg->o.learned_mode == 3) {
    ST(coarse_plain(mg, l, b, x, &its));
    mg->coarse_its += its;
    return coarse_post_correct(mg, l, b, x);
  }
  if (mg->o.learned_mode == 4 && mg->Wk > 0) {
    ST(coarse_two_level(mg, l, b, x, &its));
    mg->coarse_its += its;
    return NH_OK;
  }
  if (mg->net && mg->o.learned_mode == 2) {
    double scale = 0.0;
    ST(coarse_features(mg, b, mg->feat, &scale));
    if (scale > 0.0) {
      ST(nh_net_forward_internal(mg->net, mg->feat, mg->nout));
      CK(kn_from_net(st, l.nn, mg->nout, scale, x));
      CK(kv_mask_zero<double>(st, l.nn, l.space->bc, x));
      mg->ctx->launches += 2;
      // Scale the prediction y by the step that minimises the A-norm error along
      // it, a = y.b / y.A y (||x* - a y||_A <= ||x*||_A), and start the coarse
      // PCG from a y only if that at least halves the residual's natural norm:
      // a start that helps little would make the coarse solve, and so the
      // preconditioner, depend on r_c nonlinearly for no gain.
      double *ay = l.w[0], *z = l.w[1], *rw = l.w[2];
      ST(level_apply(mg, l, NH_F64, x, ay));
      double yb = 0.0, yay = 0.0, bb = 0.0;
      ST(dot_host(mg, l.n, x, b, &yb));
      ST(dot_host(mg, l.n, x, ay, &yay));
      CK(kv_mul<double>(st, l.n, l.dinv64, b, z));
      mg->ctx->launches++;
      ST(dot_host(mg, l.n, b, z, &bb));
      if (isfinite(yb) && isfinite(yay) && yb > 0.0 && yay > 0.0) {
        const double a = yb / yay;
        CK(cudaMemcpyAsync(rw, b, sizeof(double) * l.n, cudaMemcpyDeviceToDevice, st));
        CK(kv_axpby<double>(st, l.n, -a, ay, 1.0, rw));  // r = b - a A y
        CK(kv_mul<double>(st, l.n, l.dinv64, rw, z));
        mg->ctx->launches += 2;
        double rz = 0.0;
        ST(dot_host(mg, l.n, rw, z, &rz));
        if (isfinite(rz) && rz < 0.25 * bb) {
          CK(kv_axpby<double>(st, l.n, a, x, 0.0, z));  // x = a y
          CK(cudaMemcpyAsync(x, z, sizeof(double) * l.n, cudaMemcpyDeviceToDevice, st));
          mg->ctx->launches++;
          if (mg->o.coarse_fixed > 0) {  // the fixed polynomial, started from a y
            ST(coarse_cheb(mg, l, b, x, true));
            its = mg->o.coarse_fixed;
          } else {
            ST(pcg64(mg, l, b, x, mg->o.coarse_rtol, mg->o.coarse_maxit, false, &its, true, sqrt(bb)));
          }
          mg->coarse_its += its;
          mg->acc++;
          return NH_OK;
        }
      }
      mg->rej++;
    }
  }
  ST(coarse_plain(mg, l, b, x, &its));
  mg->coarse_its += its;
  return NH_OK;
}

}  // namespace

// network input for the fine residual r: restrict through the levels to Q1,
// scale by the RMS of the restricted residual.  Returns the scale (0 if r = 0).
static nh_status learned_features(nh_mg mg, const double* r, float* feat, double* scale) {
  cudaStream_t st = mg->ctx->stream;
  const double* cur = r;
  for (size_t l = 0; l + 1 < mg->L.size(); l++) {
    Level& c = mg->L[l + 1];
    ST(nh_transfer_internal(c.space, mg->L[l].space, NH_F64, 1, cur, c.w[4]));
    CK(kv_mask_zero<double>(st, c.nn, c.space->bc, c.w[4]));
    mg->ctx->launches++;
    cur = c.w[4];
  }
  Level& c = mg->L.back();
  double rr = 0.0;
  ST(dot_host(mg, c.n, cur, cur, &rr));
  *scale = sqrt(rr / (double)c.n);
  if (!(*scale > 0.0) || !isfinite(*scale)) {
    *scale = 0.0;
    return NH_OK;
  }
  CK(kn_features(st, c.nn, cur, 1.0 / *scale, mg->logE, feat));
  mg->ctx->launches++;
  return NH_OK;
}

static nh_status vcycle_fp64(nh_mg mg, const double* r, double* z);

// z = M r with the learned stage in front of the V-cycle (see nh_mg_set_learned)
static nh_status precond(nh_mg mg, const double* r, double* z) {
  if (!mg->net || mg->o.learned_mode != 1) return vcycle_fp64(mg, r, z);
  cudaStream_t st = mg->ctx->stream;
  double scale = 0.0;
  ST(learned_features(mg, r, mg->feat, &scale));
  if (scale == 0.0) return vcycle_fp64(mg, r, z);
  ST(nh_net_forward_internal(mg->net, mg->feat, mg->nout));
  Level& c = mg->L.back();
  CK(kn_from_net(st, c.nn, mg->nout, scale, c.w[3]));
  mg->ctx->launches++;
  const double* cur = c.w[3];
  for (int l = (int)mg->L.size() - 2; l >= 0; l--) {
    double* out = l == 0 ? mg->lz1 : mg->L[l].w[4];
    ST(nh_transfer_internal(mg->L[l + 1].space, mg->L[l].space, NH_F64, 0, cur, out));
    CK(kv_mask_zero<double>(st, mg->L[l].nn, mg->L[l].space->bc, out));
    mg->ctx->launches++;
    cur = out;
  }
  const int64_t n = mg->L[0].n;
  ST(nh_jacobian_apply(mg->fine, mg->p64, mg->lz1, mg->lw));  // lw = J z1
  bool accept = false;
  if (mg->o.learned_accept == 1) {
    // energy-optimal step: a = z1.r / z1.J z1; the A-norm of the error drops iff z1.r > 0
    double zr = 0.0, zaz = 0.0;
    ST(dot_host(mg, n, mg->lz1, r, &zr));
    ST(dot_host(mg, n, mg->lz1, mg->lw, &zaz));
    if (isfinite(zr) && isfinite(zaz) && zr > 0.0 && zaz > 0.0) {
      const double a = zr / zaz;
      CK(kv_axpby<double>(st, n, 1.0, r, -a, mg->lw));  // w = r - a J z1
      CK(kv_axpby<double>(st, n, 0.0, mg->lz1, a, mg->lz1));
      mg->ctx->launches += 2;
      accept = true;
    }
  } else {
    CK(kv_axpby<double>(st, n, 1.0, r, -1.0, mg->lw));  // w = r - J z1
    mg->ctx->launches++;
    double nw = 0.0, nr = 0.0;
    ST(dot_host(mg, n, mg->lw, mg->lw, &nw));
    ST(dot_host(mg, n, r, r, &nr));
    accept = isfinite(nw) && nw < nr;
  }
  if (accept) {
    ST(vcycle_fp64(mg, mg->lw, z));
    CK(kv_axpby<double>(st, n, 1.0, mg->lz1, 1.0, z));
    mg->ctx->launches++;
    mg->acc++;
  } else {
    ST(vcycle_fp64(mg, r, z));
    mg->rej++;
  }
  return NH_OK;
}

static nh_status record_pair(nh_mg mg, Collect* col, const double* r, const double* x) {
  if (!col || col->n >= col->max) return NH_OK;
  cudaStream_t st = mg->ctx->stream;
  Level& c = mg->L.back();
  const int64_t nc = c.nn;
  float* f = col->feats + (int64_t)col->n * 4 * nc;
  float* t = col->tgts + (int64_t)col->n * 3 * nc;
  double scale = 0.0;
  ST(learned_features(mg, r, f, &scale));
  if (scale == 0.0) return NH_OK;
  const int64_t n = mg->L[0].n;
  CK(cudaMemcpyAsync(mg->lt, col->xs, 8 * n, cudaMemcpyDeviceToDevice, st));
  CK(kv_axpby<double>(st, n, -1.0, x, 1.0, mg->lt));  // x* - x
  nh_space fs = mg->L[0].space;
  CK(kn_inject(st, c.space->Nx, fs->p, fs->Nx, mg->lt, 1.0 / scale, t));
  mg->ctx->launches += 2;
  col->n++;
  return NH_OK;
}

// FCG(1): J x = b, x in/out; returns iterations, final relative norm
static nh_status fcg(nh_mg mg, const double* b, double* x, double rtol, int maxit, int norm, int* its_out,
                     double* rel_out, Collect* col = nullptr) {
  cudaStream_t st = mg->ctx->stream;
  nh_op A = mg->fine;
  const int64_t n = mg->L[0].n;
  double *r = mg->fr, *z = mg->fz, *p = mg->fp, *q = mg->fq;
  ST(nh_jacobian_apply(A, mg->p64, x, r));
  CK(kv_axpby<double>(st, n, 1.0, b, -1.0, r));  // r = b - A x
  mg->ctx->launches++;
  ST(record_pair(mg, col, r, x));
  ST(precond(mg, r, z));
  CK(cudaMemcpyAsync(p, z, 8 * n, cudaMemcpyDeviceToDevice, st));
  ST(nh_jacobian_apply(A, mg->p64, p, q));
  double nrm0 = 0.0;
  ST(norm == 0 ? dot(mg, n, r, z, S_FRR) : dot(mg, n, r, r, S_FRR));
  ST(read_sc(mg, S_FRR, 1, &nrm0));
  nrm0 = sqrt(fabs(nrm0));
  if (!isfinite(nrm0)) return nh_fail(mg->ctx, NH_ERR_NAN, "FCG: non-finite initial residual");
  double nrm = nrm0;
  int k = 0;
  if (nrm0 == 0.0) {
    *its_out = 0;
    *rel_out = 0.0;
    return NH_OK;
  }
  while (k < maxit) {
    ST(dot(mg, n, p, q, S_FPQ));
    ST(dot(mg, n, p, r, S_FPR));
    CK(kv_cg_update<double>(st, n, p, q, x, r, mg->sc, S_FPR, S_FPQ));  // x += a p, r -= a q
    mg->ctx->launches++;
    k++;
    ST(record_pair(mg, col, r, x));
    ST(precond(mg, r, z));
    ST(norm == 0 ? dot(mg, n, r, z, S_FRR) : dot(mg, n, r, r, S_FRR));
    ST(read_sc(mg, S_FRR, 1, &nrm));
    nrm = sqrt(fabs(nrm));
    if (!isfinite(nrm)) return nh_fail(mg->ctx, NH_ERR_NAN, "FCG: non-finite residual");
    if (nrm <= rtol * nrm0) break;
    ST(dot(mg, n, z, q, S_FZQ));
    CK(kv_xpby_dev<double>(st, n, z, p, mg->sc, S_FZQ, S_FPQ, -1.0));  // p = z - (z.q / p.q) p
    mg->ctx->launches++;
    ST(nh_jacobian_apply(A, mg->p64, p, q));
  }
  *its_out = k;
  *rel_out = nrm / nrm0;
  return NH_OK;
}

extern "C" nh_status nh_linear_solve(nh_mg mg, const double* b, double* x, double rtol, int maxit, int norm,
                                     nh_solve_report* rep) {
  if (!mg || !b || !x) return NH_ERR_ARG;
  if (!mg->setup_done) return nh_fail(mg->ctx, NH_ERR_STATE, "nh_linear_solve: call nh_mg_setup first");
  CK(cudaSetDevice(mg->ctx->device));
  auto t0 = std::chrono::steady_clock::now();
  mg->vcycles = mg->coarse_its = 0;
  mg->acc = mg->rej = 0;
  int its = 0;
  double rel = 0.0;
  nh_status s = fcg(mg, b, x, rtol, maxit, norm, &its, &rel);
  CK(cudaStreamSynchronize(mg->ctx->stream));
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    rep->krylov_its = its;
    rep->vcycles = mg->vcycles;
    rep->coarse_its = mg->coarse_its;
    rep->rel_residual = rel;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rep->t_krylov = rep->seconds;
    rep->learned_accepted = mg->acc;
    rep->learned_rejected = mg->rej;
  }
  if (s == NH_OK && rel > rtol) s = nh_fail(mg->ctx, NH_ERR_NOT_CONVERGED, "nh_linear_solve: maxit reached");
  if (rep) rep->status = s;
  return s;
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ||F(v)||_2 with F evaluated into `out`; non-finite when v inverts an element
static nh_status resid_norm(nh_mg mg, const double* v, const double* g, double* out, double* nrm) {
  ST(nh_residual(mg->fine, v, g, out));
  double s2 = 0.0;
  ST(dot_host(mg, mg->L[0].n, out, out, &s2));
  *nrm = sqrt(s2);
  return NH_OK;
}

// L-BFGS direction (Sec. III-A, the quasi-Newton alternative to Newton-Krylov):
// d = -H F by the two-loop recursion over the stored pairs (s_i, y_i), oldest
// last, with one V-cycle of the load step's tangent as the initial inverse
// Hessian H_0.  hist[j] indexes the pairs from newest to oldest; rho[j] = 1 / y.s.
static nh_status lbfgs_direction(nh_mg mg, const double* F, double* d, double* q, const std::vector<int>& hist,
                                 const std::vector<double>& rho) {
  cudaStream_t st = mg->ctx->stream;
  const int64_t n = mg->L[0].n;
  const int k = (int)hist.size();
  std::vector<double> alpha(k, 0.0);
  CK(cudaMemcpyAsync(q, F, 8 * n, cudaMemcpyDeviceToDevice, st));
  for (int j = 0; j < k; j++) {
    double sq = 0.0;
    ST(dot_host(mg, n, mg->lbs[hist[j]], q, &sq));
    alpha[j] = rho[j] * sq;
    CK(kv_axpby<double>(st, n, -alpha[j], mg->lby[hist[j]], 1.0, q));
    mg->ctx->launches++;
  }
  ST(precond(mg, q, d));  // d = H_0 q
  for (int j = k - 1; j >= 0; j--) {
    double yd = 0.0;
    ST(dot_host(mg, n, mg->lby[hist[j]], d, &yd));
    CK(kv_axpby<double>(st, n, alpha[j] - rho[j] * yd, mg->lbs[hist[j]], 1.0, d));
    mg->ctx->launches++;
  }
  CK(kv_axpby<double>(st, n, 0.0, d, -1.0, d));  // d = -H F
  mg->ctx->launches++;
  return NH_OK;
}

extern "C" nh_status nh_solve(nh_mg mg, const double* g_bc, double* u, nh_solve_report* rep) {
  if (!mg || !u) return NH_ERR_ARG;
  nh_ctx ctx = mg->ctx;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  nh_op F = mg->fine;
  nh_space fs = F->space;
  const nh_mg_opts& o = mg->o;
  const int64_t n = fs->n_dof;
  double *r = mg->fu, *gk = mg->fg, *du = mg->fx, *rhs = mg->fb;
  double *ut = mg->ft, *rt = mg->fs;  // trial point and its residual; ut also holds the lift w
  nh_solve_report R;
  memset(&R, 0, sizeof(R));
  mg->acc = mg->rej = 0;
  const double T0 = now_s();
  double tS = 0, tK = 0, tR = 0;
  nh_status status = NH_OK;
  const int K = std::max(1, o.load_steps);
  double rel = 0.0, nr = 0.0;
  double t_prev = 0.0;
  int halvings = 0;
  double nr_step = 0.0;  // initial residual of the current load step's first attempt
  auto setup = [&](const double* v, double* minJ) -> nh_status {
    const double t1 = now_s();
    nh_status s = nh_qdata_setup(F, v, minJ);
    if (s == NH_OK) s = nh_mg_setup(mg);
    tS += now_s() - t1;
    return s;
  };
  auto krylov = [&](const double* b, double* x) -> nh_status {
    const double t1 = now_s();
    int kits = 0;
    double krel = 0.0;
    mg->vcycles = 0;
    mg->coarse_its = 0;
    CK(cudaMemsetAsync(x, 0, 8 * n, st));
    nh_status s = fcg(mg, b, x, o.krylov_rtol, o.krylov_maxit, 0, &kits, &krel);
    R.krylov_its += kits;
    R.vcycles += mg->vcycles;
    R.coarse_its += mg->coarse_its;
    tK += now_s() - t1;
    return s;
  };
  int step = 0;
  while (step < K && status == NH_OK) {
    const double t_target = (double)(step + 1) / K;
    const double t = t_prev + (t_target - t_prev) / (double)(1 << halvings);
    double t1 = now_s();
    if (g_bc) {
      CK(cudaMemcpyAsync(gk, g_bc, 8 * n, cudaMemcpyDeviceToDevice, st));
      CK(kv_axpby<double>(st, n, 0.0, gk, t, gk));
    } else {
      CK(cudaMemsetAsync(gk, 0, 8 * n, st));
    }
    ctx->launches++;
    tR += now_s() - t1;
    CK(cudaMemcpyAsync(mg->fsave, u, 8 * n, cudaMemcpyDeviceToDevice, st));
    // --- predictor: carry the boundary increment w = g_k - u (constrained DoFs) into
    // the interior through the tangent at the current state:
    //   J_uu du = -(F_u(u) + J_uc w),   u <- u + w + du
    double minJ = 0.0;
    status = setup(u, &minJ);
    if (status != NH_OK) break;
    t1 = now_s();
    CK(cudaMemcpyAsync(ut, gk, 8 * n, cudaMemcpyDeviceToDevice, st));
    CK(kv_axpby<double>(st, n, -1.0, u, 1.0, ut));  // ut = g_k - u
    CK(kv_mask_keep(st, fs->n_nodes, fs->bc, ut));   // w: constrained entries only
    ctx->launches += 2;
    ST(nh_residual(F, u, gk, r));
    CK(kv_mask_zero<double>(st, fs->n_nodes, fs->bc, r));  // F_u(u)
    ST(nh_jacobian_apply_lift(F, ut, rhs));                 // J_uc w
    CK(kv_axpby<double>(st, n, -1.0, r, -1.0, rhs));       // rhs = -(F_u + J_uc w)
    ctx->launches += 2;
    tR += now_s() - t1;
    status = krylov(rhs, du);
    if (status != NH_OK) break;
    t1 = now_s();
    CK(kv_axpby<double>(st, n, 1.0, ut, 1.0, du));  // du = w + du
    CK(cudaMemcpyAsync(ut, u, 8 * n, cudaMemcpyDeviceToDevice, st));
    CK(kv_axpby<double>(st, n, 1.0, du, 1.0, ut));  // ut = u + w + du
    ctx->launches += 2;
    double nr0 = 0.0;
    ST(resid_norm(mg, ut, gk, r, &nr0));
    tR += now_s() - t1;
    if (!isfinite(nr0)) {
      // the predicted state inverts an element: halve this load increment
      if (++halvings > 8) {
        status = nh_fail(ctx, NH_ERR_INVERTED, "nh_solve: load increment cannot be halved further");
        break;
      }
      continue;
    }
    CK(cudaMemcpyAsync(u, ut, 8 * n, cudaMemcpyDeviceToDevice, st));
    nr = nr0;
    // the tolerance refers to the load step, not to a halved sub-increment of it
    if (t_target - t_prev >= (t_target - t) * 1.000001 && halvings == 0) nr_step = nr0;
    nr0 = std::max(nr0, nr_step);
    int it = 0;
    if (o.nonlinear == 1) {
      // --- L-BFGS corrector at fixed t, H_0 = V-cycle of the tangent at the predicted state
      status = setup(u, &minJ);
      if (status != NH_OK) break;
      if (mg->lbs.empty()) {
        for (int j = 0; j < o.lbfgs_m; j++) {
          double *sv = nullptr, *yv = nullptr;
          ST(dalloc(mg, (void**)&sv, 8 * n));
          mg->lbs.push_back(sv);
          ST(dalloc(mg, (void**)&yv, 8 * n));
          mg->lby.push_back(yv);
        }
        ST(dalloc(mg, (void**)&mg->lbr, 8 * n));
      }
      std::vector<int> hist;     // slots, newest first
      std::vector<double> rho;
      int next = 0;
      const int maxit = 4 * o.newton_maxit;
      while (!(nr <= o.newton_rtol * nr0) && !(nr <= o.newton_atol)) {
        if (it >= maxit || (it >= 40 && nr > 1e-4 * nr0)) {
          status = nh_fail(ctx, NH_ERR_NOT_CONVERGED, "nh_solve: L-BFGS iteration limit");
          break;
        }
        t1 = now_s();
        mg->vcycles = 0;
        mg->coarse_its = 0;
        ST(lbfgs_direction(mg, r, du, rhs, hist, rho));
        R.vcycles += mg->vcycles;
        R.coarse_its += mg->coarse_its;
        tK += now_s() - t1;
        t1 = now_s();
        double at = 1.0, nrt = 0.0;
        for (int bt = 0;; bt++) {
          CK(cudaMemcpyAsync(ut, u, 8 * n, cudaMemcpyDeviceToDevice, st));
          CK(kv_axpby<double>(st, n, at, du, 1.0, ut));
          ctx->launches++;
          ST(resid_norm(mg, ut, gk, rt, &nrt));
          if (isfinite(nrt)) break;
          if (bt >= 12) {
            status = nh_fail(ctx, NH_ERR_INVERTED, "nh_solve: every trial step inverts an element");
            break;
          }
          at *= 0.5;
        }
        if (status != NH_OK) break;
        double alpha = at;
        if (o.line_search) {
          double phi0 = 0.0, phi1 = 0.0;
          ST(dot_host(mg, n, r, du, &phi0));
          ST(dot_host(mg, n, rt, du, &phi1));
          if (phi0 * phi1 < 0.0) {
            const double a = at * phi0 / (phi0 - phi1);
            if (isfinite(a)) alpha = std::min(at < 1.0 ? at : 1.5, std::max(0.1 * at, a));
          }
        }
        // new pair in slot `next`: s = alpha du, y = F(u + s) - F(u)
        double* sv = mg->lbs[next];
        double* yv = mg->lby[next];
        CK(cudaMemcpyAsync(mg->lbr, r, 8 * n, cudaMemcpyDeviceToDevice, st));
        if (alpha == at) {
          CK(cudaMemcpyAsync(u, ut, 8 * n, cudaMemcpyDeviceToDevice, st));
          CK(cudaMemcpyAsync(r, rt, 8 * n, cudaMemcpyDeviceToDevice, st));
          nr = nrt;
        } else {
          CK(cudaMemcpyAsync(ut, u, 8 * n, cudaMemcpyDeviceToDevice, st));
          CK(kv_axpby<double>(st, n, alpha, du, 1.0, ut));
          ctx->launches++;
          double nra = 0.0;
          ST(resid_norm(mg, ut, gk, rt, &nra));
          if (!isfinite(nra)) {  // keep the backtracked trial step
            alpha = at;
            CK(cudaMemcpyAsync(ut, u, 8 * n, cudaMemcpyDeviceToDevice, st));
            CK(kv_axpby<double>(st, n, at, du, 1.0, ut));
            ctx->launches++;
            ST(resid_norm(mg, ut, gk, rt, &nra));
          }
          CK(cudaMemcpyAsync(u, ut, 8 * n, cudaMemcpyDeviceToDevice, st));
          CK(cudaMemcpyAsync(r, rt, 8 * n, cudaMemcpyDeviceToDevice, st));
          nr = nra;
        }
        CK(kv_axpby<double>(st, n, alpha, du, 0.0, sv));          // s
        CK(cudaMemcpyAsync(yv, r, 8 * n, cudaMemcpyDeviceToDevice, st));
        CK(kv_axpby<double>(st, n, -1.0, mg->lbr, 1.0, yv));     // y (constrained rows are zero in both)
        ctx->launches += 2;
        double ys = 0.0;
        ST(dot_host(mg, n, yv, sv, &ys));
        if (ys > 0.0 && isfinite(ys)) {  // curvature condition, else the pair is dropped
          if ((int)hist.size() == o.lbfgs_m) {
            hist.pop_back();
            rho.pop_back();
          }
          hist.insert(hist.begin(), next);
          rho.insert(rho.begin(), 1.0 / ys);
          next = (next + 1) % o.lbfgs_m;
        }
        tR += now_s() - t1;
        it++;
        R.newton_its++;
        if (o.verbose)
          fprintf(stderr, "nh_solve t %.4f lbfgs %d |F| %.3e rel %.3e vcyc %d alpha %.3f pairs %d\n", t, it, nr,
                  nr / nr0, R.vcycles, alpha, (int)hist.size());
      }
    }
    // --- Newton corrector at fixed t
    while (o.nonlinear == 0 && !(nr <= o.newton_rtol * nr0) && !(nr <= o.newton_atol)) {
      if (it >= o.newton_maxit || (it >= 10 && nr > 1e-4 * nr0)) {  // limit, or stagnation
        status = nh_fail(ctx, NH_ERR_NOT_CONVERGED, "nh_solve: Newton iteration limit");
        break;
      }
      status = setup(u, &minJ);
      if (status != NH_OK) break;
      CK(kv_axpby<double>(st, n, -1.0, r, 0.0, rhs));  // rhs = -F(u)
      ctx->launches++;
      status = krylov(rhs, du);
      if (status != NH_OK) break;
      // line search: backtrack while the trial state inverts, then one secant
      // step on phi(a) = F(u + a du) . du (critical point)
      t1 = now_s();
      double at = 1.0, nrt = 0.0;
      for (int bt = 0;; bt++) {
        CK(cudaMemcpyAsync(ut, u, 8 * n, cudaMemcpyDeviceToDevice, st));
        CK(kv_axpby<double>(st, n, at, du, 1.0, ut));
        ctx->launches++;
        ST(resid_norm(mg, ut, gk, rt, &nrt));
        if (isfinite(nrt)) break;
        if (bt >= 12) {
          status = nh_fail(ctx, NH_ERR_INVERTED, "nh_solve: every trial step inverts an element");
          break;
        }
        at *= 0.5;
      }
      if (status != NH_OK) break;
      double alpha = at;
      if (o.line_search) {
        double phi0 = 0.0, phi1 = 0.0;
        ST(dot_host(mg, n, r, du, &phi0));
        ST(dot_host(mg, n, rt, du, &phi1));
        if (phi0 * phi1 < 0.0) {
          const double a = at * phi0 / (phi0 - phi1);
          if (isfinite(a)) alpha = std::min(at < 1.0 ? at : 1.5, std::max(0.1 * at, a));
        }
      }
      bool took_trial = (alpha == at);
      if (!took_trial) {
        CK(cudaMemcpyAsync(rhs, u, 8 * n, cudaMemcpyDeviceToDevice, st));
        CK(kv_axpby<double>(st, n, alpha, du, 1.0, rhs));
        ctx->launches++;
        double nra = 0.0;
        ST(resid_norm(mg, rhs, gk, r, &nra));
        if (isfinite(nra)) {
          CK(cudaMemcpyAsync(u, rhs, 8 * n, cudaMemcpyDeviceToDevice, st));
          nr = nra;
        } else {
          took_trial = true;
          alpha = at;
        }
      }
      if (took_trial) {
        CK(cudaMemcpyAsync(u, ut, 8 * n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(r, rt, 8 * n, cudaMemcpyDeviceToDevice, st));
        nr = nrt;
      }
      tR += now_s() - t1;
      it++;
      R.newton_its++;
      if (o.verbose)
        fprintf(stderr, "nh_solve t %.4f newton %d |F| %.3e rel %.3e fcg %d vcyc %d coarse %d alpha %.3f minJ %.3f\n",
                t, it, nr, nr / nr0, R.krylov_its, mg->vcycles, mg->coarse_its, alpha, minJ);
    }
    rel = nr0 > 0 ? nr / nr0 : 0.0;
    if (status == NH_ERR_NOT_CONVERGED || status == NH_ERR_INVERTED) {
      // the increment was too large for Newton: restore its start state and halve it
      CK(cudaMemcpyAsync(u, mg->fsave, 8 * n, cudaMemcpyDeviceToDevice, st));
      if (++halvings > 8) {
        status = nh_fail(ctx, NH_ERR_NOT_CONVERGED, "nh_solve: load increment cannot be halved further");
        break;
      }
      if (o.verbose) fprintf(stderr, "nh_solve t %.4f: Newton failed, halving the increment\n", t);
      status = NH_OK;
      continue;
    }
    if (status != NH_OK) break;
    t_prev = t;
    if (halvings > 0 && t < t_target) {
      halvings--;  // retry the rest of the increment with a larger step
    } else {
      halvings = 0;
      nr_step = 0.0;
      step++;
      R.load_steps = step;
    }
  }
  CK(cudaStreamSynchronize(st));
  R.status = status;
  R.rel_residual = rel;
  R.abs_residual = nr;
  R.seconds = now_s() - T0;
  R.t_setup = tS;
  R.t_krylov = tK;
  R.t_residual = tR;
  R.learned_accepted = mg->acc;
  R.learned_rejected = mg->rej;
  if (rep) *rep = R;
  return status;
}

// ---------------------------------------------------------------------------
// learned stage: buffers, ABI
// ---------------------------------------------------------------------------
static nh_status learned_buffers(nh_mg mg) {
  if (mg->feat) return NH_OK;
  Level& c = mg->L.back();
  nh_space fs = mg->L[0].space;
  if (mg->L.size() < 2 || c.p != 1 || fs->nx != fs->ny || fs->nx != fs->nz || !(fs->nx % 2 == 0))
    return nh_fail(mg->ctx, NH_ERR_UNSUPPORTED,
                   "learned stage: needs a hierarchy ending at p = 1 on an n^3 mesh with n even");
  const int64_t nc = c.nn, n = mg->L[0].n;
  nh_status s;
  for (void** v : {(void**)&mg->feat, (void**)&mg->logE})
    if ((s = dalloc(mg, v, sizeof(float) * 4 * nc)) != NH_OK) return s;
  if ((s = dalloc(mg, (void**)&mg->nout, sizeof(float) * 3 * nc)) != NH_OK) return s;
  for (double** v : {&mg->lz1, &mg->lw, &mg->lxs, &mg->lx, &mg->lt})
    if ((s = dalloc(mg, (void**)v, 8 * n)) != NH_OK) return s;
  for (double** v : {&mg->lc1, &mg->lc2})
    if ((s = dalloc(mg, (void**)v, 8 * c.n)) != NH_OK) return s;
  // log10 E at the vertices: mean over the adjacent elements, E = 2 mu (1 + nu)
  nh_op root = mg->fine;
  std::vector<double> mu((size_t)fs->ne);
  CK(cudaMemcpy(mu.data(), root->mu, 8 * fs->ne, cudaMemcpyDeviceToHost));
  const int nx = fs->nx, V = nx + 1;
  std::vector<float> le((size_t)nc, 0.f);
  for (int k = 0; k < V; k++)
    for (int j = 0; j < V; j++)
      for (int i = 0; i < V; i++) {
        double acc = 0.0;
        int cnt = 0;
        for (int dk = -1; dk <= 0; dk++)
          for (int dj = -1; dj <= 0; dj++)
            for (int di = -1; di <= 0; di++) {
              const int ei = i + di, ej = j + dj, ek = k + dk;
              if (ei < 0 || ej < 0 || ek < 0 || ei >= nx || ej >= nx || ek >= nx) continue;
              acc += log10(2.0 * mu[ei + (int64_t)nx * (ej + (int64_t)nx * ek)] * (1.0 + root->nu));
              cnt++;
            }
        le[i + (int64_t)V * (j + (int64_t)V * k)] = (float)(acc / cnt);
      }
  CK(cudaMemcpy(mg->logE, le.data(), sizeof(float) * nc, cudaMemcpyHostToDevice));
  return NH_OK;
}

extern "C" nh_status nh_mg_set_learned(nh_mg mg, nh_net net) {
  if (!mg) return NH_ERR_ARG;
  if (!net) {
    mg->net = nullptr;
    return NH_OK;
  }
  if (mg->L[0].space->hex)
    return nh_fail(mg->ctx, NH_ERR_UNSUPPORTED, "nh_mg_set_learned: the network runs on the box mesh's Q1 grid");
  CK(cudaSetDevice(mg->ctx->device));
  ST(learned_buffers(mg));
  if (nh_net_grid(net) != (int)mg->L.back().space->Nx)
    return nh_fail(mg->ctx, NH_ERR_ARG, "nh_mg_set_learned: network grid does not match the Q1 vertex grid");
  mg->net = net;
  return NH_OK;
}

extern "C" nh_status nh_mg_collect(nh_mg mg, const double* b, int max_pairs, float* feats, float* targets,
                                   int* n_pairs) {
  if (!mg || !b || !feats || !targets || !n_pairs || max_pairs < 1) return NH_ERR_ARG;
  if (!mg->setup_done) return nh_fail(mg->ctx, NH_ERR_STATE, "nh_mg_collect: call nh_mg_setup first");
  if (mg->L[0].space->hex)
    return nh_fail(mg->ctx, NH_ERR_UNSUPPORTED, "nh_mg_collect: pairs live on the box mesh's Q1 grid");
  CK(cudaSetDevice(mg->ctx->device));
  ST(learned_buffers(mg));
  nh_net keep = mg->net;
  mg->net = nullptr;  // pairs describe the plain V-cycle's iterates
  const int64_t n = mg->L[0].n;
  cudaStream_t st = mg->ctx->stream;
  int its = 0;
  double rel = 0.0;
  if (mg->o.learned_mode == 2 || mg->o.learned_mode == 3) {
    Collect col{nullptr, feats, targets, max_pairs, 0};
    mg->coll = &col;
    CK(cudaMemsetAsync(mg->lx, 0, 8 * n, st));
    nh_status s = fcg(mg, b, mg->lx, mg->o.krylov_rtol, mg->o.krylov_maxit, 0, &its, &rel);
    mg->coll = nullptr;
    mg->net = keep;
    *n_pairs = col.n;
    CK(cudaStreamSynchronize(st));
    return s;
  }
  CK(cudaMemsetAsync(mg->lxs, 0, 8 * n, st));
  nh_status s = fcg(mg, b, mg->lxs, 1e-10, 2000, 1, &its, &rel);
  if (s == NH_OK) {
    Collect col{mg->lxs, feats, targets, max_pairs, 0};
    CK(cudaMemsetAsync(mg->lx, 0, 8 * n, st));
    s = fcg(mg, b, mg->lx, mg->o.krylov_rtol, std::min(mg->o.krylov_maxit, max_pairs), 0, &its, &rel, &col);
    *n_pairs = col.n;
  }
  mg->net = keep;
  CK(cudaStreamSynchronize(st));
  return s;
}

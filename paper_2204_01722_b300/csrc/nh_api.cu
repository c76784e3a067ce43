// C ABI of the nh library (declared in include/nh.h): contexts, spaces,
// operators and the stream-ordered calls that launch the fused kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nh_internal.cuh"
#include "nh_krylov.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
nh_status nh_fail(nh_ctx ctx, nh_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

nh_status nh_cuda_check(nh_ctx ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // clear the non-sticky error
    return nh_fail(ctx, NH_ERR_OOM, m);
  }
  return nh_fail(ctx, NH_ERR_CUDA, m);
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// ---------------------------------------------------------------------------
// launcher dispatch over P
// ---------------------------------------------------------------------------
cudaError_t nh_launch_apply(int P, int Q, nh_prec prec, const OpArgs& a, cudaStream_t s) {
  switch (P) {
    case 2: return nh_launch_apply_P2(Q, prec, a, s);
    case 3: return nh_launch_apply_P3(Q, prec, a, s);
    case 4: return nh_launch_apply_P4(Q, prec, a, s);
    case 5: return nh_launch_apply_P5(Q, prec, a, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t nh_launch_setup(int P, int Q, const OpArgs& a, cudaStream_t s) {
  switch (P) {
    case 2: return nh_launch_setup_P2(Q, a, s);
    case 3: return nh_launch_setup_P3(Q, a, s);
    case 4: return nh_launch_setup_P4(Q, a, s);
    case 5: return nh_launch_setup_P5(Q, a, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t nh_launch_diag(int P, int Q, const OpArgs& a, cudaStream_t s) {
  switch (P) {
    case 2: return nh_launch_diag_P2(Q, a, s);
    case 3: return nh_launch_diag_P3(Q, a, s);
    case 4: return nh_launch_diag_P4(Q, a, s);
    case 5: return nh_launch_diag_P5(Q, a, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
static const int kRedBlocks = 148 * 8;
static const size_t kMaxProfEvents = 2 * 65536;

extern "C" nh_status nh_create(nh_ctx* out, int device, void* cuda_stream) {
  if (!out) return NH_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return NH_ERR_CUDA;
  nh_ctx c = new nh_ctx_s();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return NH_ERR_CUDA;
    }
    c->own_stream = true;
  }
  c->red_len = kRedBlocks + 8;
  if (cudaMalloc(&c->red, c->red_len * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->minj, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->dev_err, sizeof(int)) != cudaSuccess || cudaMemset(c->dev_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->red_host, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (c->red) cudaFree(c->red);
    if (c->minj) cudaFree(c->minj);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NH_ERR_OOM;
  }
  *out = c;
  return NH_OK;
}

extern "C" nh_status nh_destroy(nh_ctx c) {
  if (!c) return NH_ERR_ARG;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c->ev_chunk) cudaEventDestroy(ev);
  if (c->s_in) cudaStreamDestroy(c->s_in);
  if (c->s_out) cudaStreamDestroy(c->s_out);
  if (c->s_k2) cudaStreamDestroy(c->s_k2);
  cudaFree(c->red);
  cudaFree(c->minj);
  cudaFree(c->dev_err);
  cudaFreeHost(c->red_host);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return NH_OK;
}

extern "C" nh_status nh_debug_wait_timeout(nh_ctx c, int kind) {
  if (!c || (kind != 0 && kind != 1)) return NH_ERR_ARG;
  NH_CUDA(c, cudaSetDevice(c->device));
  if (kind == 0) {
    NH_CUDA(c, nh_launch_wait_timeout_mbar(c->stream, c->dev_err));
  } else {
    unsigned* bar = nullptr;
    NH_CUDA(c, cudaMalloc(&bar, 2 * sizeof(unsigned)));
    cudaError_t e = ks_wait_timeout_grid(c->stream, bar, c->dev_err);
    cudaStreamSynchronize(c->stream);
    cudaFree(bar);
    NH_CUDA(c, e);
  }
  c->launches++;
  return NH_OK;
}

extern "C" const char* nh_last_error(nh_ctx c) { return c ? c->err.c_str() : "null context"; }

extern "C" nh_status nh_sync(nh_ctx c) {
  if (!c) return NH_ERR_ARG;
  NH_CUDA(c, cudaSetDevice(c->device));
  NH_CUDA(c, cudaStreamSynchronize(c->stream));
  NH_CUDA(c, cudaGetLastError());
  int err = 0;
  NH_CUDA(c, cudaMemcpy(&err, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    NH_CUDA(c, cudaMemset(c->dev_err, 0, sizeof(int)));
    return nh_fail(c, NH_ERR_TIMEOUT, "a kernel's bounded wait for its shared-memory copy expired");
  }
  return NH_OK;
}

extern "C" int64_t nh_launch_count(nh_ctx c) { return c ? c->launches : -1; }

// ---------------------------------------------------------------------------
// spaces
// ---------------------------------------------------------------------------
static nh_status space_upload(nh_ctx ctx, nh_space s, const std::vector<int>& emap, const std::vector<double>& mult);

// FNV-1a over raw bytes: spaces on the same mesh (the p-multigrid levels) get
// the same value, so the per-call mesh checks of the transfers cost O(1)
static uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

extern "C" nh_status nh_space_box(nh_ctx ctx, int nx, int ny, int nz, const double* vxyz, int p, int q,
                                  nh_space* out, int64_t* n_nodes, int64_t* n_dof) {
  if (!ctx || !out) return NH_ERR_ARG;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return nh_fail(ctx, NH_ERR_ARG, "nh_space_box: element counts must be >= 1");
  if (p < 1 || p > 4 || q < p + 1 || q > NH_MAXQ)
    return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_space_box: need 1 <= p <= 4 and p+1 <= q <= 6");
  const int P = p + 1;
  const int64_t Nx = (int64_t)p * nx + 1, Ny = (int64_t)p * ny + 1, Nz = (int64_t)p * nz + 1;
  const int64_t ne = (int64_t)nx * ny * nz, nn = Nx * Ny * Nz;
  if (nn >= ((int64_t)1 << 29) || ne > INT32_MAX / 8)
    return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_space_box: mesh too large (node ids must fit 29 bits)");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  nh_space s = new nh_space_s();
  s->ctx = ctx;
  s->nx = nx; s->ny = ny; s->nz = nz; s->p = p; s->q = q; s->P = P; s->Q = q;
  s->ne = ne; s->n_nodes = nn; s->n_dof = 3 * nn;
  s->Nx = (int)Nx; s->Ny = (int)Ny; s->Nz = (int)Nz;
  nh_tabulate(p, q, &s->tab);
  if (vxyz) s->verts_host.assign(vxyz, vxyz + 3 * (size_t)(nx + 1) * (ny + 1) * (nz + 1));
  const int dims[3] = {nx, ny, nz};
  s->mesh_hash = fnv1a(s->verts_host.data(), sizeof(double) * s->verts_host.size(), fnv1a(dims, sizeof(dims)));

  // element restriction and node coordinates (trilinear image of the GLL lattice)
  const int P3 = P * P * P;
  std::vector<int> emap((size_t)ne * P3);
  s->coords_host.assign((size_t)nn * 3, 0.0);
  std::vector<double> mult((size_t)nn, 0.0);
  double xn[NH_MAXP];
  nh_lobatto(P, xn);
  double sh[NH_MAXP][2];  // 1-D trilinear factors at the GLL nodes
  for (int i = 0; i < P; i++) {
    sh[i][0] = 0.5 * (1.0 - xn[i]);
    sh[i][1] = 0.5 * (1.0 + xn[i]);
  }
  const int64_t VX = nx + 1, VY = ny + 1;
  for (int64_t ez = 0; ez < nz; ez++)
    for (int64_t ey = 0; ey < ny; ey++)
      for (int64_t ex = 0; ex < nx; ex++) {
        const int64_t e = ex + nx * (ey + ny * ez);
        double V[8][3];
        for (int v = 0; v < 8; v++) {
          const int64_t vi = ex + (v & 1), vj = ey + ((v >> 1) & 1), vk = ez + ((v >> 2) & 1);
          const int64_t vid = vi + VX * (vj + VY * vk);
          if (vxyz) {
            for (int d = 0; d < 3; d++) V[v][d] = vxyz[3 * vid + d];
          } else {
            V[v][0] = (double)vi / nx;
            V[v][1] = (double)vj / ny;
            V[v][2] = (double)vk / nz;
          }
        }
        for (int k = 0; k < P; k++)
          for (int j = 0; j < P; j++)
            for (int i = 0; i < P; i++) {
              const int64_t gi = p * ex + i, gj = p * ey + j, gk = p * ez + k;
              const int64_t nid = gi + Nx * (gj + Ny * gk);
              emap[(size_t)e * P3 + (k * P + j) * P + i] = (int)nid;
              mult[nid] += 1.0;
              double X[3] = {0, 0, 0};
              for (int v = 0; v < 8; v++) {
                const double w = sh[i][v & 1] * sh[j][(v >> 1) & 1] * sh[k][(v >> 2) & 1];
                for (int d = 0; d < 3; d++) X[d] += w * V[v][d];
              }
              for (int d = 0; d < 3; d++) s->coords_host[3 * nid + d] = X[d];
            }
      }
  nh_status st = space_upload(ctx, s, emap, mult);
  if (st != NH_OK) return st;
  *out = s;
  if (n_nodes) *n_nodes = nn;
  if (n_dof) *n_dof = 3 * nn;
  return NH_OK;
}

// device copies of a space's element restriction, coordinates and inverse
// multiplicities; frees the space on failure
static nh_status space_upload(nh_ctx ctx, nh_space s, const std::vector<int>& emap, const std::vector<double>& mult) {
  const int64_t nn = s->n_nodes;
  std::vector<double> im(nn);
  std::vector<float> imf(nn);
  for (int64_t n = 0; n < nn; n++) {
    im[n] = 1.0 / mult[n];
    imf[n] = (float)im[n];
  }
  cudaError_t e1 = cudaMalloc(&s->emap, sizeof(int) * emap.size());
  cudaError_t e2 = cudaMalloc(&s->coords, sizeof(double) * 3 * nn);
  cudaError_t e3 = cudaMalloc(&s->bc, nn);
  cudaError_t e4 = cudaMalloc(&s->inv_mult, sizeof(double) * nn);
  cudaError_t e5 = cudaMalloc(&s->inv_mult_f, sizeof(float) * nn);
  cudaError_t e6 = cudaMalloc(&s->emapb, sizeof(unsigned) * emap.size());
  if (e1 || e2 || e3 || e4 || e5 || e6) {
    cudaGetLastError();
    nh_space_destroy(s);
    return nh_fail(ctx, NH_ERR_OOM, "space: device allocation failed");
  }
  cudaError_t e = cudaMemcpy(s->emap, emap.data(), sizeof(int) * emap.size(), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(s->coords, s->coords_host.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemset(s->bc, 0, nn);
  if (!e) e = cudaMemcpy(s->inv_mult, im.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(s->inv_mult_f, imf.data(), sizeof(float) * nn, cudaMemcpyHostToDevice);
  if (!e) e = cudaDeviceSynchronize();
  if (!e) e = nh_launch_pack_emap(ctx->stream, (int64_t)emap.size(), s->emap, s->bc, s->emapb);
  if (!e) e = cudaDeviceSynchronize();
  if (e) {
    nh_space_destroy(s);
    return nh_cuda_check(ctx, e, "space upload");
  }
  return NH_OK;
}

extern "C" nh_status nh_space_hex(nh_ctx ctx, int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int p,
                                  int q, nh_space* out, int64_t* n_nodes, int64_t* n_dof) {
  if (!ctx || !out || !xyz || !hex8) return NH_ERR_ARG;
  *out = nullptr;
  if (nv < 8 || ne < 1 || ne > INT32_MAX / 8) return nh_fail(ctx, NH_ERR_ARG, "nh_space_hex: need nv >= 8 and ne >= 1");
  if (p < 1 || p > 4 || q < p + 1 || q > NH_MAXQ)
    return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_space_hex: need 1 <= p <= 4 and p+1 <= q <= 6");
  std::vector<int> emap;
  std::vector<double> coords;
  int64_t nn = 0;
  const std::string msg = nh_hex_numbering(nv, xyz, ne, hex8, p, emap, coords, nn);
  if (!msg.empty())
    return nh_fail(ctx, msg.find("too large") != std::string::npos ? NH_ERR_UNSUPPORTED : NH_ERR_ARG,
                   "nh_space_hex: " + msg);
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  nh_space s = new nh_space_s();
  s->ctx = ctx;
  s->hex = true;
  s->p = p; s->q = q; s->P = p + 1; s->Q = q;
  s->ne = ne; s->n_nodes = nn; s->n_dof = 3 * nn;
  nh_tabulate(p, q, &s->tab);
  s->verts_host.assign(xyz, xyz + 3 * (size_t)nv);
  s->hex8_host.assign(hex8, hex8 + 8 * (size_t)ne);
  s->mesh_hash = fnv1a(s->verts_host.data(), sizeof(double) * s->verts_host.size(),
                       fnv1a(s->hex8_host.data(), sizeof(int64_t) * s->hex8_host.size()));
  s->coords_host = std::move(coords);
  std::vector<double> mult((size_t)nn, 0.0);
  for (int n : emap) mult[n] += 1.0;
  s->emap_host = emap;
  // first-touch numbering: the nodes of elements [0, e] are a prefix of the ids, so
  // the host-buffer apply can upload du and download y in element chunks
  const int P3 = s->P * s->P * s->P;
  s->hex_need.resize(ne);
  s->hex_fin.assign(ne + 1, nn);
  int64_t hi = 0;
  for (int64_t e = 0; e < ne; e++) {
    int64_t lo = nn;
    for (int l = 0; l < P3; l++) {
      hi = std::max<int64_t>(hi, emap[(size_t)e * P3 + l] + 1);
      lo = std::min<int64_t>(lo, emap[(size_t)e * P3 + l]);
    }
    s->hex_need[e] = hi;
    s->hex_fin[e] = lo;
  }
  for (int64_t e = ne - 1; e >= 0; e--) s->hex_fin[e] = std::min(s->hex_fin[e], s->hex_fin[e + 1]);
  nh_status st = space_upload(ctx, s, emap, mult);
  if (st != NH_OK) return st;
  *out = s;
  if (n_nodes) *n_nodes = nn;
  if (n_dof) *n_dof = 3 * nn;
  return NH_OK;
}

extern "C" nh_status nh_hex_mesh_numbering(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int p,
                                           int64_t* n_nodes, int* emap, double* coords, char* err, int64_t err_len) {
  if (!xyz || !hex8 || !n_nodes || nv < 8 || ne < 1 || ne > INT32_MAX / 8) return NH_ERR_ARG;
  if (p < 1 || p > 4) return NH_ERR_UNSUPPORTED;
  std::vector<int> em;
  std::vector<double> X;
  int64_t nn = 0;
  const std::string msg = nh_hex_numbering(nv, xyz, ne, hex8, p, em, X, nn);
  if (!msg.empty()) {
    if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", msg.c_str());
    return msg.find("too large") != std::string::npos ? NH_ERR_UNSUPPORTED : NH_ERR_ARG;
  }
  *n_nodes = nn;
  if (emap) memcpy(emap, em.data(), sizeof(int) * em.size());
  if (coords) memcpy(coords, X.data(), sizeof(double) * X.size());
  return NH_OK;
}

extern "C" nh_status nh_hex_morton_order(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8,
                                         int64_t* perm) {
  if (!xyz || !hex8 || !perm || nv < 1 || ne < 1) return NH_ERR_ARG;
  for (int64_t i = 0; i < 8 * ne; i++)
    if (hex8[i] < 0 || hex8[i] >= nv) return NH_ERR_ARG;
  nh_hex_morton(nv, xyz, ne, hex8, perm);
  return NH_OK;
}

extern "C" nh_status nh_q1_block_pattern(int64_t ne, int64_t n_nodes, const int* emap, int64_t* nnzb, int64_t* rowptr,
                                         int* col) {
  if (!emap || !nnzb || ne < 0 || n_nodes < 1) return NH_ERR_ARG;
  for (int64_t i = 0; i < 8 * ne; i++)
    if (emap[i] < 0 || emap[i] >= n_nodes) return NH_ERR_ARG;
  std::vector<int64_t> rp, js, pm;
  std::vector<int> cl;
  ks_coo_symbolic(ne, n_nodes, emap, rp, cl, js, pm);
  *nnzb = (int64_t)cl.size();
  if (rowptr) memcpy(rowptr, rp.data(), sizeof(int64_t) * rp.size());
  if (col) memcpy(col, cl.data(), sizeof(int) * cl.size());
  return NH_OK;
}

bool nh_same_mesh(nh_space a, nh_space b) {
  if (a->hex != b->hex || a->ne != b->ne || a->mesh_hash != b->mesh_hash) return false;
  return a->hex || (a->nx == b->nx && a->ny == b->ny && a->nz == b->nz);
}

extern "C" nh_status nh_space_coords(nh_space s, double* xyz) {
  if (!s || !xyz) return NH_ERR_ARG;
  memcpy(xyz, s->coords_host.data(), sizeof(double) * 3 * s->n_nodes);
  return NH_OK;
}

extern "C" nh_status nh_space_set_dirichlet(nh_space s, const uint8_t* mask) {
  if (!s || !mask) return NH_ERR_ARG;
  std::vector<uint8_t> bits((size_t)s->n_nodes, 0);
  int64_t nc = 0;
  for (int64_t n = 0; n < s->n_nodes; n++)
    for (int c = 0; c < 3; c++)
      if (mask[3 * n + c]) {
        bits[n] |= (uint8_t)(1u << c);
        nc++;
      }
  s->n_constrained = nc;
  NH_CUDA(s->ctx, cudaSetDevice(s->ctx->device));
  NH_CUDA(s->ctx, cudaMemcpyAsync(s->bc, bits.data(), s->n_nodes, cudaMemcpyHostToDevice, s->ctx->stream));
  NH_CUDA(s->ctx, nh_launch_pack_emap(s->ctx->stream, s->ne * (int64_t)s->P * s->P * s->P, s->emap, s->bc, s->emapb));
  NH_CUDA(s->ctx, cudaStreamSynchronize(s->ctx->stream));
  return NH_OK;
}

extern "C" nh_status nh_space_destroy(nh_space s) {
  if (!s) return NH_ERR_ARG;
  cudaFree(s->emap);
  cudaFree(s->emapb);
  cudaFree(s->coords);
  cudaFree(s->bc);
  cudaFree(s->inv_mult);
  cudaFree(s->inv_mult_f);
  delete s;
  return NH_OK;
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------
static int scalars_for(int layout) { return nh_layout_scalars(layout); }

extern "C" nh_status nh_op_create(nh_space fine, double nu, const double* Epe, double E, int layout, nh_op* out) {
  if (!fine || !out) return NH_ERR_ARG;
  *out = nullptr;
  nh_ctx ctx = fine->ctx;
  if (layout != NH_LAYOUT_CURRENT && layout != NH_LAYOUT_INITIAL && layout != NH_LAYOUT_TAPE)
    return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_op_create: unknown layout");
  if (!(nu > -1.0 && nu < 0.5)) return nh_fail(ctx, NH_ERR_ARG, "nh_op_create: need -1 < nu < 0.5");
  std::vector<double> lam(fine->ne), mu(fine->ne);
  for (int64_t e = 0; e < fine->ne; e++) {
    const double Ee = Epe ? Epe[e] : E;
    if (!(Ee > 0.0)) return nh_fail(ctx, NH_ERR_ARG, "nh_op_create: Young's modulus must be > 0");
    lam[e] = Ee * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mu[e] = Ee / (2.0 * (1.0 + nu));
  }
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  nh_op op = new nh_op_s();
  op->space = fine;
  op->layout = layout;
  op->S = scalars_for(layout);
  op->nu = nu;
  const int64_t nq = fine->ne * (int64_t)fine->Q * fine->Q * fine->Q;
  if (cudaMalloc(&op->lam, sizeof(double) * fine->ne) || cudaMalloc(&op->mu, sizeof(double) * fine->ne) ||
      cudaMalloc(&op->qd, sizeof(double) * nq * op->S)) {
    cudaGetLastError();
    nh_op_destroy(op);
    return nh_fail(ctx, NH_ERR_OOM, "nh_op_create: device allocation failed");
  }
  NH_CUDA(ctx, cudaMemcpy(op->lam, lam.data(), sizeof(double) * fine->ne, cudaMemcpyHostToDevice));
  NH_CUDA(ctx, cudaMemcpy(op->mu, mu.data(), sizeof(double) * fine->ne, cudaMemcpyHostToDevice));
  *out = op;
  return NH_OK;
}

extern "C" nh_status nh_op_level(nh_op fine, nh_space coarse, nh_op* out) {
  if (!fine || !coarse || !out) return NH_ERR_ARG;
  *out = nullptr;
  nh_op root = fine->parent ? fine->parent : fine;
  nh_space fs = root->space;
  nh_ctx ctx = fs->ctx;
  if (!nh_same_mesh(coarse, fs) || coarse->Q != fs->Q || coarse->p > fs->p)
    return nh_fail(ctx, NH_ERR_ARG, "nh_op_level: coarse space must share the mesh and q, with p_c <= p_f");
  nh_op op = new nh_op_s();
  op->space = coarse;
  op->parent = root;
  op->layout = root->layout;
  op->S = root->S;
  op->nu = root->nu;
  *out = op;
  return NH_OK;
}

extern "C" nh_status nh_op_rediscretize(nh_op fine, nh_space coarse, nh_op* out) {
  if (!fine || !coarse || !out) return NH_ERR_ARG;
  *out = nullptr;
  nh_ctx ctx = fine->space->ctx;
  if (fine->parent) return nh_fail(ctx, NH_ERR_ARG, "nh_op_rediscretize: needs the fine operator");
  nh_space fs = fine->space;
  if (!nh_same_mesh(coarse, fs) || coarse->p > fs->p)
    return nh_fail(ctx, NH_ERR_ARG, "nh_op_rediscretize: coarse space must share the mesh, with p_c <= p_f");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  nh_op op = new nh_op_s();
  op->space = coarse;
  op->layout = fine->layout;
  op->S = fine->S;
  op->nu = fine->nu;
  const int64_t ne = coarse->ne, nq = ne * (int64_t)coarse->Q * coarse->Q * coarse->Q;
  if (cudaMalloc(&op->lam, sizeof(double) * ne) != cudaSuccess || cudaMalloc(&op->mu, sizeof(double) * ne) != cudaSuccess ||
      cudaMalloc(&op->qd, sizeof(double) * nq * op->S) != cudaSuccess) {
    cudaGetLastError();
    nh_op_destroy(op);
    return nh_fail(ctx, NH_ERR_OOM, "nh_op_rediscretize: device allocation failed");
  }
  NH_CUDA(ctx, cudaMemcpyAsync(op->lam, fine->lam, sizeof(double) * ne, cudaMemcpyDeviceToDevice, ctx->stream));
  NH_CUDA(ctx, cudaMemcpyAsync(op->mu, fine->mu, sizeof(double) * ne, cudaMemcpyDeviceToDevice, ctx->stream));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *out = op;
  return NH_OK;
}

extern "C" nh_status nh_qdata_setup_rediscretized(nh_op op, nh_op fine, const double* u_fine, double* min_J) {
  if (!op || !fine || !u_fine) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  nh_space fs = fine->space, cs = op->space;
  if (op->parent || fine->parent) return nh_fail(ctx, NH_ERR_ARG, "nh_qdata_setup_rediscretized: needs two root operators");
  if (!nh_same_mesh(cs, fs) || cs->p > fs->p || op->layout != fine->layout)
    return nh_fail(ctx, NH_ERR_ARG, "nh_qdata_setup_rediscretized: operators must share the mesh and layout, p_c <= p_f");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  const int64_t nq = cs->ne * (int64_t)cs->Q * cs->Q * cs->Q;
  NH_CUDA(ctx, cudaMemsetAsync(ctx->minj, 0xff, sizeof(unsigned long long), ctx->stream));
  NH_CUDA(ctx, nh_launch_setup_pts(fs->P, cs->Q, op->layout, ctx->stream, fs->ne, fs->emap, fs->coords, u_fine, op->lam,
                                   op->mu, op->qd, nq, ctx->minj));
  ctx->launches++;
  unsigned long long bits = 0;
  NH_CUDA(ctx, cudaMemcpyAsync(ctx->red_host, ctx->minj, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(&bits, ctx->red_host, sizeof(bits));
  bits = (bits >> 63) ? (bits & 0x7fffffffffffffffull) : ~bits;
  double mj;
  memcpy(&mj, &bits, sizeof(mj));
  if (min_J) *min_J = mj;
  op->qd_f_valid = false;
  op->qd_ff_valid = false;
  if (!(mj > 0.0) || !isfinite(mj)) {
    op->have_qd = false;
    return nh_fail(ctx, NH_ERR_INVERTED, "nh_qdata_setup_rediscretized: inverted element");
  }
  op->have_qd = true;
  return NH_OK;
}

extern "C" nh_status nh_op_destroy(nh_op op) {
  if (!op) return NH_ERR_ARG;
  if (!op->parent) {
    cudaFree(op->lam);
    cudaFree(op->mu);
    cudaFree(op->qd);
    cudaFree(op->qd_f);
    cudaFree(op->qd_ff);
    cudaFree(op->geom);
  }
  cudaFree(op->u_state);
  cudaFree(op->hbuf_in);
  cudaFree(op->hbuf_out);
  delete op;
  return NH_OK;
}

extern "C" nh_status nh_op_info(nh_op op, nh_prec prec, int* S, int64_t* bytes) {
  if (!op) return NH_ERR_ARG;
  nh_op root = op->parent ? op->parent : op;
  const int64_t nq = root->space->ne * (int64_t)root->space->Q * root->space->Q * root->space->Q;
  if (S) *S = root->S;
  if (bytes) *bytes = nq * root->S * (prec == NH_F64 ? 8 : 4);  // algorithmic size (the FP32 copy is padded per batch)
  return NH_OK;
}

static OpArgs base_args(nh_op op) {
  nh_op root = op->parent ? op->parent : op;
  OpArgs a;
  memset(&a, 0, sizeof(a));
  a.ne = op->space->ne;
  a.nx = op->space->nx;
  a.ny = op->space->ny;
  a.nz = op->space->nz;
  a.colour = -1;
  a.emap = op->space->emap;
  a.emapb = op->space->emapb;
  a.bc = op->space->bc;
  a.qstride = root->space->ne * (int64_t)root->space->Q * root->space->Q * root->space->Q;
  a.layout = root->layout;
  a.tab = &op->space->tab;
  a.coords = op->space->coords;
  a.lam = root->lam;
  a.mu = root->mu;
  a.err = op->space->ctx->dev_err;
  return a;
}

#ifndef NH_GEOM_CACHE
#define NH_GEOM_CACHE 1
#endif
// The setup kernel's geometry factors (grad_X xi, det(dX/dxi): 10 doubles per
// point) are kept on the fine operator after its first setup or residual launch;
// later launches read them instead of recomputing them from the coordinates.
// Without memory for them every launch recomputes.
static void attach_geom(nh_op op, OpArgs& a) {
  if (!NH_GEOM_CACHE) return;
  if (!op->geom && cudaMalloc(&op->geom, sizeof(double) * 10 * a.qstride) != cudaSuccess) {
    cudaGetLastError();
    op->geom = nullptr;
  }
  a.geom = op->geom;
  a.geom_mode = op->geom_valid ? 2 : 1;
}

extern "C" nh_status nh_qdata_setup(nh_op op, const double* u, double* min_J) {
  if (!op || !u) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  if (op->parent) return nh_fail(ctx, NH_ERR_STATE, "nh_qdata_setup: coarse operators share the fine data");
  if (!aligned(u, 16)) return nh_fail(ctx, NH_ERR_ARG, "nh_qdata_setup: u must be 16-byte aligned");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  OpArgs a = base_args(op);
  a.in = u;
  a.qd_out = op->qd;
  a.store = 1;
  a.resid = 0;
  a.minj = ctx->minj;
  attach_geom(op, a);
  NH_CUDA(ctx, cudaMemsetAsync(ctx->minj, 0xff, sizeof(unsigned long long), ctx->stream));
  NH_CUDA(ctx, nh_launch_setup(op->space->P, op->space->Q, a, ctx->stream));
  ctx->launches++;
  if (a.geom) op->geom_valid = true;
  unsigned long long bits = 0;
  NH_CUDA(ctx, cudaMemcpyAsync(ctx->red_host, ctx->minj, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(&bits, ctx->red_host, sizeof(bits));
  bits = (bits >> 63) ? (bits & 0x7fffffffffffffffull) : ~bits;
  double mj;
  memcpy(&mj, &bits, sizeof(mj));
  if (min_J) *min_J = mj;
  op->qd_f_valid = false;
  op->qd_ff_valid = false;
  if (!(mj > 0.0) || !isfinite(mj)) {
    op->have_qd = false;
    char buf[128];
    snprintf(buf, sizeof(buf), "nh_qdata_setup: inverted element, min det F = %g", mj);
    return nh_fail(ctx, NH_ERR_INVERTED, buf);
  }
  // the state, for rediscretised coarse levels set up later from it
  if (!op->u_state && cudaMalloc(&op->u_state, sizeof(double) * op->space->n_dof) != cudaSuccess) {
    cudaGetLastError();
    op->u_state = nullptr;
    return nh_fail(ctx, NH_ERR_OOM, "nh_qdata_setup: device allocation failed");
  }
  NH_CUDA(ctx, cudaMemcpyAsync(op->u_state, u, sizeof(double) * op->space->n_dof, cudaMemcpyDeviceToDevice,
                               ctx->stream));
  op->have_qd = true;
  return NH_OK;
}

extern "C" nh_status nh_residual(nh_op op, const double* u, const double* g_bc, double* r) {
  if (!op || !u || !r) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  if (op->parent) return nh_fail(ctx, NH_ERR_STATE, "nh_residual: only on the fine operator");
  if ((const void*)u == (const void*)r) return nh_fail(ctx, NH_ERR_ARG, "nh_residual: u and r must not alias");
  if (!aligned(u, 16) || !aligned(r, 16)) return nh_fail(ctx, NH_ERR_ARG, "nh_residual: misaligned vector");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  OpArgs a = base_args(op);
  a.in = u;
  a.out = r;
  a.gbc = g_bc;
  a.store = 0;
  a.resid = 1;
  attach_geom(op, a);
  NH_CUDA(ctx, cudaMemsetAsync(r, 0, sizeof(double) * op->space->n_dof, ctx->stream));
  NH_CUDA(ctx, nh_launch_setup(op->space->P, op->space->Q, a, ctx->stream));
  ctx->launches++;
  if (a.geom) op->geom_valid = true;
  return NH_OK;
}

static nh_status ensure_f32(nh_op root) {
  nh_ctx ctx = root->space->ctx;
  if (root->qd_f_valid) return NH_OK;
  const int Q = root->space->Q;
  const int64_t nb = (root->space->ne + nh_epb(Q) - 1) / nh_epb(Q);
  if (!root->qd_f) NH_CUDA(ctx, cudaMalloc(&root->qd_f, sizeof(float) * nb * nh_f32_batch_floats(Q, root->S)));
  NH_CUDA(ctx, nh_launch_f32_blocked(Q, root->S, root->space->ne, root->qd, root->qd_f, ctx->stream));
  ctx->launches++;
  root->qd_f_valid = true;
  return NH_OK;
}

static nh_status ensure_ff(nh_op root) {
  nh_ctx ctx = root->space->ctx;
  if (root->qd_ff_valid) return NH_OK;
  const int64_t n = root->S * root->space->ne * (int64_t)root->space->Q * root->space->Q * root->space->Q;
  if (!root->qd_ff) NH_CUDA(ctx, cudaMalloc(&root->qd_ff, 2 * sizeof(float) * n));
  NH_CUDA(ctx, nh_launch_f64_to_ff(n, root->qd, root->qd_ff, ctx->stream));
  ctx->launches++;
  root->qd_ff_valid = true;
  return NH_OK;
}

extern "C" nh_status nh_jacobian_apply(nh_op op, nh_prec prec, const void* du, void* y) {
  if (!op || !du || !y) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  nh_op root = op->parent ? op->parent : op;
  if (prec != NH_F64 && prec != NH_F32 && prec != NH_F64X)
    return nh_fail(ctx, NH_ERR_ARG, "nh_jacobian_apply: bad precision");
  if (du == (const void*)y) return nh_fail(ctx, NH_ERR_ARG, "nh_jacobian_apply: du and y must not alias");
  if (!aligned(du, 16) || !aligned(y, 16)) return nh_fail(ctx, NH_ERR_ARG, "nh_jacobian_apply: misaligned vector");
  if (!root->have_qd) return nh_fail(ctx, NH_ERR_STATE, "nh_jacobian_apply: call nh_qdata_setup first");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  if (prec == NH_F32) {
    nh_status st = ensure_f32(root);
    if (st != NH_OK) return st;
  } else if (prec == NH_F64X) {
    nh_status st = ensure_ff(root);
    if (st != NH_OK) return st;
  }
  OpArgs a = base_args(op);
  a.in = du;
  a.out = y;
  a.prec = prec;
  a.qd = prec == NH_F64 ? (const void*)root->qd : prec == NH_F32 ? (const void*)root->qd_f : (const void*)root->qd_ff;
  const size_t w = prec == NH_F32 ? 4 : 8;
  NH_CUDA(ctx, cudaMemsetAsync(y, 0, w * op->space->n_dof, ctx->stream));
  cudaEvent_t* ev = nullptr;
  if (ctx->prof_on && ctx->ev_used + 2 <= kMaxProfEvents) {
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
      cudaEvent_t e;
      NH_CUDA(ctx, cudaEventCreate(&e));
      ctx->ev_pool.push_back(e);
    }
    ev = &ctx->ev_pool[ctx->ev_used];
    ctx->ev_used += 2;
    NH_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
  }
  if (op->scatter == 1) {  // eight launches, one per parity class, no atomics
    for (int c = 0; c < 8; c++) {
      a.colour = c;
      NH_CUDA(ctx, nh_launch_apply(op->space->P, op->space->Q, prec, a, ctx->stream));
      ctx->launches++;
    }
  } else {
    NH_CUDA(ctx, nh_launch_apply(op->space->P, op->space->Q, prec, a, ctx->stream));
    ctx->launches++;
  }
  if (ev) NH_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
  return NH_OK;
}

extern "C" nh_status nh_op_set_scatter(nh_op op, int mode) {
  if (!op || (mode != 0 && mode != 1)) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  if (mode == 1) {
    const nh_space s = op->space;
    if (s->hex || s->nx <= 0)
      return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_op_set_scatter: the eight-colour scatter needs a box mesh");
    if (s->nx % nh_epb(s->Q) != 0)
      return nh_fail(ctx, NH_ERR_UNSUPPORTED,
                     "nh_op_set_scatter: the eight-colour scatter needs an x-element count that is a multiple of "
                     "the FP32 kernel's elements per block");
  }
  op->scatter = mode;
  return NH_OK;
}

extern "C" nh_status nh_profile_enable(nh_ctx ctx, int on) {
  if (!ctx) return NH_ERR_ARG;
  ctx->prof_on = on != 0;
  return NH_OK;
}

extern "C" nh_status nh_profile_read(nh_ctx ctx, double* total_ms, int64_t* launches) {
  if (!ctx) return NH_ERR_ARG;
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float ms = 0.f;
    NH_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = (int64_t)(ctx->ev_used / 2);
  ctx->ev_used = 0;
  return NH_OK;
}

nh_status nh_jacobian_apply_lift(nh_op op, const double* x, double* y) {
  nh_ctx ctx = op->space->ctx;
  nh_op root = op->parent ? op->parent : op;
  if (!root->have_qd) return nh_fail(ctx, NH_ERR_STATE, "lift apply: no quadrature data");
  OpArgs a = base_args(op);
  a.in = x;
  a.out = y;
  a.prec = NH_F64;
  a.lift = 1;
  a.qd = root->qd;
  NH_CUDA(ctx, cudaMemsetAsync(y, 0, 8 * op->space->n_dof, ctx->stream));
  NH_CUDA(ctx, nh_launch_apply(op->space->P, op->space->Q, NH_F64, a, ctx->stream));
  ctx->launches++;
  return NH_OK;
}

// Launch the apply for elements [e0, e1) of op's space (arguments offset into
// the element maps and quadrature data; y must have been zeroed).
static nh_status launch_apply_range(nh_op op, nh_prec prec, const void* du, void* y, int64_t e0, int64_t e1,
                                    cudaStream_t s) {
  nh_ctx ctx = op->space->ctx;
  nh_op root = op->parent ? op->parent : op;
  nh_space sp = op->space;
  const int64_t P3 = (int64_t)sp->P * sp->P * sp->P, Q3 = (int64_t)sp->Q * sp->Q * sp->Q;
  OpArgs a = base_args(op);
  a.ne = e1 - e0;
  a.emap = sp->emap + e0 * P3;
  a.emapb = sp->emapb + e0 * P3;
  a.in = du;
  a.out = y;
  a.prec = prec;
  if (prec == NH_F64) {
    a.qd = root->qd + e0 * Q3;
  } else if (prec == NH_F64X) {
    a.qd = root->qd_ff + 2 * e0 * Q3;
  } else {
    const int epb = nh_epb(sp->Q);
    a.qd = root->qd_f + (e0 / epb) * nh_f32_batch_floats(sp->Q, root->S);
  }
  NH_CUDA(ctx, nh_launch_apply(sp->P, sp->Q, prec, a, s));
  ctx->launches++;
  return NH_OK;
}

// Host vectors in and out.  On the box mesh the elements of z-layers [z0, z1)
// need du on node layers [z0 p, z1 p] only, a contiguous range of the L-vector,
// and leave y final on the layers below z1 p: the apply runs in chunks of
// z-layers with the upload of the next chunk and the download of finished node
// layers on two copy streams, overlapping the transfers with the kernels.
extern "C" nh_status nh_jacobian_apply_host(nh_op op, nh_prec prec, const void* du_h, void* y_h) {
  if (!op || !du_h || !y_h) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  nh_op root = op->parent ? op->parent : op;
  nh_space sp = op->space;
  if (prec != NH_F64 && prec != NH_F32 && prec != NH_F64X)
    return nh_fail(ctx, NH_ERR_ARG, "nh_jacobian_apply_host: bad precision");
  if (!root->have_qd) return nh_fail(ctx, NH_ERR_STATE, "nh_jacobian_apply_host: call nh_qdata_setup first");
  const size_t w = prec == NH_F32 ? 4 : 8;
  const size_t bytes = w * (size_t)sp->n_dof;
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  if (op->hbuf_bytes < bytes) {
    NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(op->hbuf_in);
    cudaFree(op->hbuf_out);
    op->hbuf_in = op->hbuf_out = nullptr;
    op->hbuf_bytes = 0;
    NH_CUDA(ctx, cudaMalloc(&op->hbuf_in, bytes));
    NH_CUDA(ctx, cudaMalloc(&op->hbuf_out, bytes));
    op->hbuf_bytes = bytes;
  }
  if (prec == NH_F32) {
    nh_status st = ensure_f32(root);
    if (st != NH_OK) return st;
  } else if (prec == NH_F64X) {
    nh_status st = ensure_ff(root);
    if (st != NH_OK) return st;
  }
  if (!ctx->s_in) {
    NH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking));
    NH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
    NH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_k2, cudaStreamNonBlocking));
  }
  if (sp->hex) {
    // unstructured mesh in first-touch numbering: elements [e0, e1) read du on the
    // node prefix [0, hex_need[e1 - 1]) and leave y final below hex_fin[e1]; chunks
    // of elements (FP32: whole kernel batches) with the same three-stream overlap
    const int64_t ne = sp->ne, al = prec == NH_F32 ? nh_epb(sp->Q) : 1;
    const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(8, ne / al));
    while (ctx->ev_chunk.size() < 2 * (size_t)nch) {
      cudaEvent_t ev;
      NH_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      ctx->ev_chunk.push_back(ev);
    }
    const char* hin = static_cast<const char*>(du_h);
    char* hout = static_cast<char*>(y_h);
    char* din = static_cast<char*>(op->hbuf_in);
    char* dout = static_cast<char*>(op->hbuf_out);
    NH_CUDA(ctx, cudaMemsetAsync(dout, 0, bytes, ctx->stream));
    NH_CUDA(ctx, cudaEventRecord(ctx->ev_chunk[0], ctx->stream));
    NH_CUDA(ctx, cudaStreamWaitEvent(ctx->s_in, ctx->ev_chunk[0], 0));
    NH_CUDA(ctx, cudaStreamWaitEvent(ctx->s_k2, ctx->ev_chunk[0], 0));
    int64_t up = 0, down = 0;  // DoF uploaded / downloaded so far
    int lastk[2] = {-1, -1};   // event of the last kernel per compute stream (as on the box)
    for (int c = 0; c < nch; c++) {
      const int64_t e0 = ne * c / nch / al * al;
      const int64_t e1 = c + 1 == nch ? ne : ne * (c + 1) / nch / al * al;
      if (e1 <= e0) continue;
      const int64_t need = 3 * sp->hex_need[e1 - 1];
      if (need > up) {
        NH_CUDA(ctx, cudaMemcpyAsync(din + w * up, hin + w * up, w * (need - up), cudaMemcpyHostToDevice, ctx->s_in));
        up = need;
      }
      const int ks = prec == NH_F32 ? 0 : c & 1;  // FP32 chunks are transfer-bound: one kernel stream
      cudaStream_t kst = ks ? ctx->s_k2 : ctx->stream;
      NH_CUDA(ctx, cudaEventRecord(ctx->ev_chunk[2 * c], ctx->s_in));
      NH_CUDA(ctx, cudaStreamWaitEvent(kst, ctx->ev_chunk[2 * c], 0));
      nh_status st = launch_apply_range(op, prec, din, dout, e0, e1, kst);
      if (st != NH_OK) return st;
      NH_CUDA(ctx, cudaEventRecord(ctx->ev_chunk[2 * c + 1], kst));
      lastk[ks] = 2 * c + 1;
      const int64_t fin = c + 1 == nch ? sp->n_dof : 3 * sp->hex_fin[e1];
      if (fin > down) {
        for (int k = 0; k < 2; k++)
          if (lastk[k] >= 0) NH_CUDA(ctx, cudaStreamWaitEvent(ctx->s_out, ctx->ev_chunk[lastk[k]], 0));
        NH_CUDA(ctx, cudaMemcpyAsync(hout + w * down, dout + w * down, w * (fin - down), cudaMemcpyDeviceToHost,
                                     ctx->s_out));
        down = fin;
      }
    }
    NH_CUDA(ctx, cudaStreamSynchronize(ctx->s_out));
    NH_CUDA(ctx, cudaStreamSynchronize(ctx->s_k2));
    NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return NH_OK;
  }
  // chunks of z-layers; with FP32 each chunk starts on a kernel batch of EPB elements
  const int64_t nxy = (int64_t)sp->nx * sp->ny, lay = (int64_t)sp->Nx * sp->Ny * 3;  // elements, DoF per layer
  int64_t step = 1;
  if (prec == NH_F32) {
    const int64_t epb = nh_epb(sp->Q);
    int64_t g = epb, r = nxy % epb;
    while (r) {
      const int64_t t2 = g % r;
      g = r;
      r = t2;
    }
    step = epb / g;  // layers per aligned boundary
  }
  const int64_t nsteps = (sp->nz + step - 1) / step;
  const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(8, nsteps));
  while (ctx->ev_chunk.size() < 2 * (size_t)nch) {
    cudaEvent_t e;
    NH_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->ev_chunk.push_back(e);
  }
  const char* hin = static_cast<const char*>(du_h);
  char* hout = static_cast<char*>(y_h);
  char* din = static_cast<char*>(op->hbuf_in);
  char* dout = static_cast<char*>(op->hbuf_out);
  // y = 0 on the compute stream, ordered before every chunk's kernel.  FP64 and
  // float-float chunks' kernels alternate between the compute stream and a second
  // one, so that a chunk's kernel starts while the previous one drains its last
  // blocks (they meet only in atomic adds on their shared node layer); a download
  // waits for the latest kernel on both.  (FP32 keeps one stream: its transfers
  // dominate, and on Z-ordered unstructured meshes the alternation measured slower.)
  NH_CUDA(ctx, cudaMemsetAsync(dout, 0, bytes, ctx->stream));
  NH_CUDA(ctx, cudaEventRecord(ctx->ev_chunk[0], ctx->stream));
  NH_CUDA(ctx, cudaStreamWaitEvent(ctx->s_in, ctx->ev_chunk[0], 0));  // hbuf reuse after earlier work
  NH_CUDA(ctx, cudaStreamWaitEvent(ctx->s_k2, ctx->ev_chunk[0], 0));
  int64_t up = 0, down = 0;                                          // DoF uploaded / downloaded so far
  int lastk[2] = {-1, -1};                                           // event of the last kernel per stream
  for (int c = 0; c < nch; c++) {
    const int64_t z0 = std::min<int64_t>(sp->nz, nsteps * c / nch * step);
    const int64_t z1 = c + 1 == nch ? sp->nz : std::min<int64_t>(sp->nz, nsteps * (c + 1) / nch * step);
    if (z1 <= z0) continue;
    const int64_t need = std::min<int64_t>(sp->n_dof, (z1 * sp->p + 1) * lay);
    if (need > up) {
      NH_CUDA(ctx, cudaMemcpyAsync(din + w * up, hin + w * up, w * (need - up), cudaMemcpyHostToDevice, ctx->s_in));
      up = need;
    }
    const int ks = prec == NH_F32 ? 0 : c & 1;  // FP32 chunks are transfer-bound: one kernel stream
    cudaStream_t kst = ks ? ctx->s_k2 : ctx->stream;
    NH_CUDA(ctx, cudaEventRecord(ctx->ev_chunk[2 * c], ctx->s_in));
    NH_CUDA(ctx, cudaStreamWaitEvent(kst, ctx->ev_chunk[2 * c], 0));
    nh_status st = launch_apply_range(op, prec, din, dout, z0 * nxy, z1 * nxy, kst);
    if (st != NH_OK) return st;
    NH_CUDA(ctx, cudaEventRecord(ctx->ev_chunk[2 * c + 1], kst));
    lastk[ks] = 2 * c + 1;
    const int64_t fin = c + 1 == nch ? sp->n_dof : std::min<int64_t>(sp->n_dof, z1 * sp->p * lay);
    if (fin > down) {
      for (int k = 0; k < 2; k++)
        if (lastk[k] >= 0) NH_CUDA(ctx, cudaStreamWaitEvent(ctx->s_out, ctx->ev_chunk[lastk[k]], 0));
      NH_CUDA(ctx, cudaMemcpyAsync(hout + w * down, dout + w * down, w * (fin - down), cudaMemcpyDeviceToHost,
                                   ctx->s_out));
      down = fin;
    }
  }
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->s_out));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->s_k2));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return NH_OK;
}

extern "C" nh_status nh_jacobian_diagonal(nh_op op, nh_prec prec, void* diag) {
  if (!op || !diag) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  nh_op root = op->parent ? op->parent : op;
  if (prec != NH_F64 && prec != NH_F32) return nh_fail(ctx, NH_ERR_ARG, "nh_jacobian_diagonal: bad precision");
  if (!aligned(diag, 16)) return nh_fail(ctx, NH_ERR_ARG, "nh_jacobian_diagonal: misaligned vector");
  if (!root->have_qd) return nh_fail(ctx, NH_ERR_STATE, "nh_jacobian_diagonal: call nh_qdata_setup first");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  OpArgs a = base_args(op);
  a.out = diag;
  a.prec = prec;
  a.qd = root->qd;
  NH_CUDA(ctx, cudaMemsetAsync(diag, 0, (prec == NH_F64 ? 8 : 4) * op->space->n_dof, ctx->stream));
  NH_CUDA(ctx, nh_launch_diag(op->space->P, op->space->Q, a, ctx->stream));
  ctx->launches++;
  return NH_OK;
}

// Assembled Q1 operator as 3x3 block rows (split-phase COO assembly of the
// element matrices B^T D B at the operator's quadrature points).
extern "C" nh_status nh_op_assemble_q1(nh_op op, int64_t* nnzb, int64_t* rowptr, int* col, double* val) {
  if (!op || !nnzb) return NH_ERR_ARG;
  nh_ctx ctx = op->space->ctx;
  nh_op root = op->parent ? op->parent : op;
  nh_space sp = op->space;
  if (sp->p != 1) return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_op_assemble_q1: needs an operator on a p = 1 space");
  if (!root->have_qd) return nh_fail(ctx, NH_ERR_STATE, "nh_op_assemble_q1: call nh_qdata_setup first");
  if (sp->Q != root->space->Q) return nh_fail(ctx, NH_ERR_ARG, "nh_op_assemble_q1: quadrature rule mismatch");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<int> emap((size_t)sp->ne * 8);
  NH_CUDA(ctx, cudaMemcpy(emap.data(), sp->emap, sizeof(int) * emap.size(), cudaMemcpyDeviceToHost));
  std::vector<int64_t> rp, js, pm;
  std::vector<int> cl;
  ks_coo_symbolic(sp->ne, sp->n_nodes, emap.data(), rp, cl, js, pm);
  *nnzb = (int64_t)cl.size();
  if (!rowptr || !col || !val) return NH_OK;  // size query
  int64_t *d_js = nullptr, *d_pm = nullptr;
  double *d_coo = nullptr, *d_val = nullptr;
  auto release = [&]() {
    cudaFree(d_js);
    cudaFree(d_pm);
    cudaFree(d_coo);
    cudaFree(d_val);
  };
  cudaError_t e = cudaMalloc(&d_js, sizeof(int64_t) * js.size());
  if (!e) e = cudaMalloc(&d_pm, sizeof(int64_t) * pm.size());
  if (!e) e = cudaMalloc(&d_coo, sizeof(double) * 9 * pm.size());
  if (!e) e = cudaMalloc(&d_val, sizeof(double) * 9 * cl.size());
  if (!e) e = cudaMemcpy(d_js, js.data(), sizeof(int64_t) * js.size(), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(d_pm, pm.data(), sizeof(int64_t) * pm.size(), cudaMemcpyHostToDevice);
  const int64_t Q3 = (int64_t)sp->Q * sp->Q * sp->Q;
  if (!e) e = ks_element_blocks_q1(sp->Q, ctx->stream, sp->ne, root->qd, root->space->ne * Q3, root->layout, &sp->tab,
                                   d_coo);
  if (!e) e = ks_coo_sum(ctx->stream, (int64_t)cl.size(), d_js, d_pm, d_coo, d_val);
  if (!e) e = cudaMemcpyAsync(val, d_val, sizeof(double) * 9 * cl.size(), cudaMemcpyDeviceToHost, ctx->stream);
  if (!e) e = cudaStreamSynchronize(ctx->stream);
  std::vector<uint8_t> bc((size_t)sp->n_nodes);
  if (!e) e = cudaMemcpy(bc.data(), sp->bc, sp->n_nodes, cudaMemcpyDeviceToHost);
  release();
  if (e) return nh_cuda_check(ctx, e, "nh_op_assemble_q1");
  ctx->launches += 2;
  // Dirichlet convention: constrained rows are identity rows, constrained columns dropped
  for (int64_t n = 0; n < sp->n_nodes; n++)
    for (int64_t s = rp[n]; s < rp[n + 1]; s++)
      for (int c = 0; c < 3; c++)
        for (int c2 = 0; c2 < 3; c2++) {
          double& v = val[s * 9 + 3 * c + c2];
          if ((bc[n] >> c) & 1u) v = (cl[s] == n && c == c2) ? 1.0 : 0.0;
          else if ((bc[cl[s]] >> c2) & 1u) v = 0.0;
        }
  memcpy(rowptr, rp.data(), sizeof(int64_t) * rp.size());
  memcpy(col, cl.data(), sizeof(int) * cl.size());
  return NH_OK;
}

// ---------------------------------------------------------------------------
// transfer
// ---------------------------------------------------------------------------
nh_status nh_transfer_internal(nh_space c, nh_space f, nh_prec prec, int dir, const void* in, void* out) {
  if (!c || !f || !in || !out) return NH_ERR_ARG;
  nh_ctx ctx = f->ctx;
  if (!nh_same_mesh(c, f) || c->p >= f->p)
    return nh_fail(ctx, NH_ERR_ARG, "nh_prolong/nh_restrict: spaces must share the mesh with p_c < p_f");
  if (prec != NH_F64 && prec != NH_F32) return nh_fail(ctx, NH_ERR_ARG, "transfer: bad precision");
  if (in == (const void*)out) return nh_fail(ctx, NH_ERR_ARG, "transfer: in and out must not alias");
  if (!aligned(in, 16) || !aligned(out, 16)) return nh_fail(ctx, NH_ERR_ARG, "transfer: misaligned vector");
  double xc[NH_MAXP], xf[NH_MAXP], B[NH_MAXP * NH_MAXP];
  nh_lobatto(c->P, xc);
  nh_lobatto(f->P, xf);
  nh_lagrange(c->P, xc, f->P, xf, B, nullptr);  // [Pf][Pc]
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  nh_space dst = dir == 0 ? f : c;
  NH_CUDA(ctx, cudaMemsetAsync(out, 0, (prec == NH_F64 ? 8 : 4) * dst->n_dof, ctx->stream));
  cudaError_t e = nh_launch_transfer(c->P, f->P, prec, dir, f->ne, c->emap, f->emap, f->inv_mult, f->inv_mult_f, in,
                                     out, B, ctx->stream);
  if (e == cudaErrorInvalidValue) return nh_fail(ctx, NH_ERR_UNSUPPORTED, "transfer: (p_c, p_f) not compiled");
  NH_CUDA(ctx, e);
  ctx->launches++;
  return NH_OK;
}

extern "C" nh_status nh_prolong(nh_space coarse, nh_space fine, nh_prec prec, const void* uc, void* uf) {
  return nh_transfer_internal(coarse, fine, prec, 0, uc, uf);
}

extern "C" nh_status nh_restrict(nh_space fine, nh_space coarse, nh_prec prec, const void* rf, void* rc) {
  return nh_transfer_internal(coarse, fine, prec, 1, rf, rc);
}

// ---------------------------------------------------------------------------
// vectors
// ---------------------------------------------------------------------------
extern "C" nh_status nh_dot(nh_ctx ctx, int64_t n, const double* x, const double* y, double* res) {
  if (!ctx || !res || n < 0) return NH_ERR_ARG;
  if (n == 0) {
    *res = 0.0;
    return NH_OK;
  }
  if (!x || !y) return NH_ERR_ARG;
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  NH_CUDA(ctx, nh_launch_dot_partials(n, x, y, ctx->red, kRedBlocks, ctx->stream));
  NH_CUDA(ctx, nh_launch_sum_partials(ctx->red, kRedBlocks, ctx->red + kRedBlocks, ctx->stream));
  ctx->launches += 2;
  NH_CUDA(ctx, cudaMemcpyAsync(ctx->red_host, ctx->red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  NH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *res = ctx->red_host[0];
  return NH_OK;
}

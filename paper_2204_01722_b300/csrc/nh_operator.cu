// Fused element kernels of the Neo-Hookean operator (Sec. II-B, II-C):
//   Jacobian action  y = E^T B^T D B E du     (Eq. Jacobian-discrete-ref)
//   residual/qdata   r = E^T B_xi^T W f1(u)   (Eq. residual-discrete-ref)
//   diagonal of J for Jacobi smoothing         (Sec. III-B)
// E (gather/scatter through the element map), B (sum-factorised tensor
// contractions, gradients by the collocated derivative B_xi B_I^+ so a gradient
// costs 6 instead of 9 contractions) and D (pointwise quadrature function) run in
// one kernel; E-vectors and Q-vectors live only in registers and shared memory.
//
// Thread layout: each element is handled by Q*Q threads, thread (a, b) owning the
// quadrature column (qi = a, qj = b) and looping over qk in registers; the
// x- and y-contractions exchange data through shared memory.  A block holds EPB
// elements (about 128 threads).  Scatter-add uses atomics.
//
// This file is compiled once per P (nodes per direction), with -DNH_P_INST=P.
#include "nh_internal.cuh"
#include "nh_pointwise.cuh"
#include "nh_ff.cuh"
#include "nh_setup_point.cuh"

#ifndef NH_P_INST
#error "compile with -DNH_P_INST=<P>"
#endif

namespace {

__host__ __device__ constexpr int epb_for(int Q) { return nh_epb(Q); }

// Resident blocks per SM requested from the register allocator.  The float-float
// kernel runs on the FP32 pipes, which need more warps in flight than the FP64
// pipe to stay busy; left unconstrained it takes up to 255 registers (2 blocks of
// ~128 threads).  Measured on B300 (Q3 on 48^3): 2 blocks 2.97, 3 blocks 4.20,
// 4 blocks 4.78 GDoF/s; for q = 5 three blocks beat four (4.32 vs 4.06), the
// spills of a 128-register cap outweigh the extra warps.
// FP32 block-row scatter: tried when every block lies in one row of elements (the
// x-element count a multiple of the block's elements), or always (blocks that
// straddle two rows fall back at run time) when NH_F32_ROWS_ANY or q <= 3.
// Measured on B300 with rows straddled: q = 3 +0.9%, q = 5 -0.4%, q = 4 unchanged.
#ifndef NH_F32_ROWS_ANY
#define NH_F32_ROWS_ANY 0
#endif

#ifndef NH_FF_MIN_BLOCKS_SMALLQ
#define NH_FF_MIN_BLOCKS_SMALLQ 4
#endif
#ifndef NH_FF_MIN_BLOCKS_Q3
#define NH_FF_MIN_BLOCKS_Q3 5
#endif
// Rolled float-float kernel (Q2 / Q3 / Q4 GDoF/s on B300 with 3, 4, 5 blocks of
// registers per SM): q = 3 6.08 / 6.08 / 6.40, q = 4 6.99 / 7.58 / 7.26, q = 5
// 7.07 / 7.06 / 7.09 (2, 3, 4 blocks).
// z-fluxes of the rolled float-float kernel in thread-local memory instead of a
// fourth shared buffer (each thread reads back only its own column): for q with
// the bit set in NH_FF_ZLOCAL_QMASK, where the shared buffer bounds the resident
// blocks (q = 5: 3 -> 4 blocks per SM)
#ifndef NH_FF_ZLOCAL_QMASK
#define NH_FF_ZLOCAL_QMASK (1 << 5)
#endif
__host__ __device__ constexpr bool ffr_zlocal(int Q) { return (NH_FF_ZLOCAL_QMASK >> Q) & 1; }

template <typename T, int Q>
__host__ __device__ constexpr int apply_min_blocks() {
  return std::is_same<T, ff>::value
             ? (Q <= 3 ? NH_FF_MIN_BLOCKS_Q3 : Q == 4 ? NH_FF_MIN_BLOCKS_SMALLQ : ffr_zlocal(Q) ? 4 : 3)
             : 1;
}

// Shared-memory stride of one element's [9][Q^3] work area, padded so that the
// Q*Q threads of consecutive elements in a warp fall on different banks
// (stride = Q^2 modulo the number of T words that cover the 32 banks).
template <int Q, typename T>
__host__ __device__ constexpr int elem_stride() {
  constexpr int base = 9 * Q * Q * Q, W = 128 / (int)sizeof(T), want = (Q * Q) % W;
  return Q * Q >= W ? base : base + ((want - base % W) % W + W) % W;
}

// ---- TMA (1-D bulk copy) and mbarrier helpers -----------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// read-only global load that does not allocate in L1 (streamed data read once)
__device__ __forceinline__ float ldg_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// global -> shared bulk copy completing on the mbarrier (addresses 16-B aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: after kMaxSpin polls the kernel flags the error and goes on
constexpr unsigned kMaxSpin = 1u << 26;
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err) {
  for (unsigned it = 0; !mbar_try_wait(bar, parity); it++) {
    if (it >= kMaxSpin) {
      if (err) atomicExch(err, 1);
      return;
    }
  }
}

template <int Q>
__device__ __forceinline__ int sidx(int c, int k, int j, int i) {
  return ((c * Q + k) * Q + j) * Q + i;
}

#if NH_P_INST == 2
// Failure-detection test: an mbarrier that no copy or thread ever completes; the
// bounded wait gives up after `limit` polls and sets the error flag.
__global__ void k_wait_timeout_mbar(int* err, unsigned limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  for (unsigned it = 0; !mbar_try_wait(&bar, 0); it++) {
    if (it >= limit) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      break;
    }
  }
}
#endif

using nhpw::pointwise;

// Float-float pointwise stage as one out-of-line copy: inlined once per
// quadrature plane, the double-single code overflows the instruction cache.
template <int LAYOUT>
__device__ __noinline__ void pointwise_ff(const ff* q, int64_t s, const ff (&g)[3][3], ff (&f)[3][3]) {
  pointwise<LAYOUT, ff>(q, s, g, f);
}

// s + a * b as one fused operation: FMA for float and double; for float-float
// the product's error terms and the running sum share one renormalisation.
__device__ __forceinline__ float madd(float s, float a, float b) { return s + a * b; }
__device__ __forceinline__ double madd(double s, double a, double b) { return fma(a, b, s); }
__device__ __forceinline__ ff madd(ff s, ff a, ff b) { return ff_madd(s, a, b); }

// ---------------------------------------------------------------------------
// Sum-factorised element stages.  Shared buffers bA, bB, bC are [3][Q][Q][Q].
// ---------------------------------------------------------------------------

// E then B_I: gather the element's P^3 nodes (masking constrained components if
// mask_in) and interpolate to the Q^3 points.  Leaves the point values in U
// (registers, this thread's column) and in bC; remembers node ids in nid.
template <int P, int Q, typename T, typename TS = T>
__device__ __forceinline__ void gather_interp(bool live, bool mask_in, int64_t e, int a, int b, const int* __restrict__ emap,
                                              const uint8_t* __restrict__ bc, const TS* __restrict__ src,
                                              const KTab<P, Q, T>& tab, T* bA, T* bB, T* bC, T (&U)[3][Q],
                                              int (&nid)[P]) {
  constexpr int P3 = P * P * P;
  if (a < P && b < P) {
    T r[3][P];
#pragma unroll
    for (int k = 0; k < P; k++) {
      int n = live ? __ldg(&emap[e * P3 + (k * P + b) * P + a]) : 0;
      nid[k] = n;
      unsigned m = (mask_in && live) ? (unsigned)__ldg(&bc[n]) : 0u;
#pragma unroll
      for (int c = 0; c < 3; c++) r[c][k] = (live && !((m >> c) & 1u)) ? T(src[3 * (int64_t)n + c]) : T(0);
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int qk = 0; qk < Q; qk++) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < P; k++) s = madd(s, tab.B[qk][k], r[c][k]);
        bA[sidx<Q>(c, qk, b, a)] = s;
      }
  } else {
#pragma unroll
    for (int k = 0; k < P; k++) nid[k] = 0;
  }
  __syncthreads();
  if (a < P) {
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int qk = 0; qk < Q; qk++) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < P; j++) s = madd(s, tab.B[b][j], bA[sidx<Q>(c, qk, j, a)]);
        bB[sidx<Q>(c, qk, b, a)] = s;
      }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int qk = 0; qk < Q; qk++) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < P; i++) s = madd(s, tab.B[a][i], bB[sidx<Q>(c, qk, b, i)]);
      U[c][qk] = s;
      bC[sidx<Q>(c, qk, b, a)] = s;
    }
}

// Collocated gradient at point (a, b, qk): g[c][d] = d u_c / d xi_d.
template <int P, int Q, typename T>
__device__ __forceinline__ void colloc_grad(int a, int b, int qk, const KTab<P, Q, T>& tab, const T* bC,
                                            const T (&U)[3][Q], T (&g)[3][3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
    for (int m = 0; m < Q; m++) {
      gx = madd(gx, tab.D[a][m], bC[sidx<Q>(c, qk, b, m)]);
      gy = madd(gy, tab.D[b][m], bC[sidx<Q>(c, qk, m, a)]);
      gz = madd(gz, tab.D[qk][m], U[c][m]);
    }
    g[c][0] = gx;
    g[c][1] = gy;
    g[c][2] = gz;
  }
}

// Transposed collocated derivative and B_I^T: from fluxes f_x (bA), f_y (bB) and
// f_z (registers Fz) back to the element's nodes.  Leaves the nodal result of
// thread (i = a, j = b) in out[c][k].  The caller must have synchronised after
// writing bA/bB and after the last read of bC.
template <int P, int Q, typename T>
__device__ __forceinline__ void transpose_to_nodes(int a, int b, const KTab<P, Q, T>& tab, T* bA, T* bB, T* bC,
                                                   const T (&Fz)[3][Q], T (&out)[3][P]) {
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int qk = 0; qk < Q; qk++) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < Q; m++) {
        s = madd(s, tab.D[m][a], bA[sidx<Q>(c, qk, b, m)]);
        s = madd(s, tab.D[m][b], bB[sidx<Q>(c, qk, m, a)]);
        s = madd(s, tab.D[m][qk], Fz[c][m]);
      }
      bC[sidx<Q>(c, qk, b, a)] = s;
    }
  __syncthreads();
  if (a < P) {
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int qk = 0; qk < Q; qk++) {
        T s = T(0);
#pragma unroll
        for (int qi = 0; qi < Q; qi++) s = madd(s, tab.B[qi][a], bC[sidx<Q>(c, qk, b, qi)]);
        bA[sidx<Q>(c, qk, b, a)] = s;
      }
  }
  __syncthreads();
  if (a < P && b < P) {
    T w[3][Q];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int qk = 0; qk < Q; qk++) {
        T s = T(0);
#pragma unroll
        for (int qj = 0; qj < Q; qj++) s = madd(s, tab.B[qj][b], bA[sidx<Q>(c, qk, qj, a)]);
        w[c][qk] = s;
      }
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < P; k++) {
        T s = T(0);
#pragma unroll
        for (int qk = 0; qk < Q; qk++) s = madd(s, tab.B[qk][k], w[c][qk]);
        out[c][k] = s;
      }
  }
}

// ---------------------------------------------------------------------------
// Jacobian action
// ---------------------------------------------------------------------------
// T: arithmetic type (double, or ff for FP64-accurate float-float on the FP32
// pipes); TV: type of the vectors du and y.
template <int P, int Q, typename T, typename TV, int LAYOUT, bool COL = false>
__global__ void __launch_bounds__(Q* Q* epb_for(Q), apply_min_blocks<T, Q>())
    k_jacobian_apply(int64_t ne, const int* __restrict__ emap, const uint8_t* __restrict__ bc,
                     const T* __restrict__ qd, int64_t qstride, const KTab<P, Q, T> tab, const TV* __restrict__ du,
                     TV* __restrict__ y, int lift, int colour, int nx, int ny, int nz) {
  constexpr int EPB = epb_for(Q), Q2 = Q * Q, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int t = threadIdx.x;
  const int el = t / Q2, col = t - el * Q2;
  const int a = col % Q, b = col / Q;
  int64_t e = (int64_t)blockIdx.x * EPB + el;
  bool live = e < ne;
  if constexpr (COL) {  // eight-colour scatter: the launch covers the elements of one parity class
    const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
    const int64_t cx = (nx - px + 1) / 2, cy = (ny - py + 1) / 2, cz = (nz - pz + 1) / 2;
    live = e < cx * cy * cz;
    const int64_t ix = e % cx, iy = (e / cx) % cy, iz = e / (cx * cy);
    e = live ? (px + 2 * ix) + nx * ((py + 2 * iy) + (int64_t)ny * (pz + 2 * iz)) : 0;
  }
  T* bA = sm + el * elem_stride<Q, T>();
  T* bB = bA + 3 * Q3;
  T* bC = bB + 3 * Q3;

  T U[3][Q];
  int nid[P];
  gather_interp<P, Q, T, TV>(live, !lift, e, a, b, emap, bc, du, tab, bA, bB, bC, U, nid);
  __syncthreads();
  T Fz[3][Q];
  const T* qe = qd + (live ? e : 0) * Q3 + b * Q + a;
#pragma unroll
  for (int qk = 0; qk < Q; qk++) {
    T g[3][3], f[3][3];
    colloc_grad<P, Q, T>(a, b, qk, tab, bC, U, g);
    if (live) {
      if constexpr (std::is_same<T, ff>::value)
        pointwise_ff<LAYOUT>(qe + qk * Q2, qstride, g, f);
      else
        pointwise<LAYOUT, T>(qe + qk * Q2, qstride, g, f);
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) f[i / 3][i % 3] = T(0);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      bA[sidx<Q>(c, qk, b, a)] = f[c][0];
      bB[sidx<Q>(c, qk, b, a)] = f[c][1];
      Fz[c][qk] = f[c][2];
    }
  }
  __syncthreads();
  T out[3][P];
  transpose_to_nodes<P, Q, T>(a, b, tab, bA, bB, bC, Fz, out);
  if (live && a < P && b < P) {
#pragma unroll
    for (int k = 0; k < P; k++) {
      const int n = nid[k];
      const unsigned m = __ldg(&bc[n]);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const int64_t dof = 3 * (int64_t)n + c;
        if ((m >> c) & 1u) {
          if (!lift) y[dof] = du[dof];  // identity row; every writer stores the same value
        } else if constexpr (COL) {
          y[dof] += (TV)out[c][k];  // no other element of this colour touches the node
        } else {
          atomicAdd(&y[dof], (TV)out[c][k]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Float-float Jacobian action with the quadrature-plane loops rolled.  One
// float-float multiply-add is 15 FP32 instructions, so the fully unrolled kernel
// above is several times the instruction cache; here every loop over qk runs
// one copy of its body (table coefficients indexed at run time from the
// constant bank), the point values and z-fluxes live in shared memory instead
// of qk-indexed registers, and the pointwise stage stays one out-of-line copy.
// Element work area: [12][Q^3] ff (u values, x-, y-, z-fluxes / scratch).
// ---------------------------------------------------------------------------
#ifndef NH_FF_ROLLED
#define NH_FF_ROLLED 1
#endif

// element stride in ff words, padded like elem_stride so that consecutive
// elements of a warp start on different banks
#ifndef NH_FF_DOT2
#define NH_FF_DOT2 1
#endif
// sum_{m < N} a_m b_m for the terms (a_m, b_m) = term(m): a compensated dot
// product (ffd_*), or a chain of float-float multiply-adds with NH_FF_DOT2=0
struct ffpair {
  ff a, b;
};
template <int N, typename F>
__device__ __forceinline__ ff ff_dot(F term) {
#if NH_FF_DOT2
  const ffpair t0 = term(0);
  ffdot d = ffd_first(t0.a, t0.b);
#pragma unroll
  for (int m = 1; m < N; m++) {
    const ffpair t = term(m);
    ffd_add(d, t.a, t.b);
  }
  return ffd_done(d);
#else
  ff s = ff(0);
#pragma unroll
  for (int m = 0; m < N; m++) {
    const ffpair t = term(m);
    s = ff_madd(s, t.a, t.b);
  }
  return s;
#endif
}

template <int Q>
__host__ __device__ constexpr int ffr_stride() {
  constexpr int base = (ffr_zlocal(Q) ? 9 : 12) * Q * Q * Q, W = 16, want = (Q * Q) % W;
  return Q * Q >= W ? base : base + ((want - base % W) % W + W) % W;
}

template <int P, int Q, int LAYOUT, bool COL = false>
__global__ void __launch_bounds__(Q* Q* epb_for(Q), apply_min_blocks<ff, Q>())
    k_jacobian_apply_ffr(int64_t ne, const int* __restrict__ emap, const uint8_t* __restrict__ bc,
                         const ff* __restrict__ qd, int64_t qstride, const KTab<P, Q, ff> tab,
                         const double* __restrict__ du, double* __restrict__ y, int lift, int colour, int nx, int ny,
                         int nz) {
  constexpr int EPB = epb_for(Q), Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  ff* sm = reinterpret_cast<ff*>(smraw);
  const int t = threadIdx.x;
  const int el = t / Q2, col = t - el * Q2;
  const int a = col % Q, b = col / Q;
  int64_t e = (int64_t)blockIdx.x * EPB + el;
  bool live = e < ne;
  if constexpr (COL) {
    const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
    const int64_t cx = (nx - px + 1) / 2, cy = (ny - py + 1) / 2, cz = (nz - pz + 1) / 2;
    live = e < cx * cy * cz;
    const int64_t ix = e % cx, iy = (e / cx) % cy, iz = e / (cx * cy);
    e = live ? (px + 2 * ix) + nx * ((py + 2 * iy) + (int64_t)ny * (pz + 2 * iz)) : 0;
  }
  ff* bA = sm + el * ffr_stride<Q>();  // [3][Q^3] each
  ff* bB = bA + 3 * Q3;
  ff* bC = bB + 3 * Q3;                 // point values
  ff* bD = bC + 3 * Q3;                 // z-fluxes (shared form)
  ff zl[3][Q];                          // z-fluxes (thread-local form)
  // E and B_I along x: thread (a, b) < P owns node column (i = a, j = b) over k
  int nid[P];
  if (a < P && b < P) {
    ff r[3][P];
#pragma unroll
    for (int k = 0; k < P; k++) {
      const int n = live ? __ldg(&emap[e * P3 + (k * P + b) * P + a]) : 0;
      nid[k] = n;
      const unsigned m = (!lift && live) ? (unsigned)__ldg(&bc[n]) : 0u;
#pragma unroll
      for (int c = 0; c < 3; c++) r[c][k] = (live && !((m >> c) & 1u)) ? ff(du[3 * (int64_t)n + c]) : ff(0);
    }
#pragma unroll 1
    for (int qk = 0; qk < Q; qk++) {
#pragma unroll
      for (int c = 0; c < 3; c++)
        bA[sidx<Q>(c, qk, b, a)] = ff_dot<P>([&](int k) { return ffpair{tab.B[qk][k], r[c][k]}; });
    }
  } else {
#pragma unroll
    for (int k = 0; k < P; k++) nid[k] = 0;
  }
  __syncthreads();
  if (a < P) {
#pragma unroll 1
    for (int qk = 0; qk < Q; qk++) {
#pragma unroll
      for (int c = 0; c < 3; c++)
        bB[sidx<Q>(c, qk, b, a)] = ff_dot<P>([&](int j) { return ffpair{tab.B[b][j], bA[sidx<Q>(c, qk, j, a)]}; });
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int qk = 0; qk < Q; qk++) {
#pragma unroll
    for (int c = 0; c < 3; c++)
      bC[sidx<Q>(c, qk, b, a)] = ff_dot<P>([&](int i) { return ffpair{tab.B[a][i], bB[sidx<Q>(c, qk, b, i)]}; });
  }
  __syncthreads();
  // gradients, pointwise, fluxes: x-, y-flux to bA, bB; z-flux to bD
  const ff* qe = qd + (live ? e : 0) * Q3 + b * Q + a;
#pragma unroll 1
  for (int qk = 0; qk < Q; qk++) {
    ff g[3][3], f[3][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      g[c][0] = ff_dot<Q>([&](int m) { return ffpair{tab.D[a][m], bC[sidx<Q>(c, qk, b, m)]}; });
      g[c][1] = ff_dot<Q>([&](int m) { return ffpair{tab.D[b][m], bC[sidx<Q>(c, qk, m, a)]}; });
      g[c][2] = ff_dot<Q>([&](int m) { return ffpair{tab.D[qk][m], bC[sidx<Q>(c, m, b, a)]}; });
    }
    if (live) {
      pointwise_ff<LAYOUT>(qe + qk * Q2, qstride, g, f);
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) f[i / 3][i % 3] = ff(0);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      bA[sidx<Q>(c, qk, b, a)] = f[c][0];
      bB[sidx<Q>(c, qk, b, a)] = f[c][1];
      if constexpr (ffr_zlocal(Q))
        zl[c][qk] = f[c][2];
      else
        bD[sidx<Q>(c, qk, b, a)] = f[c][2];
    }
  }
  __syncthreads();
  // transposed collocated derivative, summed over the three directions -> bC
#pragma unroll 1
  for (int qk = 0; qk < Q; qk++) {
#pragma unroll
    for (int c = 0; c < 3; c++)
      bC[sidx<Q>(c, qk, b, a)] = ff_dot<3 * Q>([&](int i) {
        const int m = i / 3, d = i % 3;
        return d == 0   ? ffpair{tab.D[m][a], bA[sidx<Q>(c, qk, b, m)]}
               : d == 1 ? ffpair{tab.D[m][b], bB[sidx<Q>(c, qk, m, a)]}
                        : ffpair{tab.D[m][qk], ffr_zlocal(Q) ? zl[c][m] : bD[sidx<Q>(c, m, b, a)]};
      });
  }
  __syncthreads();
  if (a < P) {  // B_I^T along x
#pragma unroll 1
    for (int qk = 0; qk < Q; qk++) {
#pragma unroll
      for (int c = 0; c < 3; c++)
        bA[sidx<Q>(c, qk, b, a)] = ff_dot<Q>([&](int qi) { return ffpair{tab.B[qi][a], bC[sidx<Q>(c, qk, b, qi)]}; });
    }
  }
  __syncthreads();
  if (a < P && b < P) {  // B_I^T along y, then along z into the node column's registers
    ff out[3][P];
#if NH_FF_DOT2
    ffdot od[3][P];  // compensated sums over the rolled plane loop, renormalised after it
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < P; k++) od[c][k] = ffdot{0.f, 0.f};
#else
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < P; k++) out[c][k] = ff(0);
#endif
#pragma unroll 1
    for (int qk = 0; qk < Q; qk++) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const ff w = ff_dot<Q>([&](int qj) { return ffpair{tab.B[qj][b], bA[sidx<Q>(c, qk, qj, a)]}; });
#pragma unroll
        for (int k = 0; k < P; k++) {
#if NH_FF_DOT2
          ffd_add(od[c][k], tab.B[qk][k], w);
#else
          out[c][k] = madd(out[c][k], tab.B[qk][k], w);
#endif
        }
      }
    }
#if NH_FF_DOT2
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < P; k++) out[c][k] = ffd_done(od[c][k]);
#endif
    if (live) {
#pragma unroll
      for (int k = 0; k < P; k++) {
        const int n = nid[k];
        const unsigned m = __ldg(&bc[n]);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const int64_t dof = 3 * (int64_t)n + c;
          if ((m >> c) & 1u) {
            if (!lift) y[dof] = du[dof];
          } else if constexpr (COL) {
            y[dof] += (double)out[c][k];
          } else {
            atomicAdd(&y[dof], (double)out[c][k]);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 Jacobian action, line-parallel.  Each of an element's Q^2 threads owns one
// 1-D line of the Q^3 (or P x Q^2 ...) lattice per stage -- an x-line (y, z), a
// y-line (x, z) or a z-line (x, y) -- reads that line from shared memory once,
// and produces all of the line's outputs in registers, so every 1-D contraction
// reads each value once (instead of once per output) and its coefficients are
// compile-time table entries (constant bank, no loads).  Stages:
//   x-lines over nodes:  gather E, B_I along x            -> A[c][k][j][qx]
//   y-lines:             B_I along y                       -> Bf[c][k][qy][qx]
//   z-lines:             B_I along z (u in registers), D_z  -> A = u
//   x-, y-lines:         D_x, D_y                          -> A = du/dx, Bf = du/dy
//   z-lines:             pointwise (quadrature data staged by TMA since block
//                        start), D_z^T of the z-flux in registers -> A, Bf = fluxes
//   x-, y-lines:         D_x^T, D_y^T                      -> A, Bf
//   z-lines:             sum the three directions, B_I^T along z -> A
//   y-lines:             B_I^T along y                     -> Bf
//   x-lines over nodes:  B_I^T along x, E^T (atomic scatter)
// The element map carries the Dirichlet bits (node id in bits 0..28,
// constrained components in bits 29..31).
// ---------------------------------------------------------------------------
constexpr unsigned kNodeBits = 29u, kNodeMask = (1u << kNodeBits) - 1u;

// Placement of the two [3][Q][Q][Q] work buffers of each element in shared
// memory.  q = 4 (16 threads per element, two elements per warp): the two
// elements of a pair share each 32-word row, one per 16-bank half, and a
// point's word within its plane is 4 ((y + z) mod 4) + ((x + y) mod 4) -- a
// bijection of (y, x) whose bank is distinct across the 16 lanes of an x-, y-
// or z-line access alike, so no access conflicts and nothing is padded.
// Other q: line pitch LP, plane pitch PP and element slot ES chosen by an
// exhaustive search over a 32-bank model of the kernel's accesses (all lanes of
// a warp, consecutive elements included) for the fewest wavefronts.
template <int Q>
struct LineLayout {
  static constexpr int LP = Q;
  static constexpr int PP = Q == 3 ? 11 : Q == 4 ? 32 : Q == 5 ? 25 : 39;
  static constexpr int CS = Q * PP;       // component stride
  static constexpr int BUF = 3 * CS;      // one [3][Q][Q][Q] buffer
  // floats per element slot (q = 4: per pair of elements, which share the rows)
  static constexpr int ES = Q == 3 ? 201 : Q == 4 ? 2 * BUF : Q == 5 ? 761 : 1412;
  static_assert(ES >= 2 * BUF, "element slot holds two buffers");
  __host__ __device__ static constexpr int elem(int el) { return Q == 4 ? (el >> 1) * ES + (el & 1) * 16 : el * ES; }
  __host__ __device__ static constexpr int block_floats(int epb) { return Q == 4 ? (epb + 1) / 2 * ES : epb * ES; }
  __device__ static constexpr int ix(int c, int z, int y, int x) {
    return Q == 4 ? c * CS + z * PP + 4 * ((y + z) & 3) + ((x + y) & 3) : c * CS + z * PP + y * LP + x;
  }
};

// Atomic add of v[K..N) to y[K..N), y + K - A 16-byte aligned when K = 0 (A = the
// run's start modulo 4 floats): 16-byte vector atomics where aligned, 8-byte or
// single ones at the ends; the sequence is fixed at compile time per alignment.
template <int A, int K, int N>
__device__ __forceinline__ void red_run(float* y, const float (&v)[N]) {
  if constexpr (K < N) {
    constexpr int al = (A + K) & 3;
    if constexpr (al == 0 && K + 4 <= N) {
      atomicAdd(reinterpret_cast<float4*>(y + K), make_float4(v[K], v[K + 1], v[K + 2], v[K + 3]));
      red_run<A, K + 4, N>(y, v);
    } else if constexpr ((al & 1) == 0 && K + 2 <= N) {
      atomicAdd(reinterpret_cast<float2*>(y + K), make_float2(v[K], v[K + 1]));
      red_run<A, K + 2, N>(y, v);
    } else {
      atomicAdd(y + K, v[K]);
      red_run<A, K + 1, N>(y, v);
    }
  }
}

// Vector loads of du[3 n0 .. 3 (n0 + N / 3)) into v, the mirror of red_run (A = the
// run's start modulo 4 floats, the base 16-byte aligned); read-only path.
template <int A, int K, int N>
__device__ __forceinline__ void ld_run(const float* x, float (&v)[N]) {
  if constexpr (K < N) {
    constexpr int al = (A + K) & 3;
    if constexpr (al == 0 && K + 4 <= N) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(x + K));
      v[K] = q.x;
      v[K + 1] = q.y;
      v[K + 2] = q.z;
      v[K + 3] = q.w;
      ld_run<A, K + 4, N>(x, v);
    } else if constexpr ((al & 1) == 0 && K + 2 <= N) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(x + K));
      v[K] = q.x;
      v[K + 1] = q.y;
      ld_run<A, K + 2, N>(x, v);
    } else {
      v[K] = __ldg(x + K);
      ld_run<A, K + 1, N>(x, v);
    }
  }
}

#ifndef NH_F32_VGATHER
#define NH_F32_VGATHER 1
#endif

#ifndef NH_F32_DIRECT_MINB
#define NH_F32_DIRECT_MINB 7
#endif
#ifndef NH_F32_DIRECT_PF
#define NH_F32_DIRECT_PF 1
#endif
// DIRECT (= nh_f32_direct(Q)): the quadrature data is loaded straight into
// registers, plane by plane with the next plane requested ahead, instead of
// through the shared-memory plane ring; registers are then capped for
// NH_F32_DIRECT_MINB resident blocks (a minimum of 0 blocks leaves the ring form's
// register count to the compiler, as without the argument).
template <int P, int Q, int LAYOUT, bool COL = false, bool DIRECT = nh_f32_direct(Q)>
__global__ void __launch_bounds__(Q* Q* epb_for(Q), DIRECT ? NH_F32_DIRECT_MINB : 0)
    k_jacobian_apply_f32l(int64_t ne, const unsigned* __restrict__ emapb, const float* __restrict__ qdb,
                          const KTab<P, Q, float> tab, const float* __restrict__ du, float* __restrict__ y, int lift,
                          int vec_ok, int rows_ok, int* __restrict__ err, int colour, int nbx, int ny, int nz) {
  static_assert(DIRECT == nh_f32_direct(Q), "the quadrature-data layout follows nh_f32_direct");
  using L = LineLayout<Q>;
  constexpr int EPB = epb_for(Q), Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
  constexpr int S = nh_layout_scalars(LAYOUT);
  constexpr long long BS = nh_f32_batch_floats(Q, S), PL = nh_f32_plane_floats(Q, S);
  constexpr long long RING = DIRECT ? 0 : 2 * PL;  // floats of the plane ring in shared memory
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ unsigned srun[EPB * P * P];        // start node of each node line's run (or ~0)
  float* qs = reinterpret_cast<float*>(smraw);  // two plane slots [2][PL]
  const int t = threadIdx.x;
  const int el = t / Q2, r = t - el * Q2;
  const int u = r % Q, v = r / Q;  // line coordinates of this thread
  // batch of EPB consecutive elements: the block's index, or with the eight-colour
  // scatter the colour's batch number blockIdx.x of batches classed by the parities
  // of their (batch x, row y, row z) indices (rows of nbx batches; no two batches of
  // a class share a node)
  int64_t batch = blockIdx.x;
  if constexpr (COL) {
    const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
    const int64_t cx = (nbx - px + 1) / 2, cy = (ny - py + 1) / 2;
    const int64_t ix = batch % cx, iy = (batch / cx) % cy, iz = batch / (cx * cy);
    batch = (px + 2 * ix) + nbx * ((py + 2 * iy) + (int64_t)ny * (pz + 2 * iz));
  }
  const int64_t e = batch * EPB + el;
  const bool live = e < ne;
  float* A = qs + RING + L::elem(el);
  float* Bf = A + L::BUF;
  // z-plane qz of the batch's quadrature data -> slot qz & 1 (one bulk copy)
  auto issue_plane = [&](int qz) {
    const unsigned bytes = (unsigned)(PL * sizeof(float));
    uint64_t* b = &bar[qz & 1];
    mbar_expect_tx(b, bytes);
    const char* src = reinterpret_cast<const char*>(qdb + batch * BS + qz * PL);
    char* dst = reinterpret_cast<char*>(qs + (qz & 1) * PL);
    for (unsigned off = 0; off < bytes; off += 16384u) {
      const unsigned chunk = bytes - off < 16384u ? bytes - off : 16384u;
      bulk_g2s(dst + off, src + off, chunk, b);
    }
  };
  // DIRECT: plane 0 of this thread's point, loaded at the start so that it
  // arrives during the interpolation stages
  const float* qg = qdb + batch * BS + t;
  float qv[DIRECT ? S : 1];
  if constexpr (DIRECT) {
    if constexpr (NH_F32_DIRECT_PF) {
#pragma unroll
      for (int k = 0; k < S; k++) qv[k] = ldg_stream(qg + k * nh_f32_npp(Q));
    }
    (void)issue_plane;
  } else {
    if (t == 0) {
      mbar_init(&bar[0]);
      mbar_init(&bar[1]);
    }
    __syncthreads();
    if (t == 0) {
      issue_plane(0);
      issue_plane(1);
    }
  }
  // x-lines over nodes (j = u, k = v): gather and B_I along x
  const bool node_line = u < P && v < P;
  unsigned nid[P];
  if (node_line) {
    float w[3][P];
    if constexpr (P == 4) {  // the node line is 16-byte aligned: one vector load
      const uint4 q4 = live ? __ldg(reinterpret_cast<const uint4*>(emapb + e * P3 + (v * P + u) * P)) : make_uint4(0, 0, 0, 0);
      nid[0] = q4.x;
      nid[1] = q4.y;
      nid[2] = q4.z;
      nid[3] = q4.w;
    } else {
#pragma unroll
      for (int i = 0; i < P; i++) nid[i] = live ? __ldg(&emapb[e * P3 + (v * P + u) * P + i]) : 0u;
    }
    // the line's P nodes consecutive and unconstrained (or lifted): its 3P values
    // are one contiguous run of du, read with vector loads.  Taken for P >= 5 only:
    // measured at full size, +2% at q = 5, -1 to -2% at q = 3 and 4 (the extra
    // registers and branches cost more than the fewer load requests save)
    bool vrun = NH_F32_VGATHER && P >= 5 && live && (vec_ok & 2);
    const unsigned n0 = nid[0] & kNodeMask;
#pragma unroll
    for (int i = 0; i < P; i++) vrun = vrun && (lift ? (nid[i] & kNodeMask) : nid[i]) == n0 + (unsigned)i;
    if (vrun) {
      float vv[3 * P];
      const float* xr = du + 3 * (int64_t)n0;
      switch ((3u * n0) & 3u) {
        case 0: ld_run<0, 0, 3 * P>(xr, vv); break;
        case 1: ld_run<1, 0, 3 * P>(xr, vv); break;
        case 2: ld_run<2, 0, 3 * P>(xr, vv); break;
        default: ld_run<3, 0, 3 * P>(xr, vv); break;
      }
#pragma unroll
      for (int i = 0; i < P; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) w[c][i] = vv[3 * i + c];
    } else {
#pragma unroll
      for (int i = 0; i < P; i++) {
        const int64_t n = nid[i] & kNodeMask;
        const unsigned m = (live && !lift) ? nid[i] >> kNodeBits : 0u;
#pragma unroll
        for (int c = 0; c < 3; c++) w[c][i] = (live && !((m >> c) & 1u)) ? __ldg(&du[3 * n + c]) : 0.f;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int qx = 0; qx < Q; qx++) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < P; i++) s += tab.B[qx][i] * w[c][i];
        A[L::ix(c, v, u, qx)] = s;
      }
  }
  __syncthreads();
  if (v < P) {  // y-lines (x = u, z = v)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float w[P];
#pragma unroll
      for (int j = 0; j < P; j++) w[j] = A[L::ix(c, v, j, u)];
#pragma unroll
      for (int qy = 0; qy < Q; qy++) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < P; j++) s += tab.B[qy][j] * w[j];
        Bf[L::ix(c, v, qy, u)] = s;
      }
    }
  }
  __syncthreads();
  // z-lines (x = u, y = v): point values and their z-derivative in registers
  float gz[3][Q];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float w[P], U[Q];
#pragma unroll
    for (int k = 0; k < P; k++) w[k] = Bf[L::ix(c, k, v, u)];
#pragma unroll
    for (int qz = 0; qz < Q; qz++) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < P; k++) s += tab.B[qz][k] * w[k];
      U[qz] = s;
      A[L::ix(c, qz, v, u)] = s;
    }
#pragma unroll
    for (int qz = 0; qz < Q; qz++) {
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < Q; m++) s += tab.D[qz][m] * U[m];
      gz[c][qz] = s;
    }
  }
  __syncthreads();
  // x-lines (y = u, z = v) and y-lines (x = u, z = v) of the collocated derivative
  float gx[3][Q], gy[3][Q];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float wx[Q], wy[Q];
#pragma unroll
    for (int m = 0; m < Q; m++) {
      wx[m] = A[L::ix(c, v, u, m)];
      wy[m] = A[L::ix(c, v, m, u)];
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int m = 0; m < Q; m++) {
        sx += tab.D[q][m] * wx[m];
        sy += tab.D[q][m] * wy[m];
      }
      gx[c][q] = sx;
      gy[c][q] = sy;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int q = 0; q < Q; q++) {
      A[L::ix(c, v, u, q)] = gx[c][q];
      Bf[L::ix(c, v, q, u)] = gy[c][q];
    }
  __syncthreads();
  // z-lines (x = u, y = v): pointwise at (u, v, qz); each point is read and
  // rewritten by its own z-line thread only.  Plane qz's data sits in slot
  // qz & 1; once every thread is past plane qz, plane qz + 2 is copied there.
  float vz[3][Q];
  {
    float fz[3][Q];
#pragma unroll
    for (int qz = 0; qz < Q; qz++) {
      float qn[DIRECT ? S : 1];               // DIRECT: the next plane's scalars, requested before this plane's work
      const float* qp = qs + (qz & 1) * PL;  // ring: this plane's slot
      if constexpr (DIRECT) {
        if constexpr (NH_F32_DIRECT_PF) {
          if (qz + 1 < Q) {
#pragma unroll
            for (int k = 0; k < S; k++) qn[k] = ldg_stream(qg + (qz + 1) * PL + k * nh_f32_npp(Q));
          }
        } else {
#pragma unroll
          for (int k = 0; k < S; k++) qv[k] = ldg_stream(qg + qz * PL + k * nh_f32_npp(Q));
        }
      } else {
        mbar_wait_bounded(&bar[qz & 1], (qz >> 1) & 1, err);
      }
      float g[3][3], f[3][3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        g[c][0] = A[L::ix(c, qz, v, u)];
        g[c][1] = Bf[L::ix(c, qz, v, u)];
        g[c][2] = gz[c][qz];
      }
      if (live) {
        if constexpr (DIRECT) {
          nhpw::pointwise_ld<LAYOUT, float>([&](int i) { return qv[i]; }, g, f);
        } else {
          // this point's scalars: S/4 rotated 16-byte chunks, then the remainder
          constexpr int NC = S / 4, R = S - 4 * NC, NP = EPB * Q2;
          float qr[S];
#pragma unroll
          for (int k = 0; k < NC; k++) {
            const float4 c4 = *reinterpret_cast<const float4*>(qp + t * 4 * NC + ((k + nh_f32_rot(S, t)) % NC) * 4);
            qr[4 * k] = c4.x;
            qr[4 * k + 1] = c4.y;
            qr[4 * k + 2] = c4.z;
            qr[4 * k + 3] = c4.w;
          }
#pragma unroll
          for (int j = 0; j < R; j++) qr[4 * NC + j] = qp[NP * 4 * NC + t * R + j];
          nhpw::pointwise_ld<LAYOUT, float>([&](int i) { return qr[i]; }, g, f);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 9; i++) f[i / 3][i % 3] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < 3; c++) {
        A[L::ix(c, qz, v, u)] = f[c][0];
        Bf[L::ix(c, qz, v, u)] = f[c][1];
        fz[c][qz] = f[c][2];
      }
      if constexpr (DIRECT) {
        if (NH_F32_DIRECT_PF && qz + 1 < Q) {
#pragma unroll
          for (int k = 0; k < S; k++) qv[k] = qn[k];
        }
      } else {
        if (qz + 2 < Q) {
          __syncthreads();
          if (t == 0) issue_plane(qz + 2);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int qz = 0; qz < Q; qz++) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < Q; m++) s += tab.D[m][qz] * fz[c][m];
        vz[c][qz] = s;
      }
  }
  __syncthreads();
  // x-lines (y = u, z = v): D_x^T of the x-flux; y-lines (x = u, z = v): D_y^T
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float wx[Q], wy[Q];
#pragma unroll
    for (int m = 0; m < Q; m++) {
      wx[m] = A[L::ix(c, v, u, m)];
      wy[m] = Bf[L::ix(c, v, m, u)];
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int m = 0; m < Q; m++) {
        sx += tab.D[m][q] * wx[m];
        sy += tab.D[m][q] * wy[m];
      }
      gx[c][q] = sx;
      gy[c][q] = sy;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int q = 0; q < Q; q++) {
      A[L::ix(c, v, u, q)] = gx[c][q];
      Bf[L::ix(c, v, q, u)] = gy[c][q];
    }
  __syncthreads();
  // z-lines (x = u, y = v): sum of the three directions, then B_I^T along z
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float w[Q];
#pragma unroll
    for (int qz = 0; qz < Q; qz++) w[qz] = A[L::ix(c, qz, v, u)] + Bf[L::ix(c, qz, v, u)] + vz[c][qz];
#pragma unroll
    for (int k = 0; k < P; k++) {
      float s = 0.f;
#pragma unroll
      for (int qz = 0; qz < Q; qz++) s += tab.B[qz][k] * w[qz];
      A[L::ix(c, k, v, u)] = s;
    }
  }
  __syncthreads();
  if (v < P) {  // y-lines (x = u, z = v): B_I^T along y
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float w[Q];
#pragma unroll
      for (int m = 0; m < Q; m++) w[m] = A[L::ix(c, v, m, u)];
#pragma unroll
      for (int j = 0; j < P; j++) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < Q; m++) s += tab.B[m][j] * w[m];
        Bf[L::ix(c, v, j, u)] = s;
      }
    }
  }
  __syncthreads();
  // x-lines over nodes (j = u, k = v): B_I^T along x
  float o[3][P];
  unsigned n0 = 0;
  bool run = false;
  if (node_line) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float w[Q];
#pragma unroll
      for (int m = 0; m < Q; m++) w[m] = Bf[L::ix(c, v, u, m)];
#pragma unroll
      for (int i = 0; i < P; i++) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < Q; m++) s += tab.B[m][i] * w[m];
        o[c][i] = s;
      }
    }
    // the line's P nodes consecutive and unconstrained (box meshes away from
    // Dirichlet faces): their 3P values are one contiguous run of y
    n0 = nid[0] & kNodeMask;
    run = live && (vec_ok & 1) != 0;
#pragma unroll
    for (int i = 0; i < P; i++) run = run && nid[i] == n0 + (unsigned)i;
    if (rows_ok) srun[(el * P + v) * P + u] = run ? n0 : 0xffffffffu;
  }
  // E^T.  When the block's elements follow one another along x (rows_ok: the
  // box has a multiple of EPB elements along x) and every line is such a run,
  // each (j, k) row of the block is one contiguous run of
  // RN = EPB (P - 1) + 1 nodes: the rows are summed in shared memory (shared
  // element faces added once) and reduced into y by the bulk-copy engine.
  // Row pitch RS: a multiple of 4 floats (16-byte aligned bulk sources) with RS / 4
  // odd, so that the rows of 8 consecutive lines start on distinct bank quads.
  constexpr int RN = EPB * (P - 1) + 1, RL = 3 * RN, RS0 = (RL + 6) / 4 * 4;
  constexpr int RS = (RS0 / 4) % 2 ? RS0 : RS0 + 4;
  static_assert(P * P * RS <= L::block_floats(EPB), "row buffer fits the work area");
  bool chain = false;
  unsigned first = 0;
  if (rows_ok) {  // uniform: the barriers below are taken by all threads or none
    __syncthreads();
    chain = true;
    if (node_line) {
      first = srun[v * P + u];
      chain = first != 0xffffffffu && srun[(el * P + v) * P + u] == first + (unsigned)(el * (P - 1));
    }
    chain = __syncthreads_and(chain) != 0;
  }
  if (chain) {
    float* Rr = qs + RING + (v * P + u) * RS + ((3u * first) & 3u);  // node x, component c at 3 x + c
    if (node_line) {
#pragma unroll
      for (int i = 1; i < P; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) Rr[3 * (el * (P - 1) + i) + c] = o[c][i];
      if (el == 0) {
#pragma unroll
        for (int c = 0; c < 3; c++) Rr[c] = o[c][0];
      }
    }
    __syncthreads();
    if (node_line && el > 0) {
#pragma unroll
      for (int c = 0; c < 3; c++) Rr[3 * el * (P - 1) + c] += o[c][0];
    }
    if constexpr (COL) {  // colour mode: the block's rows added to y by all threads, no atomics
      __syncthreads();
      constexpr int NR = P * P;
      for (int k = t; k < NR * RL; k += Q2 * EPB) {
        const int row = k / RL, off = k - row * RL;
        const unsigned f = srun[row];
        y[3 * (int64_t)f + off] += qs[RING + row * RS + ((3u * f) & 3u) + off];
      }
      return;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // shared writes -> bulk-copy reads
    __syncthreads();
    if (node_line && el == 0) {
      float* g = y + 3 * (int64_t)first;
      const int h = (int)((4u - ((3u * first) & 3u)) & 3u);  // floats before a 16-byte boundary
      const int mid = (RL - h) / 4 * 4;
      for (int k = 0; k < h; k++) atomicAdd(g + k, Rr[k]);
      if (mid > 0) {
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(g + h),
                     "r"(smem_u32(Rr + h)), "r"((unsigned)(mid * 4))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
      for (int k = h + mid; k < RL; k++) atomicAdd(g + k, Rr[k]);
      if (mid > 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    return;
  }
  if constexpr (COL) {  // colour mode: the block's elements one after another (shared x-faces), no atomics
    for (int rr = 0; rr < EPB; rr++) {
      if (rr == el && live && node_line) {
#pragma unroll
        for (int i = 0; i < P; i++) {
          const int64_t n = nid[i] & kNodeMask;
          const unsigned m = nid[i] >> kNodeBits;
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const int64_t dof = 3 * n + c;
            if ((m >> c) & 1u) {
              if (!lift) y[dof] = du[dof];
            } else {
              y[dof] += o[c][i];
            }
          }
        }
      }
      __syncthreads();
    }
    return;
  }
  if (live && node_line) {
    if (run) {
      float v[3 * P];
#pragma unroll
      for (int i = 0; i < P; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[3 * i + c] = o[c][i];
      float* yr = y + 3 * (int64_t)n0;
      switch ((3u * n0) & 3u) {
        case 0: red_run<0, 0, 3 * P>(yr, v); break;
        case 1: red_run<1, 0, 3 * P>(yr, v); break;
        case 2: red_run<2, 0, 3 * P>(yr, v); break;
        default: red_run<3, 0, 3 * P>(yr, v); break;
      }
    } else {
#pragma unroll
      for (int i = 0; i < P; i++) {
        const int64_t n = nid[i] & kNodeMask;
        const unsigned m = nid[i] >> kNodeBits;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const int64_t dof = 3 * n + c;
          if ((m >> c) & 1u) {
            if (!lift) y[dof] = du[dof];  // identity row; every writer stores the same value
          } else {
            atomicAdd(&y[dof], o[c][i]);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Quadrature-data setup and residual (FP64).  Gradients of the node
// coordinates X (isoparametric geometry) and of u at each point give
// dX/dxi, W = w det(dX/dxi), H = grad_X u, F = I + H, J - 1 from the invariants
// of H (log J = log1p(J - 1) without cancellation), Green-Euler strain
// e = (H + H^T + H H^T)/2, Kirchhoff stress tau = 2 mu e + lambda log J I
// (Eq. Kirchhoff-stress) and grad_x xi = grad_X xi F^-1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double det3(const double (&A)[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// inverse via the adjugate; returns det
__device__ __forceinline__ double inv3(const double (&A)[3][3], double (&Ai)[3][3]) {
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

template <int P, int Q>
struct SetupTab {
  KTab<P, Q, double> k;
  double w[Q];
};

template <int P, int Q, int LAYOUT, int GEOM>
__global__ void __launch_bounds__(Q* Q* epb_for(Q))
    k_setup(int64_t ne, const int* __restrict__ emap, const uint8_t* __restrict__ bc,
            const double* __restrict__ coords, const double* __restrict__ u, const double* __restrict__ lamv,
            const double* __restrict__ muv, const SetupTab<P, Q> st, double* __restrict__ qd, int64_t qstride,
            int store, int resid, const double* __restrict__ gbc, double* __restrict__ r,
            unsigned long long* __restrict__ minj, double* __restrict__ geom) {
  constexpr int EPB = epb_for(Q), Q2 = Q * Q, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sm = reinterpret_cast<double*>(smraw);
  const int t = threadIdx.x;
  const int el = t / Q2, col = t - el * Q2;
  const int a = col % Q, b = col / Q;
  const int64_t e = (int64_t)blockIdx.x * EPB + el;
  const bool live = e < ne;
  double* bA = sm + el * 12 * Q3;
  double* bB = bA + 3 * Q3;
  double* bX = bB + 3 * Q3;
  double* bU = bX + 3 * Q3;
  const KTab<P, Q, double>& tab = st.k;

  // geometry factors grad_X xi and det(dX/dxi) per point, [10][ne Q^3] in geom:
  // GEOM 0 computes them from the node coordinates, 1 computes and keeps them,
  // 2 reads the kept ones (the mesh does not move)
  double UX[3][Q], UU[3][Q];
  int nid[P];
  if constexpr (GEOM != 2) {
    gather_interp<P, Q, double>(live, false, e, a, b, emap, bc, coords, tab, bA, bB, bX, UX, nid);
    __syncthreads();
  }
  gather_interp<P, Q, double>(live, false, e, a, b, emap, bc, u, tab, bA, bB, bU, UU, nid);
  __syncthreads();

  const double lam = live ? lamv[e] : 0.0, mu = live ? muv[e] : 0.0;
  double Fz[3][Q];
  double jmin = 1e300;
  for (int qk = 0; qk < Q; qk++) {
    double gU[3][3], R[3][3], detx = 1.0;
    colloc_grad<P, Q, double>(a, b, qk, tab, bU, UU, gU);
    const int64_t pt = e * Q3 + qk * Q2 + b * Q + a;
    if constexpr (GEOM == 2) {
      if (live) {
#pragma unroll
        for (int i = 0; i < 9; i++) R[i / 3][i % 3] = geom[i * qstride + pt];
        detx = geom[9 * qstride + pt];
      }
    } else {
      double gX[3][3];
      colloc_grad<P, Q, double>(a, b, qk, tab, bX, UX, gX);
      detx = nh_inv3(gX, R);
      if (GEOM == 1 && live) {
#pragma unroll
        for (int i = 0; i < 9; i++) geom[i * qstride + pt] = R[i / 3][i % 3];
        geom[9 * qstride + pt] = detx;
      }
    }
    double f[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (live)
      nh_setup_point_geom<LAYOUT>(R, detx, gU, st.w[a] * st.w[b] * st.w[qk], lam, mu, qd + pt, qstride, store, resid, f,
                                  jmin);
    if (resid) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        bA[sidx<Q>(c, qk, b, a)] = f[c][0];
        bB[sidx<Q>(c, qk, b, a)] = f[c][1];
        Fz[c][qk] = f[c][2];
      }
    }
  }
  if (minj) {  // block-wide min of det F (blocks may end in a partial warp), one global atomic
    __shared__ unsigned long long bmin;
    if (t == 0) bmin = ~0ull;
    __syncthreads();
    atomicMin(&bmin, ordered_bits(jmin));
    __syncthreads();
    if (t == 0) atomicMin(minj, bmin);
  }
  if (!resid) return;  // uniform across the block
  __syncthreads();
  double out[3][P];
  transpose_to_nodes<P, Q, double>(a, b, tab, bA, bB, bX, Fz, out);
  if (live && a < P && b < P) {
#pragma unroll
    for (int k = 0; k < P; k++) {
      const int n = nid[k];
      const unsigned m = __ldg(&bc[n]);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const int64_t dof = 3 * (int64_t)n + c;
        if ((m >> c) & 1u)
          r[dof] = u[dof] - (gbc ? gbc[dof] : 0.0);
        else
          atomicAdd(&r[dof], out[c][k]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Diagonal of J.  For component c the pointwise tangent block
// D^c[d][d'] = d f[c][d] / d g[c][d'] is obtained by applying the pointwise map
// to the three unit gradients e_c (x) e_d'.  Then
// diag[c](i,j,k) = sum_q sum_{d,d'} Phi_d Phi_d' D^c[d][d'], Phi_d = B_xi,d[q, node],
// contracted direction by direction with the elementwise products of the 1-D
// value/derivative tables (B.B, B.G, G.G).
// ---------------------------------------------------------------------------
template <int P, int Q, typename T = double>
struct DiagTab {
  T BB[Q][P], BG[Q][P], GG[Q][P];
};

template <int P, int Q, int LAYOUT, typename TO>
__global__ void __launch_bounds__(Q* Q* epb_for(Q))
    k_diagonal(int64_t ne, const int* __restrict__ emap, const uint8_t* __restrict__ bc,
               const double* __restrict__ qd, int64_t qstride, const DiagTab<P, Q, TO> dt, TO* __restrict__ diag) {
  using T = TO;  // arithmetic in the output's precision (FP32 for the FP32 smoothers' diagonals)
  constexpr int EPB = epb_for(Q), Q2 = Q * Q, Q3 = Q * Q * Q, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int t = threadIdx.x;
  const int el = t / Q2, col = t - el * Q2;
  const int a = col % Q, b = col / Q;
  const int64_t e = (int64_t)blockIdx.x * EPB + el;
  const bool live = e < ne;
  T* Dsm = sm + el * 11 * Q3;  // [9][Q][Q][Q]
  T* s1 = Dsm + 9 * Q3;        // [P][Q][Q]
  T* s2 = s1 + Q3;             // [P][P][Q]
  const double* qe = qd + (live ? e : 0) * Q3 + b * Q + a;

  for (int c = 0; c < 3; c++) {
    for (int qk = 0; qk < Q; qk++) {
      if (LAYOUT == NH_LAYOUT_CURRENT) {
        // closed form of Eq. dtau's tangent block: D^c[d][d'] = A_dd' + (a + h) X_dc X_d'c,
        // A = X (W tau) X^T + h X X^T, a = W lambda, h = W (mu - lambda log J)
        T Dc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (live) {
          const double* qp = qe + qk * Q2;
          T X[3][3];
#pragma unroll
          for (int i = 0; i < 9; i++) X[i / 3][i % 3] = (T)qp[i * qstride];
          const T t00 = (T)qp[9 * qstride], t11 = (T)qp[10 * qstride], t22 = (T)qp[11 * qstride];
          const T t12 = (T)qp[12 * qstride], t02 = (T)qp[13 * qstride], t01 = (T)qp[14 * qstride];
          const T tau[3][3] = {{t00, t01, t02}, {t01, t11, t12}, {t02, t12, t22}};
          const T wa = (T)qp[15 * qstride], wh = (T)qp[16 * qstride];
#pragma unroll
          for (int d = 0; d < 3; d++)
#pragma unroll
            for (int dp = 0; dp < 3; dp++) {
              T v = (wa + wh) * X[d][c] * X[dp][c];
#pragma unroll
              for (int k = 0; k < 3; k++)
                v += (X[d][0] * tau[0][k] + X[d][1] * tau[1][k] + X[d][2] * tau[2][k] + wh * X[d][k]) * X[dp][k];
              Dc[d][dp] = v;
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
          for (int dp = 0; dp < 3; dp++) Dsm[((d * 3 + dp) * Q + qk) * Q2 + b * Q + a] = Dc[d][dp];
        continue;
      }
#pragma unroll
      for (int dp = 0; dp < 3; dp++) {
        T g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, f[3][3];
        g[c][dp] = T(1);
        if (live) {
          const double* qp = qe + qk * Q2;
          nhpw::pointwise_ld<LAYOUT, T>([&](int i) { return (T)qp[i * qstride]; }, g, f);
        } else {
#pragma unroll
          for (int i = 0; i < 9; i++) f[i / 3][i % 3] = T(0);
        }
#pragma unroll
        for (int d = 0; d < 3; d++) Dsm[((d * 3 + dp) * Q + qk) * Q2 + b * Q + a] = f[c][d];
      }
    }
    __syncthreads();
    T acc[P];
#pragma unroll
    for (int k = 0; k < P; k++) acc[k] = T(0);
#pragma unroll
    for (int pr = 0; pr < 9; pr++) {
      const int d = pr / 3, dp = pr % 3;
      const T(*Mx)[P] = (d == 0 && dp == 0) ? dt.GG : ((d == 0 || dp == 0) ? dt.BG : dt.BB);
      const T(*My)[P] = (d == 1 && dp == 1) ? dt.GG : ((d == 1 || dp == 1) ? dt.BG : dt.BB);
      const T(*Mz)[P] = (d == 2 && dp == 2) ? dt.GG : ((d == 2 || dp == 2) ? dt.BG : dt.BB);
      const T* F = Dsm + pr * Q3;
      // z: thread (qi=a, qj=b)
#pragma unroll
      for (int k = 0; k < P; k++) {
        T s = T(0);
#pragma unroll
        for (int qk = 0; qk < Q; qk++) s += Mz[qk][k] * F[qk * Q2 + b * Q + a];
        s1[(k * Q + b) * Q + a] = s;
      }
      __syncthreads();
      // y: thread (qi=a, j=b<P)
      if (b < P) {
#pragma unroll
        for (int k = 0; k < P; k++) {
          T s = T(0);
#pragma unroll
          for (int qj = 0; qj < Q; qj++) s += My[qj][b] * s1[(k * Q + qj) * Q + a];
          s2[(k * P + b) * Q + a] = s;
        }
      }
      __syncthreads();
      // x: thread (i=a<P, j=b<P)
      if (a < P && b < P) {
#pragma unroll
        for (int k = 0; k < P; k++) {
          T s = T(0);
#pragma unroll
          for (int qi = 0; qi < Q; qi++) s += Mx[qi][a] * s2[(k * P + b) * Q + qi];
          acc[k] += s;
        }
      }
    }
    if (live && a < P && b < P) {
#pragma unroll
      for (int k = 0; k < P; k++) {
        const int n = __ldg(&emap[e * P3 + (k * P + b) * P + a]);
        const unsigned m = __ldg(&bc[n]);
        const int64_t dof = 3 * (int64_t)n + c;
        if ((m >> c) & 1u)
          diag[dof] = TO(1);
        else
          atomicAdd(&diag[dof], TO(acc[k]));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

// Raise the dynamic shared-memory limit of one kernel, once per device.
template <auto Kern>
cudaError_t prep(size_t smem) {
  static unsigned long long done = 0ull;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done & bit)) {
    e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    done |= bit;
  }
  return cudaSuccess;
}

template <int P, int Q, typename T, typename TV, int LAYOUT>
cudaError_t apply_launch(const OpArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_for(Q);
  const int threads = Q * Q * EPB;
  const int64_t blocks = (A.ne + EPB - 1) / EPB;
  if (blocks == 0) return cudaSuccess;
  const size_t smem = (size_t)EPB * elem_stride<Q, T>() * sizeof(T);
  const KTab<P, Q, T> tab = make_ktab<P, Q, T>(*A.tab);
  if (A.colour >= 0) {
    const int px = A.colour & 1, py = (A.colour >> 1) & 1, pz = A.colour >> 2;
    const int64_t ncol = (int64_t)((A.nx - px + 1) / 2) * ((A.ny - py + 1) / 2) * ((A.nz - pz + 1) / 2);
    const int64_t grid = (ncol + EPB - 1) / EPB;
    if (grid == 0) return cudaSuccess;
    cudaError_t e = prep<k_jacobian_apply<P, Q, T, TV, LAYOUT, true>>(smem);
    if (e != cudaSuccess) return e;
    k_jacobian_apply<P, Q, T, TV, LAYOUT, true><<<(unsigned)grid, threads, smem, s>>>(
        A.ne, A.emap, A.bc, (const T*)A.qd, A.qstride, tab, (const TV*)A.in, (TV*)A.out, A.lift, A.colour, A.nx, A.ny,
        A.nz);
    return cudaGetLastError();
  }
  cudaError_t e = prep<k_jacobian_apply<P, Q, T, TV, LAYOUT>>(smem);
  if (e != cudaSuccess) return e;
  k_jacobian_apply<P, Q, T, TV, LAYOUT><<<(unsigned)blocks, threads, smem, s>>>(
      A.ne, A.emap, A.bc, (const T*)A.qd, A.qstride, tab, (const TV*)A.in, (TV*)A.out, A.lift, -1, A.nx, A.ny, A.nz);
  return cudaGetLastError();
}

template <int P, int Q, int LAYOUT>
cudaError_t apply_ffr_launch(const OpArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_for(Q);
  const int threads = Q * Q * EPB;
  const int64_t blocks = (A.ne + EPB - 1) / EPB;
  if (blocks == 0) return cudaSuccess;
  const size_t smem = (size_t)EPB * ffr_stride<Q>() * sizeof(ff);
  const KTab<P, Q, ff> tab = make_ktab<P, Q, ff>(*A.tab);
  if (A.colour >= 0) {
    const int px = A.colour & 1, py = (A.colour >> 1) & 1, pz = A.colour >> 2;
    const int64_t ncol = (int64_t)((A.nx - px + 1) / 2) * ((A.ny - py + 1) / 2) * ((A.nz - pz + 1) / 2);
    const int64_t grid = (ncol + EPB - 1) / EPB;
    if (grid == 0) return cudaSuccess;
    cudaError_t e = prep<k_jacobian_apply_ffr<P, Q, LAYOUT, true>>(smem);
    if (e != cudaSuccess) return e;
    k_jacobian_apply_ffr<P, Q, LAYOUT, true><<<(unsigned)grid, threads, smem, s>>>(
        A.ne, A.emap, A.bc, (const ff*)A.qd, A.qstride, tab, (const double*)A.in, (double*)A.out, A.lift, A.colour,
        A.nx, A.ny, A.nz);
    return cudaGetLastError();
  }
  cudaError_t e = prep<k_jacobian_apply_ffr<P, Q, LAYOUT>>(smem);
  if (e != cudaSuccess) return e;
  k_jacobian_apply_ffr<P, Q, LAYOUT><<<(unsigned)blocks, threads, smem, s>>>(
      A.ne, A.emap, A.bc, (const ff*)A.qd, A.qstride, tab, (const double*)A.in, (double*)A.out, A.lift, -1, A.nx,
      A.ny, A.nz);
  return cudaGetLastError();
}

template <int P, int Q, int LAYOUT>
cudaError_t apply_f32l_launch(const OpArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_for(Q), S = nh_layout_scalars(LAYOUT);
  const int threads = Q * Q * EPB;
  const int64_t blocks = (A.ne + EPB - 1) / EPB;
  if (blocks == 0) return cudaSuccess;
  const size_t smem = ((nh_f32_direct(Q) ? 0 : (size_t)2 * nh_f32_plane_floats(Q, S)) +
                       (size_t)LineLayout<Q>::block_floats(EPB)) * sizeof(float);
  const KTab<P, Q, float> tab = make_ktab<P, Q, float>(*A.tab);
  const int nbx = A.nx > 0 ? A.nx / EPB : 0;
  if (A.colour >= 0) {  // batches must tile the rows: one block's elements lie in one row
    if (A.nx <= 0 || A.nx % EPB != 0 || ((uintptr_t)A.out & 15) != 0) return cudaErrorInvalidValue;
    const int px = A.colour & 1, py = (A.colour >> 1) & 1, pz = A.colour >> 2;
    const int64_t grid = (int64_t)((nbx - px + 1) / 2) * ((A.ny - py + 1) / 2) * ((A.nz - pz + 1) / 2);
    if (grid == 0) return cudaSuccess;
    constexpr auto kern = k_jacobian_apply_f32l<P, Q, LAYOUT, true>;
    cudaError_t e = prep<kern>(smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, threads, smem, s>>>(
        A.ne, A.emapb, (const float*)A.qd, tab, (const float*)A.in, (float*)A.out, A.lift,
        1 | (((uintptr_t)A.in & 15) == 0 ? 2 : 0), 1, A.err, A.colour, nbx,
        A.ny, A.nz);
    return cudaGetLastError();
  }
  constexpr auto kern = k_jacobian_apply_f32l<P, Q, LAYOUT, false>;
  cudaError_t e = prep<kern>(smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, threads, smem, s>>>(
      A.ne, A.emapb, (const float*)A.qd, tab, (const float*)A.in, (float*)A.out, A.lift,
      (((uintptr_t)A.out & 15) == 0 ? 1 : 0) | (((uintptr_t)A.in & 15) == 0 ? 2 : 0),
      ((uintptr_t)A.out & 15) == 0 && A.nx > 0 && (NH_F32_ROWS_ANY || Q <= 3 || A.nx % EPB == 0) ? 1 : 0, A.err,
      -1, nbx, A.ny, A.nz);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t apply_pq(nh_prec prec, const OpArgs& A, cudaStream_t s) {
  if (prec == NH_F64)
    return A.layout == NH_LAYOUT_CURRENT   ? apply_launch<P, Q, double, double, NH_LAYOUT_CURRENT>(A, s)
           : A.layout == NH_LAYOUT_INITIAL ? apply_launch<P, Q, double, double, NH_LAYOUT_INITIAL>(A, s)
                                           : apply_launch<P, Q, double, double, NH_LAYOUT_TAPE>(A, s);
  if (prec == NH_F64X && NH_FF_ROLLED)
    return A.layout == NH_LAYOUT_CURRENT   ? apply_ffr_launch<P, Q, NH_LAYOUT_CURRENT>(A, s)
           : A.layout == NH_LAYOUT_INITIAL ? apply_ffr_launch<P, Q, NH_LAYOUT_INITIAL>(A, s)
                                           : apply_ffr_launch<P, Q, NH_LAYOUT_TAPE>(A, s);
  if (prec == NH_F64X)
    return A.layout == NH_LAYOUT_CURRENT   ? apply_launch<P, Q, ff, double, NH_LAYOUT_CURRENT>(A, s)
           : A.layout == NH_LAYOUT_INITIAL ? apply_launch<P, Q, ff, double, NH_LAYOUT_INITIAL>(A, s)
                                           : apply_launch<P, Q, ff, double, NH_LAYOUT_TAPE>(A, s);
  return A.layout == NH_LAYOUT_CURRENT   ? apply_f32l_launch<P, Q, NH_LAYOUT_CURRENT>(A, s)
         : A.layout == NH_LAYOUT_INITIAL ? apply_f32l_launch<P, Q, NH_LAYOUT_INITIAL>(A, s)
                                         : apply_f32l_launch<P, Q, NH_LAYOUT_TAPE>(A, s);
}

template <int P, int Q, int LAYOUT, int GEOM>
cudaError_t setup_go(const OpArgs& A, const SetupTab<P, Q>& st, int64_t blocks, int threads, size_t smem,
                     cudaStream_t s) {
  cudaError_t e = prep<k_setup<P, Q, LAYOUT, GEOM>>(smem);
  if (e != cudaSuccess) return e;
  k_setup<P, Q, LAYOUT, GEOM><<<(unsigned)blocks, threads, smem, s>>>(
      A.ne, A.emap, A.bc, A.coords, (const double*)A.in, A.lam, A.mu, st, A.qd_out, A.qstride, A.store, A.resid, A.gbc,
      (double*)A.out, A.minj, A.geom);
  return cudaGetLastError();
}

template <int P, int Q, int LAYOUT>
cudaError_t setup_launch(const OpArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_for(Q), Q3 = Q * Q * Q;
  const int threads = Q * Q * EPB;
  const int64_t blocks = (A.ne + EPB - 1) / EPB;
  if (blocks == 0) return cudaSuccess;
  const size_t smem = (size_t)EPB * 12 * Q3 * sizeof(double);
  SetupTab<P, Q> st;
  st.k = make_ktab<P, Q, double>(*A.tab);
  for (int i = 0; i < Q; i++) st.w[i] = A.tab->w[i];
  const int mode = A.geom ? A.geom_mode : 0;
  return mode == 2   ? setup_go<P, Q, LAYOUT, 2>(A, st, blocks, threads, smem, s)
         : mode == 1 ? setup_go<P, Q, LAYOUT, 1>(A, st, blocks, threads, smem, s)
                     : setup_go<P, Q, LAYOUT, 0>(A, st, blocks, threads, smem, s);
}

template <int P, int Q>
cudaError_t setup_pq(const OpArgs& A, cudaStream_t s) {
  return A.layout == NH_LAYOUT_CURRENT   ? setup_launch<P, Q, NH_LAYOUT_CURRENT>(A, s)
         : A.layout == NH_LAYOUT_INITIAL ? setup_launch<P, Q, NH_LAYOUT_INITIAL>(A, s)
                                         : setup_launch<P, Q, NH_LAYOUT_TAPE>(A, s);
}

template <int P, int Q, int LAYOUT, typename TO>
cudaError_t diag_launch(const OpArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_for(Q), Q3 = Q * Q * Q;
  const int threads = Q * Q * EPB;
  const int64_t blocks = (A.ne + EPB - 1) / EPB;
  if (blocks == 0) return cudaSuccess;
  const size_t smem = (size_t)EPB * 11 * Q3 * sizeof(TO);
  DiagTab<P, Q, TO> dt;
  for (int i = 0; i < Q; i++)
    for (int j = 0; j < P; j++) {
      dt.BB[i][j] = A.tab->B[i][j] * A.tab->B[i][j];
      dt.BG[i][j] = A.tab->B[i][j] * A.tab->G[i][j];
      dt.GG[i][j] = A.tab->G[i][j] * A.tab->G[i][j];
    }
  cudaError_t e = prep<k_diagonal<P, Q, LAYOUT, TO>>(smem);
  if (e != cudaSuccess) return e;
  k_diagonal<P, Q, LAYOUT, TO><<<(unsigned)blocks, threads, smem, s>>>(A.ne, A.emap, A.bc, (const double*)A.qd,
                                                                       A.qstride, dt, (TO*)A.out);
  return cudaGetLastError();
}

template <int P, int Q>
cudaError_t diag_pq(nh_prec prec, const OpArgs& A, cudaStream_t s) {
  if (A.layout == NH_LAYOUT_CURRENT)
    return prec == NH_F64 ? diag_launch<P, Q, NH_LAYOUT_CURRENT, double>(A, s)
                          : diag_launch<P, Q, NH_LAYOUT_CURRENT, float>(A, s);
  if (A.layout == NH_LAYOUT_INITIAL)
    return prec == NH_F64 ? diag_launch<P, Q, NH_LAYOUT_INITIAL, double>(A, s)
                          : diag_launch<P, Q, NH_LAYOUT_INITIAL, float>(A, s);
  return prec == NH_F64 ? diag_launch<P, Q, NH_LAYOUT_TAPE, double>(A, s)
                        : diag_launch<P, Q, NH_LAYOUT_TAPE, float>(A, s);
}

}  // namespace

#if NH_P_INST == 2
cudaError_t nh_launch_wait_timeout_mbar(cudaStream_t s, int* err) {
  k_wait_timeout_mbar<<<1, 32, 0, s>>>(err, 1u << 12);
  return cudaGetLastError();
}
#endif

#define NH_CAT2(a, b) a##b
#define NH_CAT(a, b) NH_CAT2(a, b)
#define PI NH_P_INST
// Q >= P always holds in the instantiated set: out-of-range cases are never taken.
#define QQ(v) ((v) < PI ? PI : (v))

#define NH_QCASES(FN, ...)                                      \
  switch (Q) {                                                  \
    case 2: if (PI <= 2) return FN<PI, QQ(2)>(__VA_ARGS__); break; \
    case 3: if (PI <= 3) return FN<PI, QQ(3)>(__VA_ARGS__); break; \
    case 4: if (PI <= 4) return FN<PI, QQ(4)>(__VA_ARGS__); break; \
    case 5: if (PI <= 5) return FN<PI, QQ(5)>(__VA_ARGS__); break; \
    case 6: return FN<PI, 6>(__VA_ARGS__);                      \
    default: break;                                             \
  }                                                             \
  return cudaErrorInvalidValue;

cudaError_t NH_CAT(nh_launch_apply_P, NH_P_INST)(int Q, nh_prec prec, const OpArgs& a, cudaStream_t s) {
  NH_QCASES(apply_pq, prec, a, s)
}
cudaError_t NH_CAT(nh_launch_setup_P, NH_P_INST)(int Q, const OpArgs& a, cudaStream_t s) {
  NH_QCASES(setup_pq, a, s)
}
cudaError_t NH_CAT(nh_launch_diag_P, NH_P_INST)(int Q, const OpArgs& a, cudaStream_t s) {
  NH_QCASES(diag_pq, (nh_prec)a.prec, a, s)
}

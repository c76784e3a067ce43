// Vector kernels for the Krylov solvers and smoothers (Sec. III-A, III-B).
// Scalars that come out of a dot product stay on the device (slots of a small
// scalar array) and are read by the update kernels directly, so a CG or FCG
// step needs no host round trip; the host reads a norm only when it tests
// convergence.  Dot products accumulate in FP64 whatever the vector type, with
// a fixed grid and a fixed-order final sum (deterministic).
#include "nh_krylov.cuh"

namespace {

constexpr int kT = 256;

inline int grid_for(int64_t n) {
  int64_t b = (n + kT - 1) / kT;
  if (b > 148 * 8) b = 148 * 8;
  return b < 1 ? 1 : (int)b;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

template <typename T>
__global__ void k_axpby(int64_t n, double a, const T* __restrict__ x, double b, T* __restrict__ y) {
  if (b == 0.0) {  // y is not read: it may hold anything
    GRID_STRIDE(i, n) y[i] = (T)(a * (double)x[i]);
  } else {
    GRID_STRIDE(i, n) y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
  }
}

// y += s * (sc[num] / sc[den]) * x
template <typename T>
__global__ void k_axpy_dev(int64_t n, const T* __restrict__ x, T* __restrict__ y, const double* __restrict__ sc,
                           int num, int den, double s) {
  const double a = s * sc[num] / sc[den];
  GRID_STRIDE(i, n) y[i] = (T)((double)y[i] + a * (double)x[i]);
}

// x += a p ; r -= a q   with a = sc[num] / sc[den]
template <typename T>
__global__ void k_cg_update(int64_t n, const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ x,
                            T* __restrict__ r, const double* __restrict__ sc, int num, int den) {
  const double a = sc[num] / sc[den];
  GRID_STRIDE(i, n) {
    x[i] = (T)((double)x[i] + a * (double)p[i]);
    r[i] = (T)((double)r[i] - a * (double)q[i]);
  }
}

// p = z + s * (sc[num] / sc[den]) * p
template <typename T>
__global__ void k_xpby_dev(int64_t n, const T* __restrict__ z, T* __restrict__ p, const double* __restrict__ sc,
                           int num, int den, double s) {
  const double b = s * sc[num] / sc[den];
  GRID_STRIDE(i, n) p[i] = (T)((double)z[i] + b * (double)p[i]);
}

template <typename T>
__global__ void k_mul(int64_t n, const T* __restrict__ d, const T* __restrict__ x, T* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] = d[i] * x[i];
}

template <typename T>
__global__ void k_recip(int64_t n, T* __restrict__ d) {
  GRID_STRIDE(i, n) d[i] = T(1) / d[i];
}

template <typename TI, typename TO>
__global__ void k_convert(int64_t n, const TI* __restrict__ x, TO* __restrict__ y) {
  GRID_STRIDE(i, n) y[i] = (TO)x[i];
}

template <typename T>
__global__ void k_mask_zero(int64_t nn, const uint8_t* __restrict__ bc, T* __restrict__ v) {
  GRID_STRIDE(i, nn) {
    const unsigned m = bc[i];
    if (m) {
      if (m & 1u) v[3 * i] = T(0);
      if (m & 2u) v[3 * i + 1] = T(0);
      if (m & 4u) v[3 * i + 2] = T(0);
    }
  }
}

// unconstrained components of v are zeroed
template <typename T>
__global__ void k_mask_keep(int64_t nn, const uint8_t* __restrict__ bc, T* __restrict__ v) {
  GRID_STRIDE(i, nn) {
    const unsigned m = bc[i];
    for (int c = 0; c < 3; c++)
      if (!((m >> c) & 1u)) v[3 * i + c] = T(0);
  }
}

// constrained components of v take the values of g (scaled by s)
__global__ void k_lift(int64_t nn, const uint8_t* __restrict__ bc, double* __restrict__ v,
                       const double* __restrict__ g, double s) {
  GRID_STRIDE(i, nn) {
    const unsigned m = bc[i];
    for (int c = 0; c < 3; c++)
      if ((m >> c) & 1u) v[3 * i + c] = g ? s * g[3 * i + c] : 0.0;
  }
}

// Chebyshev step: d = c1 d + c2 dinv r ; x += d
template <typename T>
__global__ void k_cheb(int64_t n, double c1, double c2, const T* __restrict__ dinv, const T* __restrict__ r,
                       T* __restrict__ d, T* __restrict__ x) {
  GRID_STRIDE(i, n) {
    const double di = (c1 == 0.0 ? 0.0 : c1 * (double)d[i]) + c2 * (double)dinv[i] * (double)r[i];
    d[i] = (T)di;
    x[i] = (T)((double)x[i] + di);
  }
}

// splitmix64 (Steele, Lea, Flood 2014) on (seed, index) -> uniform(-1, 1)
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_uniform(int64_t n, uint64_t seed, double* __restrict__ v) {
  GRID_STRIDE(i, n) {
    const uint64_t z = splitmix64(seed * 0x100000001b3ull + (uint64_t)i);
    v[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    v = warp_sum(v);
  }
  return v;
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(kT)
    k_dotp(int64_t n, const TA* __restrict__ x, const TB* __restrict__ y, double* __restrict__ part) {
  double s = 0.0;
  GRID_STRIDE(i, n) s = fma((double)x[i], (double)y[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_dotf(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// out[j] partials of W_j . v: block (c, j) sums chunk c of row j (rows of length n,
// stride ldw); chunks of a row are summed afterwards in a fixed order
constexpr int kMdChunks = 64;
__global__ void __launch_bounds__(256)
    k_multidot_part(int64_t n, const double* __restrict__ W, int64_t ldw, const double* __restrict__ v,
                    double* __restrict__ part) {
  const int j = blockIdx.y, c = blockIdx.x;
  const int64_t len = (n + kMdChunks - 1) / kMdChunks, i0 = c * len, i1 = i0 + len < n ? i0 + len : n;
  const double* w = W + (int64_t)j * ldw;
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(w[i], v[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[(int64_t)j * kMdChunks + c] = s;
}

__global__ void k_multidot_fin(int k, const double* __restrict__ part, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int c = 0; c < kMdChunks; c++) s += part[(int64_t)j * kMdChunks + c];
  out[j] = s;
}

// y[i] += alpha sum_j c[j] W[j][i], k <= 256
__global__ void k_gemv_rows(int64_t n, int k, const double* __restrict__ W, int64_t ldw, const double* __restrict__ c,
                            double alpha, double* __restrict__ y) {
  __shared__ double cs[256];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = alpha * c[j];
  __syncthreads();
  GRID_STRIDE(i, n) {
    double s = 0.0;
    for (int j = 0; j < k; j++) s = fma(cs[j], W[(int64_t)j * ldw + i], s);
    y[i] += s;
  }
}

}  // namespace

// ---- launchers -------------------------------------------------------------------
cudaError_t kv_multidot(cudaStream_t st, int k, int64_t n, const double* W, int64_t ldw, const double* v,
                        double* part, double* out) {
  if (k <= 0) return cudaSuccess;
  k_multidot_part<<<dim3(kMdChunks, k), 256, 0, st>>>(n, W, ldw, v, part);
  k_multidot_fin<<<(k + 127) / 128, 128, 0, st>>>(k, part, out);
  return cudaGetLastError();
}
int kv_multidot_parts() { return kMdChunks; }
cudaError_t kv_gemv_rows(cudaStream_t st, int64_t n, int k, const double* W, int64_t ldw, const double* c,
                         double alpha, double* y) {
  if (k <= 0) return cudaSuccess;
  if (k > 256) return cudaErrorInvalidValue;
  k_gemv_rows<<<grid_for(n), kT, 0, st>>>(n, k, W, ldw, c, alpha, y);
  return cudaGetLastError();
}
#define L1(k, n, ...)                                     \
  do {                                                    \
    k<<<grid_for(n), kT, 0, st>>>(n, __VA_ARGS__);        \
    return cudaGetLastError();                            \
  } while (0)

template <typename T>
cudaError_t kv_axpby(cudaStream_t st, int64_t n, double a, const T* x, double b, T* y) { L1(k_axpby<T>, n, a, x, b, y); }
template <typename T>
cudaError_t kv_axpy_dev(cudaStream_t st, int64_t n, const T* x, T* y, const double* sc, int num, int den, double s) {
  L1(k_axpy_dev<T>, n, x, y, sc, num, den, s);
}
template <typename T>
cudaError_t kv_cg_update(cudaStream_t st, int64_t n, const T* p, const T* q, T* x, T* r, const double* sc, int num,
                         int den) {
  L1(k_cg_update<T>, n, p, q, x, r, sc, num, den);
}
template <typename T>
cudaError_t kv_xpby_dev(cudaStream_t st, int64_t n, const T* z, T* p, const double* sc, int num, int den, double s) {
  L1(k_xpby_dev<T>, n, z, p, sc, num, den, s);
}
template <typename T>
cudaError_t kv_mul(cudaStream_t st, int64_t n, const T* d, const T* x, T* y) { L1(k_mul<T>, n, d, x, y); }
template <typename T>
cudaError_t kv_recip(cudaStream_t st, int64_t n, T* d) { L1(k_recip<T>, n, d); }
template <typename TI, typename TO>
cudaError_t kv_convert(cudaStream_t st, int64_t n, const TI* x, TO* y) { L1((k_convert<TI, TO>), n, x, y); }
template <typename T>
cudaError_t kv_mask_zero(cudaStream_t st, int64_t nn, const uint8_t* bc, T* v) { L1(k_mask_zero<T>, nn, bc, v); }
cudaError_t kv_mask_keep(cudaStream_t st, int64_t nn, const uint8_t* bc, double* v) {
  L1(k_mask_keep<double>, nn, bc, v);
}
cudaError_t kv_lift(cudaStream_t st, int64_t nn, const uint8_t* bc, double* v, const double* g, double s) {
  L1(k_lift, nn, bc, v, g, s);
}
template <typename T>
cudaError_t kv_cheb(cudaStream_t st, int64_t n, double c1, double c2, const T* dinv, const T* r, T* d, T* x) {
  L1(k_cheb<T>, n, c1, c2, dinv, r, d, x);
}
cudaError_t kv_uniform(cudaStream_t st, int64_t n, uint64_t seed, double* v) { L1(k_uniform, n, seed, v); }

template <typename TA, typename TB>
cudaError_t kv_dot(cudaStream_t st, int64_t n, const TA* x, const TB* y, double* part, double* out) {
  const int nb = grid_for(n);
  k_dotp<TA, TB><<<nb, kT, 0, st>>>(n, x, y, part);
  k_dotf<<<1, 1024, 0, st>>>(part, nb, out);
  return cudaGetLastError();
}

#define INST(T)                                                                                            \
  template cudaError_t kv_axpby<T>(cudaStream_t, int64_t, double, const T*, double, T*);                  \
  template cudaError_t kv_axpy_dev<T>(cudaStream_t, int64_t, const T*, T*, const double*, int, int, double); \
  template cudaError_t kv_cg_update<T>(cudaStream_t, int64_t, const T*, const T*, T*, T*, const double*, int, int); \
  template cudaError_t kv_xpby_dev<T>(cudaStream_t, int64_t, const T*, T*, const double*, int, int, double); \
  template cudaError_t kv_mul<T>(cudaStream_t, int64_t, const T*, const T*, T*);                          \
  template cudaError_t kv_recip<T>(cudaStream_t, int64_t, T*);                                            \
  template cudaError_t kv_mask_zero<T>(cudaStream_t, int64_t, const uint8_t*, T*);                        \
  template cudaError_t kv_cheb<T>(cudaStream_t, int64_t, double, double, const T*, const T*, T*, T*);
INST(double)
INST(float)
template cudaError_t kv_convert<double, float>(cudaStream_t, int64_t, const double*, float*);
template cudaError_t kv_convert<float, double>(cudaStream_t, int64_t, const float*, double*);
template cudaError_t kv_dot<double, double>(cudaStream_t, int64_t, const double*, const double*, double*, double*);
template cudaError_t kv_dot<float, float>(cudaStream_t, int64_t, const float*, const float*, double*, double*);

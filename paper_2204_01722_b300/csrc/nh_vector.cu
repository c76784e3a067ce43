// Vector kernels: deterministic FP64 dot products (fixed grid, per-block
// partial sums, then one fixed-order pass, so results do not depend on timing)
// and precision conversion.
#include "nh_internal.cuh"
#include "nh_ff.cuh"

namespace {

constexpr int kDotThreads = 256;

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
  return v;  // valid in thread 0
}

__global__ void __launch_bounds__(kDotThreads)
    k_dot_partials(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                   double* __restrict__ partials) {
  double s = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s = fma(x[i], y[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ p, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += p[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (float)x[i];
}

// FP32 quadrature data per batch of EPB elements as Q z-planes (one bulk copy
// each), points in the order of the z-line threads of a block, scalars in
// rotated 16-byte chunks plus a remainder array (see nh_f32_plane_floats).
__global__ void k_f32_blocked(int Q, int EPB, int S, long long PL, int64_t ne, const double* __restrict__ qd,
                              float* __restrict__ qdf) {
  const int Q2 = Q * Q, Q3 = Q2 * Q, NP = EPB * Q2, NC = S / 4, R = S - 4 * NC;
  const int64_t n = (int64_t)S * ne * Q3;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int s = (int)(i / (ne * Q3));
    const int64_t r = i - s * ne * Q3, e = r / Q3;
    const int q = (int)(r - e * Q3), qz = q / Q2, p = (int)(e % EPB) * Q2 + (q - qz * Q2);
    const int64_t pos = nh_f32_direct(Q) ? (int64_t)s * nh_f32_npp(Q) + p
                        : s < 4 * NC ? (int64_t)p * 4 * NC + (((s >> 2) + nh_f32_rot(S, p)) % NC) * 4 + (s & 3)
                                     : (int64_t)NP * 4 * NC + (int64_t)p * R + (s - 4 * NC);
    qdf[((e / EPB) * Q + qz) * PL + pos] = (float)qd[i];
  }
}

__global__ void k_f64_to_ff(int64_t n, const double* __restrict__ x, ff* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = ff(x[i]);
}

__global__ void k_pack_emap(int64_t n, const int* __restrict__ emap, const uint8_t* __restrict__ bc,
                            unsigned* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int node = emap[i];
    out[i] = (unsigned)node | ((unsigned)(bc[node] & 7u) << 29);
  }
}

}  // namespace

cudaError_t nh_launch_pack_emap(cudaStream_t s, int64_t n, const int* emap, const uint8_t* bc, unsigned* out) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_pack_emap<<<(unsigned)blocks, 256, 0, s>>>(n, emap, bc, out);
  return cudaGetLastError();
}

cudaError_t nh_launch_f64_to_ff(int64_t n, const double* x, float* y2, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_f64_to_ff<<<(unsigned)blocks, 256, 0, s>>>(n, x, reinterpret_cast<ff*>(y2));
  return cudaGetLastError();
}

cudaError_t nh_launch_f32_blocked(int Q, int S, int64_t ne, const double* qd, float* qdf, cudaStream_t s) {
  const int64_t n = (int64_t)S * ne * Q * Q * Q;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_f32_blocked<<<(unsigned)blocks, 256, 0, s>>>(Q, nh_epb(Q), S, nh_f32_plane_floats(Q, S), ne, qd, qdf);
  return cudaGetLastError();
}

cudaError_t nh_launch_dot_partials(int64_t n, const double* x, const double* y, double* partials, int nblocks,
                                   cudaStream_t s) {
  k_dot_partials<<<nblocks, kDotThreads, 0, s>>>(n, x, y, partials);
  return cudaGetLastError();
}

cudaError_t nh_launch_sum_partials(const double* partials, int nblocks, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 1024, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

cudaError_t nh_launch_f64_to_f32(int64_t n, const double* x, float* y, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_f64_to_f32<<<(unsigned)blocks, 256, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

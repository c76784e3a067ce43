// Allocation-free deterministic FP64 dot product (nh_dot_noalloc).
//
// Some callers cannot let a library call cudaMalloc: applications whose device
// memory is owned by their own pool allocator (an allocation behind its back
// breaks its budget or fails outright), and latency-critical loops in which a
// cudaMalloc/cudaFree would synchronise the whole device.  This entry point
// gives them the dot product without any allocation and without an nh_ctx:
// the scratch it needs lives in a fixed array in the library's device image.
//
// Algorithm: one partial sum per chunk of kChunk consecutive elements (one
// block per chunk), then one block adds the partials in a fixed order, so the
// rounding depends only on n.  The partials live in g_dot_scratch, which
// every GPU that loads the library holds until the process exits.
#include <mutex>

#include "nh_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 8192;                       // elements per partial sum
constexpr int kMaxPartials = 32768;                    // scratch capacity
static_assert(NH_DOT_NOALLOC_MAX_N == kChunk * kMaxPartials, "limit must match the scratch size");

// The scratch: partial sums, then one slot kept free, 256-byte aligned.  In
// host code this name is only a stand-in for the device symbol; kernels get
// the device address looked up with cudaGetSymbolAddress.
static __device__ __align__(256) double g_dot_scratch[kMaxPartials + 32];

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

// Block b sums x[i] y[i] over i in [b kChunk, min(n, (b+1) kChunk)).
__global__ void __launch_bounds__(kThreads)
    k_dot_chunks(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                 double* __restrict__ partials) {
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int64_t end = base + kChunk < n ? base + kChunk : n;
  double s = 0.0;
  for (int64_t i = base + threadIdx.x; i < end; i += kThreads) s = fma(x[i], y[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One block: out = sum of partials[0 .. nb) in a fixed order (nb = 0 gives 0).
__global__ void __launch_bounds__(1024)
    k_sum_chunks(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// Device address of g_dot_scratch, looked up once per device with that device current.
std::mutex g_lock;
double* g_addr[64] = {nullptr};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" nh_status nh_dot_noalloc(void* cuda_stream, int64_t n, const double* x, const double* y,
                                    double* result) {
  if (n < 0 || !result) return NH_ERR_ARG;
  if (n > 0 && (!x || !y)) return NH_ERR_ARG;
  if (((uintptr_t)result % 8) || ((uintptr_t)x % 8) || ((uintptr_t)y % 8)) return NH_ERR_ARG;
  if (n > NH_DOT_NOALLOC_MAX_N) return NH_ERR_UNSUPPORTED;  // more partial sums than the scratch holds
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return NH_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nb = (int)((n + kChunk - 1) / kChunk);
  // Every partial slot that k_sum_chunks reads is written by k_dot_chunks of the
  // same call, so nothing left by an earlier call needs clearing.
  if (nb > 0) k_dot_chunks<<<nb, kThreads, 0, s>>>(n, x, y, scratch);
  k_sum_chunks<<<1, 1024, 0, s>>>(scratch, nb, result);
  return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

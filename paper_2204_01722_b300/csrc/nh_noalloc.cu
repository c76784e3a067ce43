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

// Device address of g_dot_scratch.  The address belongs to a CUDA context, not
// to a device number: after cudaDeviceReset the primary context is new and the
// module is loaded again, and a driver-API context of its own on the same device
// holds another copy.  So the lookup is cached per context, keyed by the
// driver's context id (unique within the process, never reused), and redone for
// every context met.  The two driver calls are reached through the runtime's
// entry-point query, so the library does not link libcuda.  When they cannot be
// had, or the cache is full, the address is looked up on every call.
typedef int (*ctx_get_current_fn)(void** ctx);
typedef int (*ctx_get_id_fn)(void* ctx, unsigned long long* id);

struct Slot {
  unsigned long long ctx_id;
  double* addr;
};

std::mutex g_lock;
bool g_fns_queried = false;
ctx_get_current_fn g_get_current = nullptr;
ctx_get_id_fn g_get_id = nullptr;
constexpr int kSlots = 64;
Slot g_slots[kSlots];
int g_nslots = 0;

cudaError_t lookup_symbol(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// Id of the context current on this thread, or false if it cannot be had.
bool current_ctx_id(unsigned long long* id) {
  if (!g_get_current || !g_get_id) return false;
  void* ctx = nullptr;
  if (g_get_current(&ctx) != 0 || !ctx) return false;
  return g_get_id(ctx, id) == 0;
}

cudaError_t scratch_for_current_context(double** out) {
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_fns_queried) {
    g_fns_queried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_get_current = reinterpret_cast<ctx_get_current_fn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_get_id = reinterpret_cast<ctx_get_id_fn>(f);
  }
  unsigned long long id = 0;
  if (!current_ctx_id(&id)) {
    // No context current yet (the runtime makes the primary one on its first
    // call that needs it): look up, which creates it, then try the id again.
    double* addr = nullptr;
    const cudaError_t e = lookup_symbol(&addr);
    if (e != cudaSuccess) return e;
    *out = addr;
    if (!current_ctx_id(&id)) return cudaSuccess;
    if (g_nslots < kSlots) g_slots[g_nslots++] = Slot{id, addr};
    return cudaSuccess;
  }
  for (int i = 0; i < g_nslots; ++i)
    if (g_slots[i].ctx_id == id) {
      *out = g_slots[i].addr;
      return cudaSuccess;
    }
  double* addr = nullptr;
  const cudaError_t e = lookup_symbol(&addr);
  if (e != cudaSuccess) return e;
  if (g_nslots < kSlots) g_slots[g_nslots++] = Slot{id, addr};
  *out = addr;
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
  if (scratch_for_current_context(&scratch) != cudaSuccess) return NH_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int nb = (int)((n + kChunk - 1) / kChunk);
  // Every partial slot that k_sum_chunks reads is written by k_dot_chunks of the
  // same call, so nothing left by an earlier call needs clearing.  Each launch's
  // own status is taken from cudaLaunchKernel, so an error left pending by
  // unrelated earlier work is neither reported here nor cleared.
  if (nb > 0) {
    void* args[] = {&n, (void*)&x, (void*)&y, &scratch};
    const cudaError_t e = cudaLaunchKernel((const void*)k_dot_chunks, dim3(nb), dim3(kThreads), args, 0, s);
    if (e != cudaSuccess) return NH_ERR_CUDA;
  }
  void* args2[] = {&scratch, &nb, &result};
  const cudaError_t e = cudaLaunchKernel((const void*)k_sum_chunks, dim3(1), dim3(1024), args2, 0, s);
  return e == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

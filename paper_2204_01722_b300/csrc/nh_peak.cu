// Measured arithmetic peaks (nh_fma_peak): the FP64 and FP32 fused multiply-add
// throughput of this GPU, the denominators of the ALU rooflines of the FP64 and
// float-float Jacobian applies.  Not part of the method.
//
// Every thread runs kChains independent FMA chains x <- x * a + c for `iters`
// steps (a just below 1, c small, so the values stay finite and no step can
// be removed), then stores their sum.  The grid fills every SM with 8 resident
// blocks of 256 threads; work = 2 kChains iters threads flops.
#include "nh_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int64_t iters, T a, T c, T* __restrict__ out) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) x[j] = (T)(threadIdx.x + j);
  for (int64_t i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) x[j] = fma(x[j], a, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += x[j];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" nh_status nh_fma_peak(nh_ctx ctx, nh_prec prec, int64_t iters, double* tflops, double* ms) {
  if (!ctx || !tflops || iters < 1 || (prec != NH_F64 && prec != NH_F32)) return NH_ERR_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return nh_cuda_check(ctx, e, "cudaSetDevice");
  const int blocks = ctx->num_sms * 8;
  const size_t bytes = (size_t)blocks * kThreads * 8;
  void* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMalloc(&out, bytes)) != cudaSuccess) return nh_cuda_check(ctx, e, "cudaMalloc");
  nh_status st = NH_OK;
  float t = 0.f;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = nh_cuda_check(ctx, e, "cudaEventCreate");
  } else {
    for (int rep = 0; rep < 2 && st == NH_OK; rep++) {  // the first launch is a warm-up
      cudaEventRecord(e0, ctx->stream);
      if (prec == NH_F64)
        k_fma_chains<double><<<blocks, kThreads, 0, ctx->stream>>>(iters, 0.999999999, 1e-9, (double*)out);
      else
        k_fma_chains<float><<<blocks, kThreads, 0, ctx->stream>>>(iters, 0.9999f, 1e-4f, (float*)out);
      cudaEventRecord(e1, ctx->stream);
      ctx->launches++;
      if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess)
        st = nh_cuda_check(ctx, e, "nh_fma_peak");
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != NH_OK) return st;
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return NH_OK;
}

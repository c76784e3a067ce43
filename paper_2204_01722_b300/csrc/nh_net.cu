// Learned coarse correction: a small 3-D convolution U-Net on the Q1 vertex
// grid, with hand-written forward and backward kernels (activations and
// weights in BF16 -- or FP32 for verification -- accumulation in FP32) and an
// Adam optimiser on FP32 master weights.  The paper has no learned component;
// the network is an extra preconditioner stage in flexible CG.
//
// Fields are channel-major [C][Nz][Ny][Nx] on an odd vertex grid N; a stride-2
// convolution maps N nodes to (N - 1) / 2 + 1 (vertex-centred), upsampling maps
// M to 2M - 1 by linear interpolation.  Network (levels L, channels c_l):
//   h = relu(conv(x, 4 -> c0)); s_0 = h = relu(conv(h, c0 -> c0))
//   l = 1..L-1: h = relu(conv_s2(h)); s_l = h = relu(conv(h))
//   l = L-2..0: h = relu(conv(up(h), c_{l+1} -> c_l)) + s_l; h = relu(conv(h))
//   y = conv(h, c0 -> 3)
// Parameters: layers in that order, each W [Cout][Cin][27] (tap = kx + 3 (ky + 3 kz))
// then b [Cout].
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "nh_net.cuh"

namespace {

constexpr int kCC = 4;  // input channels per shared-memory weight chunk

template <typename T>
__device__ __forceinline__ float tof(T v) { return (float)v; }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T fromf(float v) { return (T)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 fromf<__nv_bfloat16>(float v) { return __float2bfloat16(v); }

#define GSTRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

inline unsigned blocks_for(int64_t n, int t = 256) {
  int64_t b = (n + t - 1) / t;
  if (b > 148 * 32) b = 148 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---- forward convolution: one thread per output voxel, CO accumulators ----------
// y = act(conv(x) + b) (+ add); output to TA (yo) and/or FP32 (yf)
template <typename TA, int CO>
__global__ void __launch_bounds__(128)
    k_conv_fwd(const TA* __restrict__ x, int Cin, int Nin, const TA* __restrict__ W, const float* __restrict__ bias,
               int Nout, int stride, int relu, const TA* __restrict__ add, TA* __restrict__ yo, float* __restrict__ yf) {
  constexpr int COP = (CO + 3) / 4 * 4;
  __shared__ __align__(16) float ws[kCC][27][COP];
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = o < nout;
  const int oi = (int)(o % Nout), oj = (int)((o / Nout) % Nout), ok = (int)(o / ((int64_t)Nout * Nout));
  float acc[COP];
#pragma unroll
  for (int c = 0; c < COP; c++) acc[c] = 0.f;
  for (int c0 = 0; c0 < Cin; c0 += kCC) {
    __syncthreads();
    for (int t = threadIdx.x; t < kCC * 27 * COP; t += blockDim.x) {
      const int co = t % COP, tap = (t / COP) % 27, cil = t / (COP * 27);
      const int ci = c0 + cil;
      ws[cil][tap][co] = (co < CO && ci < Cin) ? tof(W[((int64_t)co * Cin + ci) * 27 + tap]) : 0.f;
    }
    __syncthreads();
    if (!live) continue;
    for (int cil = 0; cil < kCC && c0 + cil < Cin; cil++) {
      const TA* xc = x + (int64_t)(c0 + cil) * nin;
#pragma unroll
      for (int tap = 0; tap < 27; tap++) {
        const int ii = stride * oi + tap % 3 - 1, jj = stride * oj + (tap / 3) % 3 - 1, kk = stride * ok + tap / 9 - 1;
        float xv = 0.f;
        if (ii >= 0 && ii < Nin && jj >= 0 && jj < Nin && kk >= 0 && kk < Nin)
          xv = tof(xc[ii + (int64_t)Nin * (jj + (int64_t)Nin * kk)]);
        const float4* w4 = reinterpret_cast<const float4*>(&ws[cil][tap][0]);
#pragma unroll
        for (int c = 0; c < COP / 4; c++) {
          const float4 w = w4[c];
          acc[4 * c + 0] += w.x * xv;
          acc[4 * c + 1] += w.y * xv;
          acc[4 * c + 2] += w.z * xv;
          acc[4 * c + 3] += w.w * xv;
        }
      }
    }
  }
  if (!live) return;
#pragma unroll
  for (int c = 0; c < CO; c++) {
    float v = acc[c] + bias[c];
    if (relu) v = fmaxf(v, 0.f);
    if (yo) yo[(int64_t)c * nout + o] = fromf<TA>(v);  // stored activation: relu mask of the backward pass
    if (yf) yf[(int64_t)c * nout + o] = v + (add ? tof(add[(int64_t)c * nout + o]) : 0.f);
  }
}

// ---- forward convolution on the tensor cores (BF16 activations and weights) -----
// Implicit GEMM out[o][co] = sum_k A[o][k] B[k][co] over k = ci * 27 + tap, with
// A[o][k] = x[ci][neighbour(o, tap)] gathered (zero outside the grid) and
// B[k][co] = W[co][ci][tap], on mma.sync m16n8k16 (BF16 operands, FP32
// accumulation).  A warp owns 16 consecutive output voxels and all CO output
// channels (CO / 8 accumulator tiles); a block of 4 warps owns 64 voxels.  The
// gathered activations and the weights are read through the L1 cache (every warp
// of a block reads the same weights).  Same epilogue as k_conv_fwd.
__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

template <int CO>
__global__ void __launch_bounds__(128)
    k_conv_fwd_mma(const __nv_bfloat16* __restrict__ x, int Cin, int Nin, const __nv_bfloat16* __restrict__ W,
                   const float* __restrict__ bias, int Nout, int stride, int relu,
                   const __nv_bfloat16* __restrict__ add, __nv_bfloat16* __restrict__ yo, float* __restrict__ yf) {
  constexpr int NT = (CO + 7) / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t o0 = ((int64_t)blockIdx.x * 4 + warp) * 16;
  const int K = Cin * 27;
  // the two output voxels whose A rows this lane supplies (rows g and g + 8)
  int bi[2], bj[2], bk[2];
  bool ov[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int64_t o = o0 + g + 8 * r;
    ov[r] = o < nout;
    const int64_t oc = ov[r] ? o : 0;
    bi[r] = stride * (int)(oc % Nout) - 1;
    bj[r] = stride * (int)((oc / Nout) % Nout) - 1;
    bk[r] = stride * (int)(oc / ((int64_t)Nout * Nout)) - 1;
  }
  auto fetch = [&](int r, int k) -> __nv_bfloat16 {
    if (!ov[r] || k >= K) return __float2bfloat16(0.f);
    const int ci = k / 27, tap = k - ci * 27;
    const int ii = bi[r] + tap % 3, jj = bj[r] + (tap / 3) % 3, kk = bk[r] + tap / 9;
    if (ii < 0 || ii >= Nin || jj < 0 || jj >= Nin || kk < 0 || kk >= Nin) return __float2bfloat16(0.f);
    return x[(int64_t)ci * nin + ii + (int64_t)Nin * (jj + (int64_t)Nin * kk)];
  };
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[t][i] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    unsigned a[4];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
      for (int r = 0; r < 2; r++) {
        const int k = k0 + 8 * h + 2 * tq;
        a[2 * h + r] = pack_bf16(fetch(r, k), fetch(r, k + 1));
      }
#pragma unroll
    for (int t = 0; t < NT; t++) {
      const int co = t * 8 + g;
      unsigned b[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int k = k0 + 8 * h + 2 * tq;  // even, and K is even: k < K implies k + 1 < K
        b[h] = (co < CO && k < K) ? __ldg(reinterpret_cast<const unsigned*>(W + (int64_t)co * K + k)) : 0u;
      }
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
  }
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int r = i >> 1, co = t * 8 + 2 * tq + (i & 1);
      if (!ov[r] || co >= CO) continue;
      const int64_t o = o0 + g + 8 * r;
      float v = acc[t][i] + bias[co];
      if (relu) v = fmaxf(v, 0.f);
      if (yo) yo[(int64_t)co * nout + o] = __float2bfloat16(v);
      if (yf) yf[(int64_t)co * nout + o] = v + (add ? __bfloat162float(add[(int64_t)co * nout + o]) : 0.f);
    }
}

// Same GEMM with K in tap-major order, k = tap * Cin + ci, for Cin a multiple of
// 16: a k-step then stays within one tap, so each row's neighbour offset and
// bounds test are taken once per tap, and B pairs come from the tap-major copy
// Wt[co][tap][ci].
template <int CO>
__global__ void __launch_bounds__(128)
    k_conv_fwd_mma_t(const __nv_bfloat16* __restrict__ x, int Cin, int Nin, const __nv_bfloat16* __restrict__ Wt,
                     const float* __restrict__ bias, int Nout, int stride, int relu,
                     const __nv_bfloat16* __restrict__ add, __nv_bfloat16* __restrict__ yo, float* __restrict__ yf) {
  constexpr int NT = (CO + 7) / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t o0 = ((int64_t)blockIdx.x * 4 + warp) * 16;
  int bi[2], bj[2], bk[2];
  bool ov[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int64_t o = o0 + g + 8 * r;
    ov[r] = o < nout;
    const int64_t oc = ov[r] ? o : 0;
    bi[r] = stride * (int)(oc % Nout) - 1;
    bj[r] = stride * (int)((oc / Nout) % Nout) - 1;
    bk[r] = stride * (int)(oc / ((int64_t)Nout * Nout)) - 1;
  }
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[t][i] = 0.f;
  const unsigned short* xs = reinterpret_cast<const unsigned short*>(x);
  for (int tap = 0; tap < 27; tap++) {
    const int ti = tap % 3, tj = (tap / 3) % 3, tk = tap / 9;
    bool ok[2];
    int64_t off[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const int ii = bi[r] + ti, jj = bj[r] + tj, kk = bk[r] + tk;
      ok[r] = ov[r] && ii >= 0 && ii < Nin && jj >= 0 && jj < Nin && kk >= 0 && kk < Nin;
      off[r] = ok[r] ? ii + (int64_t)Nin * (jj + (int64_t)Nin * kk) : 0;
    }
    for (int ci0 = 0; ci0 < Cin; ci0 += 16) {
      unsigned a[4];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int64_t c = (int64_t)(ci0 + 8 * h + 2 * tq) * nin;
#pragma unroll
        for (int r = 0; r < 2; r++)
          a[2 * h + r] = ok[r] ? ((unsigned)xs[c + off[r]] | ((unsigned)xs[c + nin + off[r]] << 16)) : 0u;
      }
#pragma unroll
      for (int t = 0; t < NT; t++) {
        const int co = t * 8 + g;
        unsigned b[2];
#pragma unroll
        for (int h = 0; h < 2; h++)
          b[h] = co < CO ? __ldg(reinterpret_cast<const unsigned*>(Wt + ((int64_t)co * 27 + tap) * Cin + ci0 + 8 * h +
                                                                    2 * tq))
                         : 0u;
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int r = i >> 1, co = t * 8 + 2 * tq + (i & 1);
      if (!ov[r] || co >= CO) continue;
      const int64_t o = o0 + g + 8 * r;
      float v = acc[t][i] + bias[co];
      if (relu) v = fmaxf(v, 0.f);
      if (yo) yo[(int64_t)co * nout + o] = __float2bfloat16(v);
      if (yf) yf[(int64_t)co * nout + o] = v + (add ? __bfloat162float(add[(int64_t)co * nout + o]) : 0.f);
    }
}

// ---- input gradient of a convolution: one thread per input voxel ---------------
// dx[ci][x] = sum_co sum_tap W[co][ci][tap] dz[co][o],  x = stride o + tap - 1
template <typename TA, int CI>
__global__ void __launch_bounds__(128)
    k_conv_dx(const float* __restrict__ dz, int Cout, int Nout, const TA* __restrict__ W, int Nin, int stride,
              float* __restrict__ dx) {
  __shared__ __align__(16) float ws[kCC][27][CI];
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t xi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = xi < nin;
  const int ii = (int)(xi % Nin), jj = (int)((xi / Nin) % Nin), kk = (int)(xi / ((int64_t)Nin * Nin));
  float acc[CI];
#pragma unroll
  for (int c = 0; c < CI; c++) acc[c] = 0.f;
  for (int c0 = 0; c0 < Cout; c0 += kCC) {
    __syncthreads();
    for (int t = threadIdx.x; t < kCC * 27 * CI; t += blockDim.x) {
      const int ci = t % CI, tap = (t / CI) % 27, col = t / (CI * 27);
      const int co = c0 + col;
      ws[col][tap][ci] = co < Cout ? tof(W[((int64_t)co * CI + ci) * 27 + tap]) : 0.f;
    }
    __syncthreads();
    if (!live) continue;
    for (int col = 0; col < kCC && c0 + col < Cout; col++) {
      const float* dzc = dz + (int64_t)(c0 + col) * nout;
#pragma unroll
      for (int tap = 0; tap < 27; tap++) {
        const int a = ii - (tap % 3 - 1), b = jj - ((tap / 3) % 3 - 1), c = kk - (tap / 9 - 1);
        if (a < 0 || b < 0 || c < 0) continue;
        if (stride == 2 && ((a | b | c) & 1)) continue;
        const int oa = a / stride, ob = b / stride, oc = c / stride;
        if (oa >= Nout || ob >= Nout || oc >= Nout) continue;
        const float g = dzc[oa + (int64_t)Nout * (ob + (int64_t)Nout * oc)];
        const float4* w4 = reinterpret_cast<const float4*>(&ws[col][tap][0]);
#pragma unroll
        for (int q = 0; q < CI / 4; q++) {
          const float4 w = w4[q];
          acc[4 * q + 0] += w.x * g;
          acc[4 * q + 1] += w.y * g;
          acc[4 * q + 2] += w.z * g;
          acc[4 * q + 3] += w.w * g;
        }
      }
    }
  }
  if (!live) return;
#pragma unroll
  for (int c = 0; c < CI; c++) dx[(int64_t)c * nin + xi] = acc[c];
}

// ---- weight and bias gradients: block (co, ci, chunk of output voxels) ----------
__device__ __forceinline__ float block_sum_f(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = 0.f;
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

constexpr int kDWChunk = 8192;

template <typename TA>
__global__ void __launch_bounds__(256)
    k_conv_dw(const float* __restrict__ dz, int Cout, int Nout, const TA* __restrict__ x, int Cin, int Nin, int stride,
              float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float sh[32];
  const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t o0 = (int64_t)blockIdx.y * kDWChunk;
  const int64_t o1 = o0 + kDWChunk < nout ? o0 + kDWChunk : nout;
  const float* dzc = dz + (int64_t)co * nout;
  const TA* xc = x + (int64_t)ci * nin;
  float acc[27];
#pragma unroll
  for (int t = 0; t < 27; t++) acc[t] = 0.f;
  float accb = 0.f;
  for (int64_t o = o0 + threadIdx.x; o < o1; o += blockDim.x) {
    const float g = dzc[o];
    if (g == 0.f) continue;
    accb += g;
    const int oi = (int)(o % Nout), oj = (int)((o / Nout) % Nout), ok = (int)(o / ((int64_t)Nout * Nout));
#pragma unroll
    for (int tap = 0; tap < 27; tap++) {
      const int ii = stride * oi + tap % 3 - 1, jj = stride * oj + (tap / 3) % 3 - 1, kk = stride * ok + tap / 9 - 1;
      if (ii >= 0 && ii < Nin && jj >= 0 && jj < Nin && kk >= 0 && kk < Nin)
        acc[tap] += g * tof(xc[ii + (int64_t)Nin * (jj + (int64_t)Nin * kk)]);
    }
  }
  for (int tap = 0; tap < 27; tap++) {
    const float v = block_sum_f(acc[tap], sh);
    if (threadIdx.x == 0 && v != 0.f) atomicAdd(&dW[((int64_t)co * Cin + ci) * 27 + tap], v);
  }
  if (ci == 0) {
    const float v = block_sum_f(accb, sh);
    if (threadIdx.x == 0 && v != 0.f) atomicAdd(&db[co], v);
  }
}

// ---- backward convolutions on the tensor cores (TF32 operands, FP32 accumulation)
// The gradients stay FP32; mma.sync m16n8k8 rounds them to TF32 (10 explicit
// mantissa bits) on the way in, while BF16 activations and weights are exact in
// TF32.  Fragment layouts of m16n8k8 (g = lane / 4, q = lane % 4): A rows g, g + 8,
// columns q, q + 4; B rows q, q + 4, column g; C rows g, g + 8, columns 2q, 2q + 1.
__device__ __forceinline__ unsigned to_tf32(float f) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Input gradient as an implicit GEMM: dx[ci][x] = sum_k A[x][k] B[k][ci] over
// k = co * 27 + tap, A[x][k] = dz[co][o] where x = stride o + tap - 1 (zero when no
// such output voxel exists), B[k][ci] = W[co][ci][tap] read from the tap-major
// copy Wt[co][tap][ci].  A warp owns 16 input voxels and all CI channels.
template <int CI>
__global__ void __launch_bounds__(128)
    k_conv_dx_mma(const float* __restrict__ dz, int Cout, int Nout, const __nv_bfloat16* __restrict__ Wt, int Nin,
                  int stride, float* __restrict__ dx) {
  constexpr int NT = CI / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t m0 = ((int64_t)blockIdx.x * 4 + warp) * 16;
  int pi[2], pj[2], pk[2];
  bool rv[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int64_t xi = m0 + g + 8 * r;
    rv[r] = xi < nin;
    const int64_t xc = rv[r] ? xi : 0;
    pi[r] = (int)(xc % Nin) + 1;
    pj[r] = (int)((xc / Nin) % Nin) + 1;
    pk[r] = (int)(xc / ((int64_t)Nin * Nin)) + 1;
  }
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[t][i] = 0.f;
  int co_h[2] = {0, 0}, tap_h[2] = {tq, tq + 4};  // (co, tap) of this lane's columns k0 + q and k0 + q + 4
  const int K = Cout * 27;
  for (int k0 = 0; k0 < K; k0 += 8) {
    unsigned a[4];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int co = co_h[h], tap = tap_h[h];
      const int ti = tap % 3, tj = (tap / 3) % 3, tk = tap / 9;
#pragma unroll
      for (int r = 0; r < 2; r++) {
        float v = 0.f;
        int ia = pi[r] - ti, ib = pj[r] - tj, ic = pk[r] - tk;
        bool ok = rv[r] && co < Cout && ia >= 0 && ib >= 0 && ic >= 0;
        if (stride == 2) {
          ok = ok && !((ia | ib | ic) & 1);
          ia >>= 1;
          ib >>= 1;
          ic >>= 1;
        }
        if (ok && ia < Nout && ib < Nout && ic < Nout)
          v = dz[(int64_t)co * nout + ia + (int64_t)Nout * (ib + (int64_t)Nout * ic)];
        a[2 * h + r] = to_tf32(v);
      }
    }
#pragma unroll
    for (int t = 0; t < NT; t++) {
      unsigned b[2];
#pragma unroll
      for (int h = 0; h < 2; h++)
        b[h] = co_h[h] < Cout
                   ? __float_as_uint(__bfloat162float(Wt[((int64_t)co_h[h] * 27 + tap_h[h]) * CI + t * 8 + g]))
                   : 0u;
      mma_tf32(acc[t], a, b);
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
      tap_h[h] += 8;
      if (tap_h[h] >= 27) {
        tap_h[h] -= 27;
        co_h[h]++;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int r = i >> 1, c = t * 8 + 2 * tq + (i & 1);
      if (rv[r]) dx[(int64_t)c * nin + m0 + g + 8 * r] = acc[t][i];
    }
}

// Same GEMM with K in tap-outer order, k = tap * Cout + co, for Cout a multiple
// of 8: each row's source offset and tests are taken once per tap.
template <int CI>
__global__ void __launch_bounds__(128)
    k_conv_dx_mma_t(const float* __restrict__ dz, int Cout, int Nout, const __nv_bfloat16* __restrict__ Wt, int Nin,
                    int stride, float* __restrict__ dx) {
  constexpr int NT = CI / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int64_t m0 = ((int64_t)blockIdx.x * 4 + warp) * 16;
  int pi[2], pj[2], pk[2];
  bool rv[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int64_t xi = m0 + g + 8 * r;
    rv[r] = xi < nin;
    const int64_t xc = rv[r] ? xi : 0;
    pi[r] = (int)(xc % Nin) + 1;
    pj[r] = (int)((xc / Nin) % Nin) + 1;
    pk[r] = (int)(xc / ((int64_t)Nin * Nin)) + 1;
  }
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[t][i] = 0.f;
  for (int tap = 0; tap < 27; tap++) {
    const int ti = tap % 3, tj = (tap / 3) % 3, tk = tap / 9;
    bool ok[2];
    int64_t off[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      int ia = pi[r] - ti, ib = pj[r] - tj, ic = pk[r] - tk;
      bool v = rv[r] && ia >= 0 && ib >= 0 && ic >= 0;
      if (stride == 2) {
        v = v && !((ia | ib | ic) & 1);
        ia >>= 1;
        ib >>= 1;
        ic >>= 1;
      }
      ok[r] = v && ia < Nout && ib < Nout && ic < Nout;
      off[r] = ok[r] ? ia + (int64_t)Nout * (ib + (int64_t)Nout * ic) : 0;
    }
    if (!__any_sync(0xffffffffu, ok[0] || ok[1])) continue;  // stride 2: most taps have no source for the warp
    for (int co0 = 0; co0 < Cout; co0 += 8) {
      unsigned a[4];
#pragma unroll
      for (int h = 0; h < 2; h++)
#pragma unroll
        for (int r = 0; r < 2; r++)
          a[2 * h + r] = ok[r] ? to_tf32(dz[(int64_t)(co0 + tq + 4 * h) * nout + off[r]]) : 0u;
#pragma unroll
      for (int t = 0; t < NT; t++) {
        unsigned b[2];
#pragma unroll
        for (int h = 0; h < 2; h++)
          b[h] = __float_as_uint(__bfloat162float(Wt[((int64_t)(co0 + tq + 4 * h) * 27 + tap) * CI + t * 8 + g]));
        mma_tf32(acc[t], a, b);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int r = i >> 1, c = t * 8 + 2 * tq + (i & 1);
      if (rv[r]) dx[(int64_t)c * nin + m0 + g + 8 * r] = acc[t][i];
    }
}

// Weight gradient as a GEMM over the output voxels: dW[co][ci][tap] = sum_o
// A[(ci, tap)][o] B[o][co], A[(ci, tap)][o] = x[ci][stride o + tap - 1] (zero
// outside the grid), B[o][co] = dz[co][o].  A warp owns 16 (ci, tap) rows and all
// CO columns; the voxels run along x-rows, 8 per step (the row's tail padded with
// zeros), and a block sums the rows [rows_per_chunk * blockIdx.y, ...) before
// adding its partial sums atomically.  The bias gradient is k_bias_grad.
template <int CO>
__global__ void __launch_bounds__(128)
    k_conv_dw_mma(const float* __restrict__ dz, int Nout, const __nv_bfloat16* __restrict__ x, int Cin, int Nin,
                  int stride, int rows_per_chunk, float* __restrict__ dW) {
  constexpr int NT = (CO + 7) / 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int R = Cin * 27;
  const int64_t nout = (int64_t)Nout * Nout * Nout, nin = (int64_t)Nin * Nin * Nin;
  const int r0 = (blockIdx.x * 4 + warp) * 16;
  int rr[2], di[2], dj[2], dk[2];
  bool rv[2];
  const __nv_bfloat16* xc[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    rr[r] = r0 + g + 8 * r;
    rv[r] = rr[r] < R;
    const int ci = rv[r] ? rr[r] / 27 : 0, tap = rv[r] ? rr[r] % 27 : 0;
    di[r] = tap % 3 - 1;
    dj[r] = (tap / 3) % 3 - 1;
    dk[r] = tap / 9 - 1;
    xc[r] = x + (int64_t)ci * nin;
  }
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[t][i] = 0.f;
  const int nrows = Nout * Nout;
  const int y0 = blockIdx.y * rows_per_chunk;
  const int y1 = y0 + rows_per_chunk < nrows ? y0 + rows_per_chunk : nrows;
  for (int row = y0; row < y1; row++) {
    const int oj = row % Nout, ok = row / Nout;
    bool rowok[2];
    const __nv_bfloat16* base[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const int jj = stride * oj + dj[r], kk = stride * ok + dk[r];
      rowok[r] = rv[r] && jj >= 0 && jj < Nin && kk >= 0 && kk < Nin;
      base[r] = xc[r] + (rowok[r] ? (int64_t)Nin * (jj + (int64_t)Nin * kk) : 0);
    }
    const float* dzrow = dz + (int64_t)row * Nout;
    for (int oi0 = 0; oi0 < Nout; oi0 += 8) {
      unsigned a[4];
      bool colok[2];
      int oi[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        oi[h] = oi0 + tq + 4 * h;
        colok[h] = oi[h] < Nout;
#pragma unroll
        for (int r = 0; r < 2; r++) {
          const int ii = stride * oi[h] + di[r];
          const bool ok = rowok[r] && colok[h] && ii >= 0 && ii < Nin;
          a[2 * h + r] = ok ? __float_as_uint(__bfloat162float(base[r][ii])) : 0u;
        }
      }
#pragma unroll
      for (int t = 0; t < NT; t++) {
        const int co = t * 8 + g;
        unsigned b[2];
#pragma unroll
        for (int h = 0; h < 2; h++) b[h] = (co < CO && colok[h]) ? to_tf32(dzrow[(int64_t)co * nout + oi[h]]) : 0u;
        mma_tf32(acc[t], a, b);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; t++)
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int r = i >> 1, co = t * 8 + 2 * tq + (i & 1);
      if (rv[r] && co < CO && acc[t][i] != 0.f) atomicAdd(&dW[(int64_t)co * R + rr[r]], acc[t][i]);
    }
}

// db[co] += sum_o dz[co][o]: one block per output channel, fixed summation order.
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ dz, int64_t nout, float* __restrict__ db) {
  __shared__ float sh[32];
  const float* d = dz + (int64_t)blockIdx.x * nout;
  float v = 0.f;
  for (int64_t o = threadIdx.x; o < nout; o += blockDim.x) v += d[o];
  v = block_sum_f(v, sh);
  if (threadIdx.x == 0) db[blockIdx.x] += v;
}

// Tap-major copy of every layer's BF16 weights: Wt[co][tap][ci] = W[co][ci][tap]
// (blockIdx.y = layer).
struct LayerTable {
  int n;
  int64_t off[32];
  int cin[32], cout[32];
};

__global__ void k_tap_major(LayerTable tab, const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt) {
  const int l = blockIdx.y;
  const int ci_n = tab.cin[l];
  const int64_t cnt = (int64_t)tab.cout[l] * ci_n * 27, off = tab.off[l];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int tap = (int)(e % 27), ci = (int)((e / 27) % ci_n);
    const int64_t co = e / (27 * (int64_t)ci_n);
    wt[off + (co * 27 + tap) * ci_n + ci] = w[off + e];
  }
}

// ---- elementwise ---------------------------------------------------------------
template <typename TA>
__global__ void k_relu_mask(int64_t n, const TA* __restrict__ y, float* __restrict__ g) {
  GSTRIDE(i, n) if (!(tof(y[i]) > 0.f)) g[i] = 0.f;
}

template <typename TA>
__global__ void k_upsample(int C, int M, const TA* __restrict__ in, TA* __restrict__ out) {
  const int N = 2 * M - 1;
  const int64_t nf = (int64_t)N * N * N, nc = (int64_t)M * M * M;
  GSTRIDE(t, (int64_t)C * nf) {
    const int c = (int)(t / nf);
    const int64_t f = t - (int64_t)c * nf;
    const int I = (int)(f % N), J = (int)((f / N) % N), K = (int)(f / ((int64_t)N * N));
    const int i0 = I >> 1, j0 = J >> 1, k0 = K >> 1;
    const int i1 = i0 + (I & 1), j1 = j0 + (J & 1), k1 = k0 + (K & 1);
    const TA* src = in + (int64_t)c * nc;
    auto at = [&](int i, int j, int k) { return tof(src[i + (int64_t)M * (j + (int64_t)M * k)]); };
    const float v = 0.125f * (at(i0, j0, k0) + at(i1, j0, k0) + at(i0, j1, k0) + at(i1, j1, k0) + at(i0, j0, k1) +
                              at(i1, j0, k1) + at(i0, j1, k1) + at(i1, j1, k1));
    out[t] = fromf<TA>(v);
  }
}

// transpose of k_upsample: coarse node gathers its fine neighbours
__global__ void k_upsample_t(int C, int M, const float* __restrict__ g, float* __restrict__ out) {
  const int N = 2 * M - 1;
  const int64_t nf = (int64_t)N * N * N, nc = (int64_t)M * M * M;
  GSTRIDE(t, (int64_t)C * nc) {
    const int c = (int)(t / nc);
    const int64_t q = t - (int64_t)c * nc;
    const int i = (int)(q % M), j = (int)((q / M) % M), k = (int)(q / ((int64_t)M * M));
    const float* src = g + (int64_t)c * nf;
    float s = 0.f;
    for (int dk = -1; dk <= 1; dk++) {
      const int K = 2 * k + dk;
      if (K < 0 || K >= N) continue;
      const float wk = dk ? 0.5f : 1.f;
      for (int dj = -1; dj <= 1; dj++) {
        const int J = 2 * j + dj;
        if (J < 0 || J >= N) continue;
        const float wj = dj ? 0.5f : 1.f;
        for (int di = -1; di <= 1; di++) {
          const int I = 2 * i + di;
          if (I < 0 || I >= N) continue;
          s += wk * wj * (di ? 0.5f : 1.f) * src[I + (int64_t)N * (J + (int64_t)N * K)];
        }
      }
    }
    out[t] = s;
  }
}

template <typename TA>
__global__ void k_add_to(int64_t n, const TA* __restrict__ a, TA* __restrict__ y) {
  GSTRIDE(i, n) y[i] = fromf<TA>(tof(y[i]) + tof(a[i]));
}

__global__ void k_addf(int64_t n, const float* __restrict__ a, float* __restrict__ y) { GSTRIDE(i, n) y[i] += a[i]; }

template <typename TA>
__global__ void k_from_f32(int64_t n, const float* __restrict__ a, TA* __restrict__ y) {
  GSTRIDE(i, n) y[i] = fromf<TA>(a[i]);
}

// loss pieces: s[0] += sum (y - t)^2, s[1] += sum t^2
__global__ void k_loss_sums(int64_t n, const float* __restrict__ y, const float* __restrict__ t, double* __restrict__ s) {
  __shared__ float sh[32];
  float a = 0.f, b = 0.f;
  GSTRIDE(i, n) {
    const float d = y[i] - t[i];
    a += d * d;
    b += t[i] * t[i];
  }
  a = block_sum_f(a, sh);
  b = block_sum_f(b, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&s[0], (double)a);
    atomicAdd(&s[1], (double)b);
  }
}

// dy = scale * 2 (y - t) / s[1]
__global__ void k_loss_grad(int64_t n, const float* __restrict__ y, const float* __restrict__ t,
                            const double* __restrict__ s, float scale, float* __restrict__ dy) {
  const float f = (float)(2.0 * scale / s[1]);
  GSTRIDE(i, n) dy[i] = f * (y[i] - t[i]);
}

__global__ void k_adam(int64_t n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  GSTRIDE(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// He-normal initial weights from splitmix64 + Box-Muller
__device__ __forceinline__ uint64_t sm64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_init(int64_t n, int64_t off, float sd, uint64_t seed, float* __restrict__ th) {
  GSTRIDE(i, n) {
    const uint64_t a = sm64(seed * 0x100000001b3ull + 2 * (uint64_t)(off + i));
    const uint64_t b = sm64(seed * 0x100000001b3ull + 2 * (uint64_t)(off + i) + 1);
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    th[i] = sd * (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

struct Layer {
  int cin, cout, stride, relu, lin, lout;  // grid levels of input and output
  int64_t woff, boff;
};

}  // namespace

struct nh_net_s {
  nh_ctx ctx = nullptr;
  int N = 0, levels = 0, bf16 = 1;
  int mma = 1;                  // BF16 forward convolutions on the tensor cores (else the CUDA-core kernel)
  int ch[8] = {0};
  std::vector<int> Ng;
  std::vector<Layer> L;
  int64_t np = 0;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  void* wc = nullptr;           // compute copy of the parameters (TA)
  void* wt = nullptr;           // BF16 networks: tap-major copy of the weights (input-gradient GEMM)
  int64_t adam_t = 0;
  std::vector<void*> out;       // per layer: stored activation (TA), [cout][Ng[lout]^3]
  std::vector<void*> ups;       // per decoder block: upsampled input (TA)
  std::vector<void*> sums;      // per decoder block: relu(conv(up)) + skip (TA)
  void* xin = nullptr;          // TA input [4][N^3]
  float* yout = nullptr;        // FP32 output [3][N^3]
  float *g0 = nullptr, *g1 = nullptr;  // FP32 gradient ping-pong, max C N^3
  std::vector<float*> sg;       // per level: gradient arriving through the skip
  double* ls = nullptr;         // loss sums
  double* ls_host = nullptr;
  float* gy = nullptr;          // FP32 output gradient
};

namespace {

size_t tsz(const nh_net_s* n) { return n->bf16 ? 2 : 4; }
int64_t vox(const nh_net_s* n, int l) { return (int64_t)n->Ng[l] * n->Ng[l] * n->Ng[l]; }

#ifndef NH_NET_MMA
#define NH_NET_MMA 1
#endif

template <typename TA>
cudaError_t conv_fwd(nh_net n, int li, const void* x, const void* add, float* yf, bool store) {
  const Layer& y = n->L[li];
  const TA* W = (const TA*)n->wc + y.woff;
  const float* b = n->theta + y.boff;  // biases read from the FP32 master copy
  const int64_t no = vox(n, y.lout);
  TA* yo = store ? (TA*)n->out[li] : nullptr;
  const unsigned g = (unsigned)((no + 127) / 128);
  cudaStream_t st = n->ctx->stream;
  if constexpr (std::is_same<TA, __nv_bfloat16>::value) {
    if (NH_NET_MMA && n->mma && y.cin % 2 == 0 && (int64_t)W % 4 == 0 && (y.woff % 2) == 0) {
      const unsigned gm = (unsigned)((no + 63) / 64);
      const __nv_bfloat16* xb = (const __nv_bfloat16*)x;
      const __nv_bfloat16* ab = (const __nv_bfloat16*)add;
      const __nv_bfloat16* Wt = (const __nv_bfloat16*)n->wt + y.woff;
      const int Ni = n->Ng[y.lin], No = n->Ng[y.lout];
      if (y.cin % 16 == 0) {
        switch (y.cout) {
          case 3: k_conv_fwd_mma_t<3><<<gm, 128, 0, st>>>(xb, y.cin, Ni, Wt, b, No, y.stride, y.relu, ab, yo, yf); break;
          case 8: k_conv_fwd_mma_t<8><<<gm, 128, 0, st>>>(xb, y.cin, Ni, Wt, b, No, y.stride, y.relu, ab, yo, yf); break;
          case 16: k_conv_fwd_mma_t<16><<<gm, 128, 0, st>>>(xb, y.cin, Ni, Wt, b, No, y.stride, y.relu, ab, yo, yf); break;
          case 32: k_conv_fwd_mma_t<32><<<gm, 128, 0, st>>>(xb, y.cin, Ni, Wt, b, No, y.stride, y.relu, ab, yo, yf); break;
          case 48: k_conv_fwd_mma_t<48><<<gm, 128, 0, st>>>(xb, y.cin, Ni, Wt, b, No, y.stride, y.relu, ab, yo, yf); break;
          case 64: k_conv_fwd_mma_t<64><<<gm, 128, 0, st>>>(xb, y.cin, Ni, Wt, b, No, y.stride, y.relu, ab, yo, yf); break;
          default: return cudaErrorInvalidValue;
        }
        n->ctx->launches++;
        return cudaGetLastError();
      }
      switch (y.cout) {
        case 3: k_conv_fwd_mma<3><<<gm, 128, 0, st>>>(xb, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, ab, yo, yf); break;
        case 8: k_conv_fwd_mma<8><<<gm, 128, 0, st>>>(xb, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, ab, yo, yf); break;
        case 16: k_conv_fwd_mma<16><<<gm, 128, 0, st>>>(xb, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, ab, yo, yf); break;
        case 32: k_conv_fwd_mma<32><<<gm, 128, 0, st>>>(xb, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, ab, yo, yf); break;
        case 48: k_conv_fwd_mma<48><<<gm, 128, 0, st>>>(xb, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, ab, yo, yf); break;
        case 64: k_conv_fwd_mma<64><<<gm, 128, 0, st>>>(xb, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, ab, yo, yf); break;
        default: return cudaErrorInvalidValue;
      }
      n->ctx->launches++;
      return cudaGetLastError();
    }
  }
  switch (y.cout) {
    case 3: k_conv_fwd<TA, 3><<<g, 128, 0, st>>>((const TA*)x, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, (const TA*)add, yo, yf); break;
    case 8: k_conv_fwd<TA, 8><<<g, 128, 0, st>>>((const TA*)x, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, (const TA*)add, yo, yf); break;
    case 16: k_conv_fwd<TA, 16><<<g, 128, 0, st>>>((const TA*)x, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, (const TA*)add, yo, yf); break;
    case 32: k_conv_fwd<TA, 32><<<g, 128, 0, st>>>((const TA*)x, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, (const TA*)add, yo, yf); break;
    case 48: k_conv_fwd<TA, 48><<<g, 128, 0, st>>>((const TA*)x, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, (const TA*)add, yo, yf); break;
    case 64: k_conv_fwd<TA, 64><<<g, 128, 0, st>>>((const TA*)x, y.cin, n->Ng[y.lin], W, b, n->Ng[y.lout], y.stride, y.relu, (const TA*)add, yo, yf); break;
    default: return cudaErrorInvalidValue;
  }
  n->ctx->launches++;
  return cudaGetLastError();
}

template <typename TA>
cudaError_t conv_dx(nh_net n, int li, const float* dz, float* dx) {
  const Layer& y = n->L[li];
  const TA* W = (const TA*)n->wc + y.woff;
  const int64_t ni = vox(n, y.lin);
  const unsigned g = (unsigned)((ni + 127) / 128);
  cudaStream_t st = n->ctx->stream;
  if (std::is_same<TA, __nv_bfloat16>::value && NH_NET_MMA && n->mma) {
    const __nv_bfloat16* Wt = (const __nv_bfloat16*)n->wt + y.woff;
    const unsigned gm = (unsigned)((ni + 63) / 64);
    const int No = n->Ng[y.lout], Ni = n->Ng[y.lin];
    if (y.cout % 8 == 0) {
      switch (y.cin) {
        case 8: k_conv_dx_mma_t<8><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
        case 16: k_conv_dx_mma_t<16><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
        case 32: k_conv_dx_mma_t<32><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
        case 48: k_conv_dx_mma_t<48><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
        case 64: k_conv_dx_mma_t<64><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
        default: return cudaErrorInvalidValue;
      }
      n->ctx->launches++;
      return cudaGetLastError();
    }
    switch (y.cin) {
      case 8: k_conv_dx_mma<8><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
      case 16: k_conv_dx_mma<16><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
      case 32: k_conv_dx_mma<32><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
      case 48: k_conv_dx_mma<48><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
      case 64: k_conv_dx_mma<64><<<gm, 128, 0, st>>>(dz, y.cout, No, Wt, Ni, y.stride, dx); break;
      default: return cudaErrorInvalidValue;
    }
    n->ctx->launches++;
    return cudaGetLastError();
  }
  switch (y.cin) {
    case 8: k_conv_dx<TA, 8><<<g, 128, 0, st>>>(dz, y.cout, n->Ng[y.lout], W, n->Ng[y.lin], y.stride, dx); break;
    case 16: k_conv_dx<TA, 16><<<g, 128, 0, st>>>(dz, y.cout, n->Ng[y.lout], W, n->Ng[y.lin], y.stride, dx); break;
    case 32: k_conv_dx<TA, 32><<<g, 128, 0, st>>>(dz, y.cout, n->Ng[y.lout], W, n->Ng[y.lin], y.stride, dx); break;
    case 48: k_conv_dx<TA, 48><<<g, 128, 0, st>>>(dz, y.cout, n->Ng[y.lout], W, n->Ng[y.lin], y.stride, dx); break;
    case 64: k_conv_dx<TA, 64><<<g, 128, 0, st>>>(dz, y.cout, n->Ng[y.lout], W, n->Ng[y.lin], y.stride, dx); break;
    default: return cudaErrorInvalidValue;
  }
  n->ctx->launches++;
  return cudaGetLastError();
}

template <typename TA>
cudaError_t conv_dw(nh_net n, int li, const float* dz, const void* x) {
  const Layer& y = n->L[li];
  const int64_t no = vox(n, y.lout);
  if (std::is_same<TA, __nv_bfloat16>::value && NH_NET_MMA && n->mma) {
    cudaStream_t st = n->ctx->stream;
    const int No = n->Ng[y.lout], Ni = n->Ng[y.lin];
    const unsigned bx = (unsigned)((y.cin * 27 + 63) / 64);
    const int rows = No * No;
    int chunks = (148 * 8 + (int)bx - 1) / (int)bx;  // about 8 blocks per SM
    if (chunks > rows) chunks = rows;
    const int per = (rows + chunks - 1) / chunks;
    const dim3 grid(bx, (unsigned)((rows + per - 1) / per));
    const __nv_bfloat16* xb = (const __nv_bfloat16*)x;
    float* dW = n->grad + y.woff;
    switch (y.cout) {
      case 3: k_conv_dw_mma<3><<<grid, 128, 0, st>>>(dz, No, xb, y.cin, Ni, y.stride, per, dW); break;
      case 8: k_conv_dw_mma<8><<<grid, 128, 0, st>>>(dz, No, xb, y.cin, Ni, y.stride, per, dW); break;
      case 16: k_conv_dw_mma<16><<<grid, 128, 0, st>>>(dz, No, xb, y.cin, Ni, y.stride, per, dW); break;
      case 32: k_conv_dw_mma<32><<<grid, 128, 0, st>>>(dz, No, xb, y.cin, Ni, y.stride, per, dW); break;
      case 48: k_conv_dw_mma<48><<<grid, 128, 0, st>>>(dz, No, xb, y.cin, Ni, y.stride, per, dW); break;
      case 64: k_conv_dw_mma<64><<<grid, 128, 0, st>>>(dz, No, xb, y.cin, Ni, y.stride, per, dW); break;
      default: return cudaErrorInvalidValue;
    }
    k_bias_grad<<<(unsigned)y.cout, 256, 0, st>>>(dz, no, n->grad + y.boff);
    n->ctx->launches += 2;
    return cudaGetLastError();
  }
  dim3 grid((unsigned)(y.cout * y.cin), (unsigned)((no + kDWChunk - 1) / kDWChunk));
  k_conv_dw<TA><<<grid, 256, 0, n->ctx->stream>>>(dz, y.cout, n->Ng[y.lout], (const TA*)x, y.cin, n->Ng[y.lin],
                                                  y.stride, n->grad + y.woff, n->grad + y.boff);
  n->ctx->launches++;
  return cudaGetLastError();
}

// input tensor of layer li during the forward pass
const void* layer_input(nh_net n, int li) {
  const int L = n->levels;
  if (li == 0) return n->xin;
  const int enc_end = 2 * L;  // layers [0, 2L) are the encoder
  if (li < enc_end) return n->out[li - 1];
  const int d = (li - enc_end) / 2, second = (li - enc_end) % 2;
  if (li == (int)n->L.size() - 1) return n->sums.empty() ? n->out[li - 1] : n->out[li - 1];
  return second ? n->sums[d] : n->ups[d];
}

#define NCK(call)                                                \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return nh_cuda_check(n->ctx, _e, #call); \
  } while (0)

template <typename TA>
nh_status forward_t(nh_net n, const float* in, float* y) {
  cudaStream_t st = n->ctx->stream;
  const int L = n->levels;
  const int64_t n0 = vox(n, 0);
  k_from_f32<TA><<<blocks_for(4 * n0), 256, 0, st>>>(4 * n0, in, (TA*)n->xin);
  n->ctx->launches++;
  int li = 0;
  NCK(conv_fwd<TA>(n, li, layer_input(n, li), nullptr, nullptr, true)); li++;
  NCK(conv_fwd<TA>(n, li, layer_input(n, li), nullptr, nullptr, true)); li++;
  for (int l = 1; l < L; l++) {
    NCK(conv_fwd<TA>(n, li, layer_input(n, li), nullptr, nullptr, true)); li++;
    NCK(conv_fwd<TA>(n, li, layer_input(n, li), nullptr, nullptr, true)); li++;
  }
  for (int d = 0; d < L - 1; d++) {
    const int l = L - 2 - d;  // output level of this block
    const Layer& c1 = n->L[li];
    k_upsample<TA><<<blocks_for((int64_t)c1.cin * vox(n, l)), 256, 0, st>>>(c1.cin, n->Ng[l + 1],
                                                                            (const TA*)n->out[li - 1], (TA*)n->ups[d]);
    n->ctx->launches++;
    NCK(conv_fwd<TA>(n, li, n->ups[d], nullptr, nullptr, true));
    // sum = relu(conv(up)) + s_l ; s_l is the output of encoder layer 2l + 1
    const int64_t ne = (int64_t)c1.cout * vox(n, l);
    NCK(cudaMemcpyAsync(n->sums[d], n->out[li], tsz(n) * ne, cudaMemcpyDeviceToDevice, st));
    k_add_to<TA><<<blocks_for(ne), 256, 0, st>>>(ne, (const TA*)n->out[2 * l + 1], (TA*)n->sums[d]);
    n->ctx->launches++;
    li++;
    NCK(conv_fwd<TA>(n, li, n->sums[d], nullptr, nullptr, true));
    li++;
  }
  NCK(conv_fwd<TA>(n, li, n->out[li - 1], nullptr, y, false));
  return NH_OK;
}

// gradients of all parameters (accumulated into n->grad) for dL/dy = gy
template <typename TA>
nh_status backward_t(nh_net n, const float* gy) {
  cudaStream_t st = n->ctx->stream;
  const int L = n->levels;
  int li = (int)n->L.size() - 1;
  float* g = n->g0;
  float* h = n->g1;
  // output layer (no activation)
  NCK(conv_dw<TA>(n, li, gy, n->out[li - 1]));
  NCK(conv_dx<TA>(n, li, gy, g));
  li--;
  for (int d = L - 2; d >= 0; d--) {
    const int l = L - 2 - d;
    // second conv of the block: input sums[d]
    const Layer& c2 = n->L[li];
    const int64_t n2 = (int64_t)c2.cout * vox(n, c2.lout);
    k_relu_mask<TA><<<blocks_for(n2), 256, 0, st>>>(n2, (const TA*)n->out[li], g);
    NCK(conv_dw<TA>(n, li, g, n->sums[d]));
    NCK(conv_dx<TA>(n, li, g, h));  // h = d sums[d]
    n->ctx->launches++;
    li--;
    // sums = relu(conv(up)) + s_l
    const Layer& c1 = n->L[li];
    const int64_t n1 = (int64_t)c1.cout * vox(n, c1.lout);
    NCK(cudaMemcpyAsync(n->sg[l], h, sizeof(float) * n1, cudaMemcpyDeviceToDevice, st));
    k_relu_mask<TA><<<blocks_for(n1), 256, 0, st>>>(n1, (const TA*)n->out[li], h);
    NCK(conv_dw<TA>(n, li, h, n->ups[d]));
    NCK(conv_dx<TA>(n, li, h, g));  // g = d ups[d] at level l
    n->ctx->launches++;
    li--;
    // transpose of the upsampling to level l + 1
    k_upsample_t<<<blocks_for((int64_t)c1.cin * vox(n, l + 1)), 256, 0, st>>>(c1.cin, n->Ng[l + 1], g, h);
    n->ctx->launches++;
    float* t = g;
    g = h;
    h = t;
  }
  for (int l = L - 1; l >= 0; l--) {
    const int64_t nl = (int64_t)n->ch[l] * vox(n, l);
    if (l < L - 1) {
      k_addf<<<blocks_for(nl), 256, 0, st>>>(nl, n->sg[l], g);
      n->ctx->launches++;
    }
    for (int k = 0; k < 2; k++) {
      const Layer& c = n->L[li];
      const int64_t nc = (int64_t)c.cout * vox(n, c.lout);
      k_relu_mask<TA><<<blocks_for(nc), 256, 0, st>>>(nc, (const TA*)n->out[li], g);
      n->ctx->launches++;
      NCK(conv_dw<TA>(n, li, g, layer_input(n, li)));
      if (li > 0) {
        NCK(conv_dx<TA>(n, li, g, h));
        float* t = g;
        g = h;
        h = t;
      }
      li--;
    }
  }
  return NH_OK;
}

nh_status refresh_compute_copy(nh_net n) {
  if (n->bf16) {
    k_from_f32<__nv_bfloat16><<<blocks_for(n->np), 256, 0, n->ctx->stream>>>(n->np, n->theta, (__nv_bfloat16*)n->wc);
    LayerTable tab{};
    tab.n = (int)n->L.size();  // 4 L - 1 <= 23 layers for L <= 6 levels (checked at creation)
    if (tab.n > 32) return nh_fail(n->ctx, NH_ERR_UNSUPPORTED, "network: more than 32 layers");
    for (int l = 0; l < tab.n; l++) {
      tab.off[l] = n->L[l].woff;
      tab.cin[l] = n->L[l].cin;
      tab.cout[l] = n->L[l].cout;
    }
    k_tap_major<<<dim3(64, (unsigned)tab.n), 256, 0, n->ctx->stream>>>(tab, (const __nv_bfloat16*)n->wc,
                                                                        (__nv_bfloat16*)n->wt);
    n->ctx->launches++;
  } else
    k_from_f32<float><<<blocks_for(n->np), 256, 0, n->ctx->stream>>>(n->np, n->theta, (float*)n->wc);
  n->ctx->launches++;
  NCK(cudaGetLastError());
  return NH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// feature / target conversion between the solver's node-major FP64 vectors and
// the network's channel-major FP32 fields
// ---------------------------------------------------------------------------
namespace {

__global__ void k_features(int64_t nc, const double* __restrict__ rc, double inv, const float* __restrict__ logE,
                           float* __restrict__ feat) {
  GSTRIDE(i, nc) {
    feat[i] = (float)(rc[3 * i] * inv);
    feat[nc + i] = (float)(rc[3 * i + 1] * inv);
    feat[2 * nc + i] = (float)(rc[3 * i + 2] * inv);
    feat[3 * nc + i] = logE[i];
  }
}

__global__ void k_from_net(int64_t nc, const float* __restrict__ out, double scale, double* __restrict__ ec) {
  GSTRIDE(i, nc) {
    ec[3 * i] = scale * out[i];
    ec[3 * i + 1] = scale * out[nc + i];
    ec[3 * i + 2] = scale * out[2 * nc + i];
  }
}

// vertex node (i, j, k) of a Q_p lattice with Nf nodes per direction is fine node (p i, p j, p k)
__global__ void k_inject(int Nv, int p, int Nf, const double* __restrict__ ef, double inv, float* __restrict__ tgt) {
  const int64_t nc = (int64_t)Nv * Nv * Nv;
  GSTRIDE(v, nc) {
    const int i = (int)(v % Nv), j = (int)((v / Nv) % Nv), k = (int)(v / ((int64_t)Nv * Nv));
    const int64_t f = (int64_t)p * i + (int64_t)Nf * ((int64_t)p * j + (int64_t)Nf * ((int64_t)p * k));
    tgt[v] = (float)(ef[3 * f] * inv);
    tgt[nc + v] = (float)(ef[3 * f + 1] * inv);
    tgt[2 * nc + v] = (float)(ef[3 * f + 2] * inv);
  }
}

__global__ void k_to_channels(int64_t nc, const double* __restrict__ ec, double inv, float* __restrict__ t) {
  GSTRIDE(i, nc) {
    t[i] = (float)(ec[3 * i] * inv);
    t[nc + i] = (float)(ec[3 * i + 1] * inv);
    t[2 * nc + i] = (float)(ec[3 * i + 2] * inv);
  }
}

}  // namespace

cudaError_t kn_to_channels(cudaStream_t st, int64_t nc, const double* ec, double inv, float* t) {
  k_to_channels<<<blocks_for(nc), 256, 0, st>>>(nc, ec, inv, t);
  return cudaGetLastError();
}

cudaError_t kn_features(cudaStream_t st, int64_t nc, const double* rc, double inv, const float* logE, float* feat) {
  k_features<<<blocks_for(nc), 256, 0, st>>>(nc, rc, inv, logE, feat);
  return cudaGetLastError();
}
cudaError_t kn_from_net(cudaStream_t st, int64_t nc, const float* out, double scale, double* ec) {
  k_from_net<<<blocks_for(nc), 256, 0, st>>>(nc, out, scale, ec);
  return cudaGetLastError();
}
cudaError_t kn_inject(cudaStream_t st, int Nv, int p, int Nf, const double* ef, double inv, float* tgt) {
  k_inject<<<blocks_for((int64_t)Nv * Nv * Nv), 256, 0, st>>>(Nv, p, Nf, ef, inv, tgt);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// internal entry points used by the solver
// ---------------------------------------------------------------------------
int nh_net_grid(nh_net n) { return n ? n->N : 0; }

nh_status nh_net_forward_internal(nh_net n, const float* in, float* out) {
  return n->bf16 ? forward_t<__nv_bfloat16>(n, in, out) : forward_t<float>(n, in, out);
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" nh_status nh_net_set_tensor_cores(nh_net n, int on) {
  if (!n) return NH_ERR_ARG;
  n->mma = on ? 1 : 0;
  return NH_OK;
}

extern "C" nh_status nh_net_destroy(nh_net n) {
  if (!n) return NH_ERR_ARG;
  cudaStreamSynchronize(n->ctx->stream);
  for (void* p : n->out) cudaFree(p);
  for (void* p : n->ups) cudaFree(p);
  for (void* p : n->sums) cudaFree(p);
  for (float* p : n->sg) cudaFree(p);
  for (void* p : {(void*)n->theta, (void*)n->grad, (void*)n->m1, (void*)n->m2, n->wc, n->wt, n->xin, (void*)n->yout,
                  (void*)n->g0, (void*)n->g1, (void*)n->ls, (void*)n->gy})
    cudaFree(p);
  cudaFreeHost(n->ls_host);
  delete n;
  return NH_OK;
}

extern "C" nh_status nh_net_create(nh_ctx ctx, int N, int levels, const int* channels, int bf16, uint64_t seed,
                                   nh_net* out) {
  if (!ctx || !out || !channels) return NH_ERR_ARG;
  *out = nullptr;
  if (levels < 2 || levels > 6 || N < 5 || !(N & 1))
    return nh_fail(ctx, NH_ERR_ARG, "nh_net_create: need 2 <= levels <= 6 and an odd grid N >= 5");
  int M = N;
  for (int l = 1; l < levels; l++) {
    if (!(M & 1) || M < 3) return nh_fail(ctx, NH_ERR_ARG, "nh_net_create: grid too small for the levels");
    M = (M - 1) / 2 + 1;
  }
  for (int l = 0; l < levels; l++)
    if (channels[l] != 8 && channels[l] != 16 && channels[l] != 32 && channels[l] != 48 && channels[l] != 64)
      return nh_fail(ctx, NH_ERR_UNSUPPORTED, "nh_net_create: channels must be 8, 16, 32, 48 or 64");
  NH_CUDA(ctx, cudaSetDevice(ctx->device));
  nh_net n = new nh_net_s();
  n->ctx = ctx;
  n->N = N;
  n->levels = levels;
  n->bf16 = bf16 ? 1 : 0;
  for (int l = 0; l < levels; l++) n->ch[l] = channels[l];
  n->Ng.resize(levels);
  n->Ng[0] = N;
  for (int l = 1; l < levels; l++) n->Ng[l] = (n->Ng[l - 1] - 1) / 2 + 1;
  auto add = [&](int ci, int co, int s, int relu, int lin, int lout) {
    Layer y{ci, co, s, relu, lin, lout, n->np, n->np + (int64_t)co * ci * 27};
    n->np += (int64_t)co * ci * 27 + co;
    n->L.push_back(y);
  };
  add(4, channels[0], 1, 1, 0, 0);
  add(channels[0], channels[0], 1, 1, 0, 0);
  for (int l = 1; l < levels; l++) {
    add(channels[l - 1], channels[l], 2, 1, l - 1, l);
    add(channels[l], channels[l], 1, 1, l, l);
  }
  for (int l = levels - 2; l >= 0; l--) {
    add(channels[l + 1], channels[l], 1, 1, l, l);
    add(channels[l], channels[l], 1, 1, l, l);
  }
  add(channels[0], 3, 1, 0, 0, 0);
  auto fail = [&]() {
    cudaGetLastError();
    nh_net_destroy(n);
    return nh_fail(ctx, NH_ERR_OOM, "nh_net_create: device allocation failed");
  };
  const size_t ts = tsz(n);
  if (cudaMalloc(&n->theta, 4 * n->np) || cudaMalloc(&n->grad, 4 * n->np) || cudaMalloc(&n->m1, 4 * n->np) ||
      cudaMalloc(&n->m2, 4 * n->np) || cudaMalloc(&n->wc, ts * n->np) ||
      (n->bf16 && cudaMalloc(&n->wt, ts * n->np)))
    return fail();
  int64_t maxc = 4 * vox(n, 0);
  n->out.assign(n->L.size(), nullptr);
  for (size_t i = 0; i < n->L.size(); i++) {
    const int64_t e = (int64_t)n->L[i].cout * vox(n, n->L[i].lout);
    maxc = std::max(maxc, e);
    maxc = std::max(maxc, (int64_t)n->L[i].cin * vox(n, n->L[i].lin));
    if (i + 1 < n->L.size() && cudaMalloc(&n->out[i], ts * e)) return fail();
  }
  for (int d = 0; d < levels - 1; d++) {
    const int l = levels - 2 - d;
    void *u = nullptr, *s = nullptr;
    if (cudaMalloc(&u, ts * (int64_t)channels[l + 1] * vox(n, l)) || cudaMalloc(&s, ts * (int64_t)channels[l] * vox(n, l)))
      return fail();
    n->ups.push_back(u);
    n->sums.push_back(s);
  }
  n->sg.assign(levels, nullptr);
  for (int l = 0; l < levels - 1; l++)
    if (cudaMalloc(&n->sg[l], 4 * (int64_t)channels[l] * vox(n, l))) return fail();
  if (cudaMalloc(&n->xin, ts * 4 * vox(n, 0)) || cudaMalloc(&n->yout, 4 * 3 * vox(n, 0)) ||
      cudaMalloc(&n->g0, 4 * maxc) || cudaMalloc(&n->g1, 4 * maxc) || cudaMalloc(&n->ls, 16) ||
      cudaMalloc(&n->gy, 4 * 3 * vox(n, 0)) || cudaMallocHost(&n->ls_host, 16))
    return fail();
  cudaStream_t st = ctx->stream;
  NH_CUDA(ctx, cudaMemsetAsync(n->theta, 0, 4 * n->np, st));
  for (const Layer& y : n->L) {
    const int64_t nw = (int64_t)y.cout * y.cin * 27;
    k_init<<<blocks_for(nw), 256, 0, st>>>(nw, y.woff, sqrtf(2.f / (y.cin * 27.f)), seed, n->theta + y.woff);
    ctx->launches++;
  }
  NH_CUDA(ctx, cudaMemsetAsync(n->m1, 0, 4 * n->np, st));
  NH_CUDA(ctx, cudaMemsetAsync(n->m2, 0, 4 * n->np, st));
  nh_status s = refresh_compute_copy(n);
  if (s != NH_OK) { nh_net_destroy(n); return s; }
  NH_CUDA(ctx, cudaStreamSynchronize(st));
  *out = n;
  return NH_OK;
}

extern "C" nh_status nh_net_param_count(nh_net n, int64_t* count) {
  if (!n || !count) return NH_ERR_ARG;
  *count = n->np;
  return NH_OK;
}

extern "C" nh_status nh_net_get_params(nh_net n, float* host) {
  if (!n || !host) return NH_ERR_ARG;
  NH_CUDA(n->ctx, cudaMemcpyAsync(host, n->theta, 4 * n->np, cudaMemcpyDeviceToHost, n->ctx->stream));
  NH_CUDA(n->ctx, cudaStreamSynchronize(n->ctx->stream));
  return NH_OK;
}

extern "C" nh_status nh_net_set_params(nh_net n, const float* host) {
  if (!n || !host) return NH_ERR_ARG;
  NH_CUDA(n->ctx, cudaMemcpyAsync(n->theta, host, 4 * n->np, cudaMemcpyHostToDevice, n->ctx->stream));
  nh_status s = refresh_compute_copy(n);
  if (s != NH_OK) return s;
  NH_CUDA(n->ctx, cudaStreamSynchronize(n->ctx->stream));
  n->adam_t = 0;
  NH_CUDA(n->ctx, cudaMemset(n->m1, 0, 4 * n->np));
  NH_CUDA(n->ctx, cudaMemset(n->m2, 0, 4 * n->np));
  return NH_OK;
}

extern "C" nh_status nh_net_forward(nh_net n, const float* in, float* out) {
  if (!n || !in || !out) return NH_ERR_ARG;
  NH_CUDA(n->ctx, cudaSetDevice(n->ctx->device));
  return nh_net_forward_internal(n, in, out);
}

extern "C" nh_status nh_net_gradient(nh_net n, const float* in, const float* target, float* dparams, double* loss) {
  if (!n || !in || !target || !dparams) return NH_ERR_ARG;
  NH_CUDA(n->ctx, cudaSetDevice(n->ctx->device));
  cudaStream_t st = n->ctx->stream;
  nh_status s = nh_net_forward_internal(n, in, n->yout);
  if (s != NH_OK) return s;
  const int64_t ny = 3 * vox(n, 0);
  NH_CUDA(n->ctx, cudaMemsetAsync(n->ls, 0, 16, st));
  k_loss_sums<<<blocks_for(ny), 256, 0, st>>>(ny, n->yout, target, n->ls);
  k_loss_grad<<<blocks_for(ny), 256, 0, st>>>(ny, n->yout, target, n->ls, 1.f, n->gy);
  n->ctx->launches += 2;
  NH_CUDA(n->ctx, cudaMemsetAsync(n->grad, 0, 4 * n->np, st));
  s = n->bf16 ? backward_t<__nv_bfloat16>(n, n->gy) : backward_t<float>(n, n->gy);
  if (s != NH_OK) return s;
  NH_CUDA(n->ctx, cudaMemcpyAsync(dparams, n->grad, 4 * n->np, cudaMemcpyDeviceToDevice, st));
  if (loss) {
    NH_CUDA(n->ctx, cudaMemcpyAsync(n->ls_host, n->ls, 16, cudaMemcpyDeviceToHost, st));
    NH_CUDA(n->ctx, cudaStreamSynchronize(st));
    *loss = n->ls_host[0] / n->ls_host[1];
  }
  return NH_OK;
}

extern "C" nh_status nh_net_train_step(nh_net n, int batch, const float* in, const float* target, float lr,
                                       double* loss) {
  if (!n || !in || !target || batch < 1) return NH_ERR_ARG;
  NH_CUDA(n->ctx, cudaSetDevice(n->ctx->device));
  cudaStream_t st = n->ctx->stream;
  const int64_t n0 = vox(n, 0);
  NH_CUDA(n->ctx, cudaMemsetAsync(n->grad, 0, 4 * n->np, st));
  double tot = 0.0;
  for (int bi = 0; bi < batch; bi++) {
    nh_status s = nh_net_forward_internal(n, in + (int64_t)bi * 4 * n0, n->yout);
    if (s != NH_OK) return s;
    const float* t = target + (int64_t)bi * 3 * n0;
    NH_CUDA(n->ctx, cudaMemsetAsync(n->ls, 0, 16, st));
    k_loss_sums<<<blocks_for(3 * n0), 256, 0, st>>>(3 * n0, n->yout, t, n->ls);
    k_loss_grad<<<blocks_for(3 * n0), 256, 0, st>>>(3 * n0, n->yout, t, n->ls, 1.f / batch, n->gy);
    n->ctx->launches += 2;
    s = n->bf16 ? backward_t<__nv_bfloat16>(n, n->gy) : backward_t<float>(n, n->gy);
    if (s != NH_OK) return s;
    if (loss) {
      NH_CUDA(n->ctx, cudaMemcpyAsync(n->ls_host, n->ls, 16, cudaMemcpyDeviceToHost, st));
      NH_CUDA(n->ctx, cudaStreamSynchronize(st));
      tot += n->ls_host[0] / n->ls_host[1];
    }
  }
  n->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
  k_adam<<<blocks_for(n->np), 256, 0, st>>>(n->np, n->theta, n->grad, n->m1, n->m2, lr, b1, b2, 1e-8f, c1, c2);
  n->ctx->launches++;
  nh_status s = refresh_compute_copy(n);
  if (s != NH_OK) return s;
  if (loss) *loss = tot / batch;
  return NH_OK;
}

// p-multigrid transfer (Eq. mg_prolong):
//   prolongation  uf = sum_e E_f^T Lambda(m_f^-1) B_ctof E_c uc
//   restriction   rc = P^T rf      (restriction = prolongation transposed, Sec. III-B)
// B_ctof is the tensor product of the 1-D matrix that evaluates the coarse GLL
// Lagrange basis at the fine GLL nodes; m_f is the number of elements sharing a
// fine node.  One element per Pf*Pf threads, thread (a, b) owning a fine
// (x, y) node column; contractions by sum factorisation; scatter-add by atomics.
#include "nh_internal.cuh"

namespace {

template <int PC, int PF, typename T>
struct CtoF {
  T B[PF][PC];
};

__host__ __device__ constexpr int tepb(int PF) { return 128 / (PF * PF); }

template <int PF>
__device__ __forceinline__ int tix(int c, int k, int j, int i) {
  return ((c * PF + k) * PF + j) * PF + i;
}

template <int PC, int PF, typename T>
__global__ void __launch_bounds__(PF* PF* tepb(PF))
    k_prolong(int64_t ne, const int* __restrict__ emap_c, const int* __restrict__ emap_f,
              const T* __restrict__ inv_mult, const CtoF<PC, PF, T> tb, const T* __restrict__ uc,
              T* __restrict__ uf) {
  constexpr int EPB = tepb(PF), F2 = PF * PF, F3 = PF * PF * PF, C3 = PC * PC * PC;
  __shared__ T sm[EPB][2][3 * F3];
  const int t = threadIdx.x, el = t / F2, col = t - el * F2, a = col % PF, b = col / PF;
  const int64_t e = (int64_t)blockIdx.x * EPB + el;
  const bool live = e < ne;
  T* s1 = sm[el][0];
  T* s2 = sm[el][1];
  if (live && a < PC && b < PC) {
    T r[3][PC];
#pragma unroll
    for (int k = 0; k < PC; k++) {
      const int n = __ldg(&emap_c[e * C3 + (k * PC + b) * PC + a]);
#pragma unroll
      for (int c = 0; c < 3; c++) r[c][k] = uc[3 * (int64_t)n + c];
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int kf = 0; kf < PF; kf++) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < PC; k++) s += tb.B[kf][k] * r[c][k];
        s1[tix<PF>(c, kf, b, a)] = s;
      }
  }
  __syncthreads();
  if (live && a < PC) {
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int kf = 0; kf < PF; kf++) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < PC; j++) s += tb.B[b][j] * s1[tix<PF>(c, kf, j, a)];
        s2[tix<PF>(c, kf, b, a)] = s;
      }
  }
  __syncthreads();
  if (live) {
#pragma unroll
    for (int kf = 0; kf < PF; kf++) {
      const int n = __ldg(&emap_f[e * F3 + (kf * PF + b) * PF + a]);
      const T w = inv_mult[n];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        T s = T(0);
#pragma unroll
        for (int i = 0; i < PC; i++) s += tb.B[a][i] * s2[tix<PF>(c, kf, b, i)];
        atomicAdd(&uf[3 * (int64_t)n + c], w * s);
      }
    }
  }
}

template <int PC, int PF, typename T>
__global__ void __launch_bounds__(PF* PF* tepb(PF))
    k_restrict(int64_t ne, const int* __restrict__ emap_c, const int* __restrict__ emap_f,
               const T* __restrict__ inv_mult, const CtoF<PC, PF, T> tb, const T* __restrict__ rf,
               T* __restrict__ rc) {
  constexpr int EPB = tepb(PF), F2 = PF * PF, F3 = PF * PF * PF, C3 = PC * PC * PC;
  __shared__ T sm[EPB][2][3 * F3];
  const int t = threadIdx.x, el = t / F2, col = t - el * F2, a = col % PF, b = col / PF;
  const int64_t e = (int64_t)blockIdx.x * EPB + el;
  const bool live = e < ne;
  T* s1 = sm[el][0];
  T* s2 = sm[el][1];
  if (live) {
    T r[3][PF];
#pragma unroll
    for (int kf = 0; kf < PF; kf++) {
      const int n = __ldg(&emap_f[e * F3 + (kf * PF + b) * PF + a]);
      const T w = inv_mult[n];
#pragma unroll
      for (int c = 0; c < 3; c++) r[c][kf] = w * rf[3 * (int64_t)n + c];
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < PC; k++) {
        T s = T(0);
#pragma unroll
        for (int kf = 0; kf < PF; kf++) s += tb.B[kf][k] * r[c][kf];
        s1[tix<PF>(c, k, b, a)] = s;
      }
  }
  __syncthreads();
  if (live && b < PC) {
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < PC; k++) {
        T s = T(0);
#pragma unroll
        for (int jf = 0; jf < PF; jf++) s += tb.B[jf][b] * s1[tix<PF>(c, k, jf, a)];
        s2[tix<PF>(c, k, b, a)] = s;
      }
  }
  __syncthreads();
  if (live && a < PC && b < PC) {
#pragma unroll
    for (int k = 0; k < PC; k++) {
      const int n = __ldg(&emap_c[e * C3 + (k * PC + b) * PC + a]);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        T s = T(0);
#pragma unroll
        for (int i = 0; i < PF; i++) s += tb.B[i][a] * s2[tix<PF>(c, k, b, i)];
        atomicAdd(&rc[3 * (int64_t)n + c], s);
      }
    }
  }
}

template <int PC, int PF, typename T>
cudaError_t run(int dir, int64_t ne, const int* ec, const int* ef, const T* im, const void* in, void* out,
                const double* ctof, cudaStream_t s) {
  CtoF<PC, PF, T> tb;
  for (int i = 0; i < PF; i++)
    for (int j = 0; j < PC; j++) tb.B[i][j] = (T)ctof[i * PC + j];
  constexpr int EPB = tepb(PF);
  const int64_t blocks = (ne + EPB - 1) / EPB;
  if (blocks == 0) return cudaSuccess;
  if (dir == 0)
    k_prolong<PC, PF, T><<<(unsigned)blocks, PF * PF * EPB, 0, s>>>(ne, ec, ef, im, tb, (const T*)in, (T*)out);
  else
    k_restrict<PC, PF, T><<<(unsigned)blocks, PF * PF * EPB, 0, s>>>(ne, ec, ef, im, tb, (const T*)in, (T*)out);
  return cudaGetLastError();
}

template <int PC, int PF>
cudaError_t run_prec(nh_prec prec, int dir, int64_t ne, const int* ec, const int* ef, const double* im,
                     const float* imf, const void* in, void* out, const double* ctof, cudaStream_t s) {
  if (prec == NH_F64) return run<PC, PF, double>(dir, ne, ec, ef, im, in, out, ctof, s);
  return run<PC, PF, float>(dir, ne, ec, ef, imf, in, out, ctof, s);
}

}  // namespace

cudaError_t nh_launch_transfer(int Pc, int Pf, nh_prec prec, int dir, int64_t ne, const int* ec, const int* ef,
                               const double* im, const float* imf, const void* in, void* out, const double* ctof,
                               cudaStream_t s) {
#define NH_T(A, B) \
  if (Pc == A && Pf == B) return run_prec<A, B>(prec, dir, ne, ec, ef, im, imf, in, out, ctof, s);
  NH_T(2, 3) NH_T(2, 4) NH_T(2, 5) NH_T(3, 4) NH_T(3, 5) NH_T(4, 5)
#undef NH_T
  return cudaErrorInvalidValue;
}

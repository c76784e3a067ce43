// Float-float ("double-single") arithmetic: a value is the unevaluated sum h + l
// of two floats with |l| <= ulp(h) / 2, about 48 significant bits.  Built from the
// error-free transformations TwoSum (Knuth), Fast2Sum (Dekker, |a| >= |b|) and
// the FMA form of TwoProduct, with the "sloppy" addition (one TwoSum on the high
// parts, the low parts added and renormalised): error ~ 2^-47 (|a| + |b|).
// It lets the FP64-accurate Jacobian run on B300's FP32 pipes, which issue 64
// FMAs for each FP64 FMA.  Compile without fast-math: the transformations rely
// on IEEE round-to-nearest of each float operation.
#pragma once
#include <cuda_runtime.h>

struct ff {
  float h, l;
  __host__ __device__ __forceinline__ ff() : h(0.f), l(0.f) {}
  __host__ __device__ __forceinline__ ff(float a, float b) : h(a), l(b) {}
  __host__ __device__ __forceinline__ ff(double d) {
    h = (float)d;
    l = (float)(d - (double)h);
  }
  __host__ __device__ __forceinline__ ff(int i) : ff((double)i) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff(s, e);
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return ff(s, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.h, b.h);
  return ff_fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.h, -a.l); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + ff(-b.h, -b.l); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) {
  a = a + b;
  return a;
}

__device__ __forceinline__ ff& operator*=(ff& a, ff b) {
  a = a * b;
  return a;
}

// s + a * b: TwoProduct of the high parts with the cross terms folded into its
// error, one TwoSum of the high parts, then a single Fast2Sum renormalisation
// (15 float operations against 18 for a separate product and sum).
__device__ __forceinline__ ff ff_madd(ff s, ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const ff t = ff_two_sum(s.h, p);
  return ff_fast_two_sum(t.h, t.l + (s.l + e));
}

// Compensated dot product in the manner of Dot2 (Ogita, Rump and Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005), extended to float-float
// operands: each term a * b is split by TwoProduct (cross terms a.h b.l + a.l b.h
// folded into its error), the high parts are summed by TwoSum, and every error
// term is collected in one running low part (h, l) that is renormalised once, at
// the end (TwoSum).  12 float operations per term against 15 for ff_madd, and the
// error stays ~n^2 2^-48 of sum |a b| for n terms.
struct ffdot {
  float h, l;
};

__device__ __forceinline__ ffdot ffd_first(ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ffdot{p, e};
}

__device__ __forceinline__ void ffd_add(ffdot& s, ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const ff t = ff_two_sum(s.h, p);
  s.h = t.h;
  s.l = s.l + (t.l + e);
}

__device__ __forceinline__ ff ffd_done(ffdot s) { return ff_two_sum(s.h, s.l); }

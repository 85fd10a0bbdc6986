// Double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 48 bits of significand.
// The building blocks are the classical error-free transformations:
//   TwoSum (Knuth): s = fl(a + b) and the exact error e, a + b = s + e;
//   Fast2Sum (Dekker): the same when |a| >= |b|;
//   TwoProd via FMA: p = fl(a b), e = fma(a, b, -p), a b = p + e.
// Addition follows the accurate double-word sum (two TwoSums, two Fast2Sums)
// analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017); multiplication
// is the FMA-based double-word product of the same paper. Every operation uses
// explicit round-to-nearest intrinsics so the compiler cannot contract or
// reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace mdet {

struct df32 {
  float hi, lo;
  __host__ __device__ df32() {}
  __host__ __device__ df32(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df32(int v) : hi((float)v), lo(0.0f) {}
};

static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

static __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

static __device__ __forceinline__ df32 df_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

static __device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

static __device__ __forceinline__ df32 operator+(df32 x, df32 y) {
  float sh, sl, th, tl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  float vh, vl;
  fast_two_sum(sh, __fadd_rn(sl, th), vh, vl);
  float zh, zl;
  fast_two_sum(vh, __fadd_rn(tl, vl), zh, zl);
  return {zh, zl};
}

static __device__ __forceinline__ df32 operator-(df32 x) { return {-x.hi, -x.lo}; }

static __device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }

static __device__ __forceinline__ df32 operator*(df32 x, df32 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return {s, t};
}

}  // namespace mdet

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

// The rare paths of the bit-level conversions below, out of line so that the compiler
// cannot if-convert their FP64 conversions into the common path, where they would take
// the FP64 pipe on every call.
static __device__ __noinline__ df32 df_from_double_slow(double x) { return df_from_double(x); }
static __device__ __noinline__ double df_to_double_slow(float hi, float lo) { return (double)hi + (double)lo; }

// The same split from the bits of x with integer and FP32 instructions only:
// hi keeps the sign, the exponent and the 23 leading mantissa bits (truncated),
// lo the 29 remaining bits (rounded to FP32, so hi + lo = x (1 + d), |d| <= 2^-47).
// Outside 2^-74 <= |x| < 2^128 (and for Inf or NaN) it falls back to the
// conversions above.
static __device__ __forceinline__ df32 df_from_bits(long long b) {
  const unsigned hw = (unsigned)((unsigned long long)b >> 32), lw = (unsigned)b;
  const int fe = (int)((hw >> 20) & 0x7ff) - 896;  // FP32 biased exponent of x
  if (fe < 53 || fe > 254) return df_from_double_slow(__longlong_as_double(b));
  const unsigned sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // lo = (lw mod 2^29) 2^(e - 1075), e the FP64 biased exponent: 2^(fe - 179) as an FP32 scale
  const float lo = __uint2float_rn(lw & 0x1fffffffu) * __uint_as_float((unsigned)(fe - 52) << 23);
  return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

static __device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

// hi + lo as an FP64 number with integer instructions only (no FP64-pipe work):
// the significand of hi goes to bits 29..52 of a 64-bit integer, lo is aligned
// to the same unit (its bits below the unit truncated), the two are added and
// the sum is renormalised by at most one position. The result is within one FP64
// ulp of hi + lo (|lo| <= ulp(hi)/2). A zero, subnormal or non-finite hi takes
// the conversions above.
static __device__ __forceinline__ double df_to_double_int(df32 a) {
  const unsigned uh = __float_as_uint(a.hi), ul = __float_as_uint(a.lo);
  const int eh = (int)((uh >> 23) & 0xffu);
  if (eh == 0 || eh == 0xff) return df_to_double_slow(a.hi, a.lo);
  long long x = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;
  if (uh >> 31) x = -x;
  const int el = (int)((ul >> 23) & 0xffu);
  if ((ul & 0x7fffffffu) != 0u && el != 0xff) {
    const long long ml = (long long)((ul & 0x7fffffu) | (el ? 0x800000u : 0u));
    const int sh = (el ? el : 1) - eh + 29;  // <= 5 since |lo| <= ulp(hi) / 2
    long long l = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> -sh) : 0LL);
    x += (ul >> 31) ? -l : l;
  }
  const unsigned long long sgn = x < 0 ? 0x8000000000000000ULL : 0ULL;
  unsigned long long m = (unsigned long long)(x < 0 ? -x : x);
  int e = eh + 896;  // FP64 biased exponent of a significand in [2^52, 2^53)
  if (m >> 53) {
    m >>= 1;
    e++;
  } else if (!(m >> 52)) {
    m <<= 1;
    e--;
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)e << 52) | (m & 0xfffffffffffffULL)));
}

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

// Compensated sum of products of double-float numbers: the dot product Dot2 of Ogita,
// Rump and Oishi (SIAM J. Sci. Comput. 26, 2005) with double-float inputs. Each term
// x y adds its leading product hi_x hi_y into the running FP32 sum s through TwoSum; the
// product's rounding error (from FMA), the cross terms hi_x lo_y + lo_x hi_y and TwoSum's
// error go into a second FP32 word c. The pair (s, c) carries the sum with an error of
// order n^2 2^-48 sum |x y| like the double-float operations above, at about 12 FP32
// instructions per term instead of 27 for a double-float product and sum.
struct df_dot {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(df32 x, df32 y) {
    const float p = __fmul_rn(x.hi, y.hi);
    const float pe = __fmaf_rn(x.hi, y.hi, -p);
    const float cross = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, __fadd_rn(pe, cross)));
  }
  __device__ __forceinline__ void sub(df32 x, df32 y) { add(df32(-x.hi, -x.lo), y); }
  // the sum as a normalised double-float pair
  __device__ __forceinline__ df32 value() const {
    float h, l;
    two_sum(s, c, h, l);
    return {h, l};
  }
};

// exp(t) for t <= 0 in double-float. Cody-Waite reduction t = k ln2 + r with
// ln2 split into three floats of 16, 24 and 24 significant bits (k * kLn2a is
// exact for |k| < 256 and k * kLn2b is made exact with TwoProd), so r carries
// the full double-float accuracy; |r| <= ln2/2. exp(r) is the Taylor series to
// degree 13 (truncation below 5e-18 relative) in Horner form with 1/n! as
// double-float constants, then scaled by 2^k. Arguments below -87 (results
// below the FP32 normal range) return 0.
__device__ __constant__ static const float kLn2a = 0x1.62e4p-1f;       // ln 2, leading 16 bits
__device__ __constant__ static const float kLn2b = 0x1.7f7d1cp-20f;    // next 24 bits
__device__ __constant__ static const float kLn2c = 0x1.ef357ap-45f;    // next 24 bits
__device__ __constant__ static const float kInvFact[14][2] = {          // 1/n! as (hi, lo)
    {0x1p+0f, 0.0f},
    {0x1p+0f, 0.0f},
    {0x1p-1f, 0.0f},
    {0x1.555556p-3f, -0x1.555556p-28f},
    {0x1.555556p-5f, -0x1.555556p-30f},
    {0x1.111112p-7f, -0x1.dddddep-32f},
    {0x1.6c16c2p-10f, -0x1.27d27ep-35f},
    {0x1.a01a02p-13f, -0x1.7f97fap-39f},
    {0x1.a01a02p-16f, -0x1.7f97fap-42f},
    {0x1.71de3ap-19f, 0x1.55b1ccp-45f},
    {0x1.27e4fcp-22f, -0x1.10ec14p-47f},
    {0x1.ae6456p-26f, 0x1.fd5138p-52f},
    {0x1.1eed8ep-29f, 0x1.ff1b12p-54f},
    {0x1.612462p-33f, -0x1.8af25ep-58f}};

static __device__ __forceinline__ df32 df_exp_nonpos(df32 t) {
  if (!(t.hi > -87.0f)) return df32(0.0f, 0.0f);
  const float kf = rintf(__fmul_rn(t.hi, 1.44269504f));
  // r = t - k ln2, each piece of k ln2 exact in double-float
  df32 r = t + df32(__fmul_rn(-kf, kLn2a), 0.0f);
  {
    const float p = __fmul_rn(-kf, kLn2b);
    const float e = __fmaf_rn(-kf, kLn2b, -p);
    r = r + df32(p, e);
  }
  r = r + df32(__fmul_rn(-kf, kLn2c), 0.0f);
  df32 p(kInvFact[13][0], kInvFact[13][1]);
#pragma unroll
  for (int n = 12; n >= 0; n--) p = p * r + df32(kInvFact[n][0], kInvFact[n][1]);
  const int k = (int)kf;
  return df32(ldexpf(p.hi, k), ldexpf(p.lo, k));
}

}  // namespace mdet

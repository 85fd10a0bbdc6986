// Device helpers shared by the FP64 and mixed-precision kernels.
#pragma once

#include <cuda_runtime.h>

#include "df32.cuh"
#include "mdet_internal.h"

namespace mdet {

// |x| as an FP32 value, taken from the high word of the FP64 number (its
// exponent and 20 leading mantissa bits, so within 2^-20 relative), clamped to
// [0, FLT_MAX]: integer operations only, no FP64-to-FP32 conversion, for the
// magnitude sums of the error estimate.
static __device__ __forceinline__ float abs_f32_of(double x) {
  int t = (__double2hiint(x) & 0x7fffffff) - (896 << 20);  // rebias the exponent from 1023 to 127
  t = min(max(t, 0), 0x0fefffff);
  return __int_as_float(t << 3);
}

// FP32 <-> FP64 by the bits, with integer instructions only (no conversion on the FP64
// pipe). f32_of_f64_bits: x in the FP32 normal range, sign, exponent and the 23 leading
// mantissa bits (truncated: relative error below 2^-23). f64_of_f32_bits: a normal FP32
// value, exactly.
static __device__ __forceinline__ float f32_of_f64_bits(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  return __uint_as_float((hw & 0x80000000u) | ((((hw >> 20) & 0x7ffu) - 896u) << 23) | ((hw & 0xfffffu) << 3) |
                         (lw >> 29));
}
static __device__ __forceinline__ double f64_of_f32_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned hw = (u & 0x80000000u) | ((((u >> 23) & 0xffu) + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hw, (int)(u << 29));
}

// x added into a three-word FP32 accumulator (w1, w2, w3 in shared memory), the FP64
// epilogue's W. x is split exactly by its bits into 24 + 24 + 5 significand bits (hi, mid,
// lo); hi and then the carried error plus mid are added with atomics whose returned old
// values give, by TwoSum, the exact rounding errors of those additions, which go to the
// next word. Only the additions into w3 round, at about 2^-72 of the accumulated value, so
// the sum is more accurate than FP64 accumulation, and no instruction runs on the FP64
// pipe (FP64 shared-memory atomics do). |x| outside [2^-74, 2^128), zero, Inf and NaN
// take the out-of-line path.
static __device__ __noinline__ void acc3_add_slow(float* w1, float* w2, float* w3, double x) {
  const float hi = __double2float_rn(x);
  const double r = x - (double)hi;
  const float mid = __double2float_rn(r);
  const float lo = __double2float_rn(r - (double)mid);
  atomicAdd(w1, hi);
  atomicAdd(w2, mid);
  atomicAdd(w3, lo);
}
static __device__ __forceinline__ void acc3_add(float* w1, float* w2, float* w3, double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const int fe = (int)((hw >> 20) & 0x7ffu) - 896;  // FP32 biased exponent of hi
  if (fe < 53 || fe > 254) {
    acc3_add_slow(w1, w2, w3, x);
    return;
  }
  const unsigned sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // mid = bits 28..5 of the low word times 2^(e - 1070), lo = bits 4..0 times 2^(e - 1075)
  // (e the FP64 biased exponent): both exact
  const float mid = __uint_as_float(
      __float_as_uint(__uint2float_rn((lw >> 5) & 0xffffffu) * __uint_as_float((unsigned)(fe - 47) << 23)) | sign);
  const float lo =
      __uint_as_float(__float_as_uint(__uint2float_rn(lw & 0x1fu) * __uint_as_float((unsigned)(fe - 52) << 23)) | sign);
  float s, e1, t, e2, e3;
  two_sum(atomicAdd(w1, hi), hi, s, e1);
  two_sum(e1, mid, t, e2);
  two_sum(atomicAdd(w2, t), t, s, e3);
  atomicAdd(w3, __fadd_rn(__fadd_rn(e2, e3), lo));
}

// Out of line, so that the compiler cannot if-convert it into the common path below.
static __device__ __noinline__ double inv_sqrt_slow(double x) { return 1.0 / sqrt(x); }

// 1/sqrt(x) for the Coulomb sums of the local energy: an FP32 estimate refined by two
// Newton-Raphson steps for the reciprocal square root, y <- y + y (1 - x y^2) / 2, in
// FP64. A step turns a relative error e into about 3 e^2 / 2, so from the FP32
// estimate (e below 2^-21) two steps leave only the roundings of the last one, a few
// ulp. The range test is on the bits; arguments outside [2^-99, 2^100) (zero,
// negative, subnormal, huge, Inf, NaN) take 1 / sqrt(x).
static __device__ __forceinline__ double coulomb_inv_r(double x) {
  const unsigned se = (unsigned)__double2hiint(x) >> 20;  // sign and biased exponent
  if (se <= 1023u - 100u || se >= 1023u + 100u) return inv_sqrt_slow(x);
  double y = f64_of_f32_bits(rsqrtf(f32_of_f64_bits(x)));
  double e = fma(-x * y, y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-x * y, y, 1.0);
  return fma(0.5 * y, e, y);
}

static __device__ __forceinline__ double ipow_d(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; i++) r *= x;
  return r;
}

// Determinant of a k x k matrix (k <= 4), row-major in m[4][4].
template <class F>
static __device__ __forceinline__ F small_det(int k, const F (&m)[4][4]) {
  if (k == 0) return F(1);
  if (k == 1) return m[0][0];
  if (k == 2) return m[0][0] * m[1][1] - m[0][1] * m[1][0];
  if (k == 3)
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
  // Laplace expansion along rows 0 and 1: 2 x 2 minors of rows (0,1) and (2,3)
  F s01 = m[0][0] * m[1][1] - m[0][1] * m[1][0];
  F s02 = m[0][0] * m[1][2] - m[0][2] * m[1][0];
  F s03 = m[0][0] * m[1][3] - m[0][3] * m[1][0];
  F s12 = m[0][1] * m[1][2] - m[0][2] * m[1][1];
  F s13 = m[0][1] * m[1][3] - m[0][3] * m[1][1];
  F s23 = m[0][2] * m[1][3] - m[0][3] * m[1][2];
  F c01 = m[2][0] * m[3][1] - m[2][1] * m[3][0];
  F c02 = m[2][0] * m[3][2] - m[2][2] * m[3][0];
  F c03 = m[2][0] * m[3][3] - m[2][3] * m[3][0];
  F c12 = m[2][1] * m[3][2] - m[2][2] * m[3][1];
  F c13 = m[2][1] * m[3][3] - m[2][3] * m[3][1];
  F c23 = m[2][2] * m[3][3] - m[2][3] * m[3][2];
  return s01 * c23 - s02 * c13 + s03 * c12 + s12 * c03 - s13 * c02 + s23 * c01;
}

// Cofactors cof[alpha][beta] = (-1)^(alpha+beta) det(minor without row alpha, column beta), k <= 4.
template <class F>
static __device__ __forceinline__ void small_cof(int k, const F (&m)[4][4], F (&cof)[4][4]) {
  if (k == 1) {
    cof[0][0] = F(1);
    return;
  }
  if (k == 2) {
    cof[0][0] = m[1][1];
    cof[0][1] = -m[1][0];
    cof[1][0] = -m[0][1];
    cof[1][1] = m[0][0];
    return;
  }
  if (k == 3) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const int r0 = a == 0 ? 1 : 0, r1 = a == 2 ? 1 : 2;
        const int c0 = b == 0 ? 1 : 0, c1 = b == 2 ? 1 : 2;
        F d = m[r0][c0] * m[r1][c1] - m[r0][c1] * m[r1][c0];
        cof[a][b] = ((a + b) & 1) ? -d : d;
      }
    return;
  }
  // k == 4: each 3 x 3 minor is expanded along the row that shares its pair
  // ({0,1} or {2,3}) with the removed row, using precomputed 2 x 2 minors of the other pair.
  F top[4][4], bot[4][4];  // 2 x 2 minors of rows (0,1) and (2,3) for column pairs (x < y)
#pragma unroll
  for (int x = 0; x < 4; x++)
#pragma unroll
    for (int y = x + 1; y < 4; y++) {
      top[x][y] = m[0][x] * m[1][y] - m[0][y] * m[1][x];
      bot[x][y] = m[2][x] * m[3][y] - m[2][y] * m[3][x];
    }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int rho = a < 2 ? 1 - a : 5 - a;  // the remaining row of the removed row's pair
#pragma unroll
    for (int b = 0; b < 4; b++) {
      int cols[3];
      int q = 0;
#pragma unroll
      for (int x = 0; x < 4; x++)
        if (x != b) cols[q++] = x;
      // det of the 3 x 3 minor = sum_t (-1)^t m[rho][cols[t]] * D2(other two columns)
      F d = F(0);
#pragma unroll
      for (int t = 0; t < 3; t++) {
        const int x = t == 0 ? cols[1] : cols[0];
        const int y = t == 2 ? cols[1] : cols[2];
        const F d2 = a < 2 ? bot[x][y] : top[x][y];
        const F term = m[rho][cols[t]] * d2;
        d = (t & 1) ? d - term : d + term;
      }
      cof[a][b] = ((a + b) & 1) ? -d : d;
    }
  }
}


// a d - b c with double-float products and the accurate double-word difference. The 2 x 2
// minors are where an ill-conditioned table cancels; as a compensated dot product (df_dot)
// their error on the worst walkers of a 2,100-walker test set grew 6.5-fold, past the
// first-order error estimate, so they keep the accurate sum.
static __device__ __forceinline__ df32 df_minor2(df32 a, df32 b, df32 c, df32 d) { return a * d - b * c; }

// Determinant of a k x k double-float matrix (k <= 4), as small_det, with the final
// expansion over the 2 x 2 minors as a compensated dot product (df_dot).
static __device__ __forceinline__ df32 small_det_dot(int k, const df32 (&m)[4][4]) {
  if (k == 0) return df32(1.0f, 0.0f);
  if (k == 1) return m[0][0];
  if (k == 2) return df_minor2(m[0][0], m[0][1], m[1][0], m[1][1]);
  df_dot d;
  if (k == 3) {  // expansion along row 0
    d.add(m[0][0], df_minor2(m[1][1], m[1][2], m[2][1], m[2][2]));
    d.sub(m[0][1], df_minor2(m[1][0], m[1][2], m[2][0], m[2][2]));
    d.add(m[0][2], df_minor2(m[1][0], m[1][1], m[2][0], m[2][1]));
    return d.value();
  }
  // Laplace expansion along rows 0 and 1: 2 x 2 minors of rows (0,1) and (2,3)
  auto s = [&](int x, int y) { return df_minor2(m[0][x], m[0][y], m[1][x], m[1][y]); };
  auto c = [&](int x, int y) { return df_minor2(m[2][x], m[2][y], m[3][x], m[3][y]); };
  d.add(s(0, 1), c(2, 3));
  d.sub(s(0, 2), c(1, 3));
  d.add(s(0, 3), c(1, 2));
  d.add(s(1, 2), c(0, 3));
  d.sub(s(1, 3), c(0, 2));
  d.add(s(2, 3), c(0, 1));
  return d.value();
}

// Cofactors of a K x K double-float matrix (K <= 4, compile time), as small_cof: the
// expansions of the 3 x 3 minors over the 2 x 2 ones (df_minor2) are compensated dot
// products (df_dot) instead of double-float products and sums.
template <int K>
static __device__ __forceinline__ void small_cof_dot(const df32 (&m)[4][4], df32 (&cof)[4][4]) {
  if constexpr (K == 1) {
    cof[0][0] = df32(1.0f, 0.0f);
  } else if constexpr (K == 2) {
    cof[0][0] = m[1][1];
    cof[0][1] = -m[1][0];
    cof[1][0] = -m[0][1];
    cof[1][1] = m[0][0];
  } else if constexpr (K == 3) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const int r0 = a == 0 ? 1 : 0, r1 = a == 2 ? 1 : 2;
        const int c0 = b == 0 ? 1 : 0, c1 = b == 2 ? 1 : 2;
        const df32 d = df_minor2(m[r0][c0], m[r0][c1], m[r1][c0], m[r1][c1]);
        cof[a][b] = ((a + b) & 1) ? -d : d;
      }
  } else {
    // 2 x 2 minors of rows (0,1) and (2,3) for column pairs (x < y), then each 3 x 3 minor
    // expanded along the row that shares its pair with the removed row
    df32 top[4][4], bot[4][4];
#pragma unroll
    for (int x = 0; x < 4; x++)
#pragma unroll
      for (int y = x + 1; y < 4; y++) {
        top[x][y] = df_minor2(m[0][x], m[0][y], m[1][x], m[1][y]);
        bot[x][y] = df_minor2(m[2][x], m[2][y], m[3][x], m[3][y]);
      }
#pragma unroll
    for (int a = 0; a < 4; a++) {
      const int rho = a < 2 ? 1 - a : 5 - a;
#pragma unroll
      for (int b = 0; b < 4; b++) {
        int cols[3];
        int q = 0;
#pragma unroll
        for (int x = 0; x < 4; x++)
          if (x != b) cols[q++] = x;
        df_dot d;
#pragma unroll
        for (int t = 0; t < 3; t++) {
          const int x = t == 0 ? cols[1] : cols[0];
          const int y = t == 2 ? cols[1] : cols[2];
          const df32 d2 = a < 2 ? bot[x][y] : top[x][y];
          if (t & 1)
            d.sub(m[rho][cols[t]], d2);
          else
            d.add(m[rho][cols[t]], d2);
        }
        const df32 v = d.value();
        cof[a][b] = ((a + b) & 1) ? -v : v;
      }
    }
  }
}

// Values, gradient and Laplacian of the (l+1)(l+2)/2 Cartesian AOs of one shell
// at one point (FP64). AO chi = P(x, y, z) f(r^2) with P = x^a y^b z^c of degree
// l and f(s) = sum_p c_p exp(-alpha_p s):
//   d_x chi = P_x f + 2 x P f',   Lap chi = (Lap P) f + P ((4 l + 6) f' + 4 s f'')
// (Euler: x P_x + y P_y + z P_z = l P). store(c, q, value) receives component
// c (0 value, 1..3 gradient, 4 Laplacian) of the q-th AO of the shell, in the
// order xx, xy, xz, yy, yz, zz (a descending, then b descending).
template <class Store>
static __device__ __forceinline__ void ao_shell_values(const DevProblem& P, int s, const double* r, Store store) {
  const int l = P.shell_l[s];
  const double* C = P.nuc_xyz + 3 * P.shell_center[s];
  const double x = r[0] - C[0], y = r[1] - C[1], z = r[2] - C[2];
  const double s2 = x * x + y * y + z * z;
  double f0 = 0, f1 = 0, f2 = 0;
  const int p0 = P.shell_prim0[s], np = P.shell_nprim[s];
  for (int p = 0; p < np; p++) {
    const double al = P.alpha[p0 + p], cf = P.coef[p0 + p];
    const double ex = cf * exp(-al * s2);
    f0 += ex;
    f1 -= al * ex;
    f2 += al * al * ex;
  }
  const double lapf = (4.0 * l + 6.0) * f1 + 4.0 * s2 * f2;
  int q = 0;
  for (int a = l; a >= 0; a--)
    for (int b = l - a; b >= 0; b--, q++) {
      const int cc = l - a - b;
      const double xa = ipow_d(x, a), yb = ipow_d(y, b), zc = ipow_d(z, cc);
      const double P0 = xa * yb * zc;
      const double Px = a ? a * ipow_d(x, a - 1) * yb * zc : 0.0;
      const double Py = b ? b * xa * ipow_d(y, b - 1) * zc : 0.0;
      const double Pz = cc ? cc * xa * yb * ipow_d(z, cc - 1) : 0.0;
      double lapP = 0.0;
      if (a >= 2) lapP += a * (a - 1) * ipow_d(x, a - 2) * yb * zc;
      if (b >= 2) lapP += b * (b - 1) * xa * ipow_d(y, b - 2) * zc;
      if (cc >= 2) lapP += cc * (cc - 1) * xa * yb * ipow_d(z, cc - 2);
      store(0, q, P0 * f0);
      store(1, q, Px * f0 + 2.0 * x * P0 * f1);
      store(2, q, Py * f0 + 2.0 * y * P0 * f1);
      store(3, q, Pz * f0 + 2.0 * z * P0 * f1);
      store(4, q, lapP * f0 + P0 * lapf);
    }
}

// The same AO values in double-float arithmetic on the FP32 pipe (mixed
// path): coordinates, exponents and coefficients arrive as (hi, lo) pairs and
// exp is df_exp_nonpos. Same formulas, component order and store() contract.
static __device__ __forceinline__ df32 df_ipow(df32 x, int n) {
  df32 r(1);
  for (int i = 0; i < n; i++) r = r * x;
  return r;
}

template <class Store>
static __device__ __forceinline__ void ao_shell_values_df(const DevProblem& P, int s, const df32* r, Store store) {
  const int l = P.shell_l[s];
  const float2* C = P.nuc_df + 3 * P.shell_center[s];
  const df32 x = r[0] - df32(C[0].x, C[0].y);
  const df32 y = r[1] - df32(C[1].x, C[1].y);
  const df32 z = r[2] - df32(C[2].x, C[2].y);
  const df32 s2 = x * x + y * y + z * z;
  df32 f0(0), f1(0), f2(0);
  const int p0 = P.shell_prim0[s], np = P.shell_nprim[s];
  for (int p = 0; p < np; p++) {
    const float2 a2 = P.alpha_df[p0 + p], c2 = P.coef_df[p0 + p];
    const df32 al(a2.x, a2.y), cf(c2.x, c2.y);
    const df32 ex = cf * df_exp_nonpos(-(al * s2));
    const df32 ae = al * ex;
    f0 = f0 + ex;
    f1 = f1 - ae;
    f2 = f2 + al * ae;
  }
  const df32 lapf = df32(4 * l + 6) * f1 + df32(4) * (s2 * f2);
  const df32 two(2);
  int q = 0;
  for (int a = l; a >= 0; a--)
    for (int b = l - a; b >= 0; b--, q++) {
      const int cc = l - a - b;
      const df32 xa = df_ipow(x, a), yb = df_ipow(y, b), zc = df_ipow(z, cc);
      const df32 yz = yb * zc;
      const df32 P0 = xa * yz;
      const df32 Px = a ? df32(a) * (df_ipow(x, a - 1) * yz) : df32(0);
      const df32 Py = b ? df32(b) * (xa * df_ipow(y, b - 1) * zc) : df32(0);
      const df32 Pz = cc ? df32(cc) * (xa * yb * df_ipow(z, cc - 1)) : df32(0);
      df32 lapP(0);
      if (a >= 2) lapP = lapP + df32(a * (a - 1)) * (df_ipow(x, a - 2) * yz);
      if (b >= 2) lapP = lapP + df32(b * (b - 1)) * (xa * df_ipow(y, b - 2) * zc);
      if (cc >= 2) lapP = lapP + df32(cc * (cc - 1)) * (xa * yb * df_ipow(z, cc - 2));
      const df32 P0f1 = two * (P0 * f1);
      store(0, q, P0 * f0);
      store(1, q, Px * f0 + x * P0f1);
      store(2, q, Py * f0 + y * P0f1);
      store(3, q, Pz * f0 + z * P0f1);
      store(4, q, lapP * f0 + P0 * lapf);
    }
}

}  // namespace mdet

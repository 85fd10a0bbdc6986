// Mixed-precision kernels: the orbital product and the determinant ratios on
// the FP32 pipe with double-float (compensated) arithmetic (df32.cuh). The
// reference LU, log|D_ref|, the tables T = A Phi and the CI contraction stay in
// FP64 (mdet_kernels.cu).
//
// Why not FP32: the ratio-table method loses about log10 cond(S_ref) digits in
// every k x k determinant of table entries, and on the chlorine-like walkers
// cond(S_ref) reaches 1e6 at the 99th percentile; plain FP32 (or BF16/TF32 with
// FP32 accumulation) then misses a 1e-5 relative target, while double-float
// keeps about 48 significand bits at a fraction of the FP64 cost on GB300.
#include <cmath>

#include "df32.cuh"
#include "mdet_device.cuh"
#include "mdet_internal.h"

namespace mdet {

namespace {

// Orbitals. grid (n_walk, ceil(n_elec / kECm)), block 128. AO values and
// derivatives are formed in double-float arithmetic on the FP32 pipe
// (ao_shell_values_df), stored as FP32 pairs x = xh + xl in shared memory, and
// multiplied by B = Bh + Bl with a compensated dot product: the leading
// product xh*bh is made exact with an FMA (TwoProd), accumulated with TwoSum,
// and the cross terms xh*bl + xl*bh plus all rounding errors go into a second
// FP32 accumulator (the Dot2 scheme of Ogita, Rump and Oishi, extended to split
// inputs). Phi = s + c is stored as a renormalised double-float pair.
template <int kECm>
__global__ void __launch_bounds__(128) k_mo_mixed(DevProblem P, float2* __restrict__ phi,
                                                  const double* __restrict__ R) {
  extern __shared__ float smf[];
  __shared__ df32 rdf[kECm][3];
  const int K = P.n_ao, M = P.n_mo, N = P.n_elec;
  const int64_t w = blockIdx.x;
  const int e_begin = blockIdx.y * kECm;
  const int ne = min(kECm, N - e_begin);
  float* Xh = smf;                  // [(c * kECm + e) * K + mu]
  float* Xl = smf + 5 * kECm * K;
  if (threadIdx.x < 3 * ne) {
    const int e = threadIdx.x / 3, d = threadIdx.x - 3 * e;
    rdf[e][d] = df_from_double(R[(w * N + e_begin + e) * 3 + d]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kECm * P.n_shell; t += blockDim.x) {
    const int e = t / P.n_shell, s = t - e * P.n_shell;
    const int l = P.shell_l[s], ao0 = P.shell_ao0[s], nc = (l + 1) * (l + 2) / 2;
    if (e >= ne) {
      for (int c = 0; c < 5; c++)
        for (int q = 0; q < nc; q++) {
          Xh[(c * kECm + e) * K + ao0 + q] = 0.0f;
          Xl[(c * kECm + e) * K + ao0 + q] = 0.0f;
        }
      continue;
    }
    ao_shell_values_df(P, s, rdf[e], [&](int c, int q, df32 d) {
      Xh[(c * kECm + e) * K + ao0 + q] = d.hi;
      Xl[(c * kECm + e) * K + ao0 + q] = d.lo;
    });
  }
  __syncthreads();
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    float s[5 * kECm], c[5 * kECm];
#pragma unroll
    for (int q = 0; q < 5 * kECm; q++) s[q] = c[q] = 0.0f;
    for (int mu = 0; mu < K; mu++) {
      const float bh = __ldg(P.B_hi + (size_t)mu * M + m);
      const float bl = __ldg(P.B_lo + (size_t)mu * M + m);
#pragma unroll
      for (int q = 0; q < 5 * kECm; q++) {
        const float a = Xh[q * K + mu], al = Xl[q * K + mu];
        const float p = __fmul_rn(a, bh);
        const float pe = __fmaf_rn(a, bh, -p);
        const float cross = __fmaf_rn(a, bl, __fmul_rn(al, bh));
        float t, e;
        two_sum(s[q], p, t, e);
        s[q] = t;
        c[q] = __fadd_rn(c[q], __fadd_rn(e, __fadd_rn(pe, cross)));
      }
    }
#pragma unroll
    for (int cc = 0; cc < 5; cc++)
#pragma unroll
      for (int e = 0; e < kECm; e++)
        if (e < ne) {
          float hi, lo;
          two_sum(s[cc * kECm + e], c[cc * kECm + e], hi, lo);
          phi[((w * 5 + cc) * N + e_begin + e) * M + m] = make_float2(hi, lo);
        }
  }
}

// Orbitals on the tensor cores with exact digit products (an Ozaki-type
// scheme). grid (n_walk, ceil(n_elec / kECm)), block 128 (4 warps).
// The AO values X (double-float, as in k_mo_mixed) of each row r (quantity,
// electron) are written as 2^e_r * sum_i d_i 2^(-8 i), i = 1..7, with integer
// digits |d_1| <= 256, |d_i| <= 128 (exact in BF16); the MO coefficients of
// each column m likewise with 2^f_m (precomputed on the host, B_dig). A digit
// product is an integer, and for one K chunk of 112 the sum of |products| over
// the pairs (i, j) of one order t = i + j <= 8 (at most 7 pairs) is at most
// 2*112*256*128 + 5*112*128*128 < 2^24, so every partial sum of the BF16 MMA
// with FP32 accumulation is an exact integer. The groups t = 2..8 are scaled by
// 2^(-8 t) and summed in double-float. The representation error, 2^-57 of the
// row and column maxima per element, and the dropped orders t >= 9 stay below
// the error of the double-float path.
constexpr int kDig = 7;   // digits per operand
constexpr int kKc = 112;  // K chunk whose group sums are exact (7 MMA k-steps)

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_pair(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// BF16 bits of an integer |d| <= 256 (exact: its FP32 form has no bits below the top 8)
__device__ __forceinline__ uint16_t bf16_int(float d) { return (uint16_t)(__float_as_uint(d) >> 16); }

template <int kECm>
__global__ void __launch_bounds__(128) k_mo_tc(DevProblem P, float2* __restrict__ phi, const double* __restrict__ R) {
  constexpr int kRows = 5 * kECm, kMt = (kRows + 15) / 16, kRowsP = kMt * 16;
  extern __shared__ float smf[];
  __shared__ df32 rdf[kECm][3];
  __shared__ int er[kRowsP];
  const int K = P.n_ao, M = P.n_mo, N = P.n_elec, Kp = P.tc_kp, Mp = P.tc_mp, Sx = P.tc_sx;
  const int64_t w = blockIdx.x;
  const int e_begin = blockIdx.y * kECm;
  const int ne = min(kECm, N - e_begin);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* Xh = smf;  // [(c * kECm + e) * K + mu]
  float* Xl = smf + kRows * K;
  uint16_t* Xd = reinterpret_cast<uint16_t*>(Xl + kRows * K);  // [kDig][kRowsP][Sx] BF16 digits
  if (threadIdx.x < 3 * ne) {
    const int e = threadIdx.x / 3, d = threadIdx.x - 3 * e;
    rdf[e][d] = df_from_double(R[(w * N + e_begin + e) * 3 + d]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kECm * P.n_shell; t += blockDim.x) {
    const int e = t / P.n_shell, s = t - e * P.n_shell;
    const int l = P.shell_l[s], ao0 = P.shell_ao0[s], nc = (l + 1) * (l + 2) / 2;
    if (e >= ne) {
      for (int c = 0; c < 5; c++)
        for (int q = 0; q < nc; q++) {
          Xh[(c * kECm + e) * K + ao0 + q] = 0.0f;
          Xl[(c * kECm + e) * K + ao0 + q] = 0.0f;
        }
      continue;
    }
    ao_shell_values_df(P, s, rdf[e], [&](int c, int q, df32 d) {
      Xh[(c * kECm + e) * K + ao0 + q] = d.hi;
      Xl[(c * kECm + e) * K + ao0 + q] = d.lo;
    });
  }
  __syncthreads();
  // row exponents: |x| < 2^e_r for every entry of the row
  for (int r = warp; r < kRowsP; r += 4) {
    float mx = 0.0f;
    if (r < kRows)
      for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(Xh[r * K + k]));
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) er[r] = mx > 0.0f ? ilogbf(mx) + 1 : 0;
  }
  __syncthreads();
  // digits of (xh + xl) 2^-e_r: d = rint(256 v), v <- 256 v - d (exact), renormalised with TwoSum
  for (int t = threadIdx.x; t < kRowsP * Kp; t += blockDim.x) {
    const int r = t / Kp, k = t - r * Kp;
    float vh = 0.0f, vl = 0.0f;
    if (r < kRows && k < K) {
      vh = ldexpf(Xh[r * K + k], -er[r]);
      vl = ldexpf(Xl[r * K + k], -er[r]);
    }
#pragma unroll
    for (int i = 0; i < kDig; i++) {
      vh *= 256.0f;
      vl *= 256.0f;
      const float d = rintf(vh);
      float sh, sl;
      two_sum(vh - d, vl, sh, sl);
      vh = sh;
      vl = sl;
      Xd[((size_t)i * kRowsP + r) * Sx + k] = bf16_int(d);
    }
  }
  __syncthreads();
  const int g = lane >> 2, c4 = lane & 3;
  const int n_nt = Mp / 8;
  // each warp takes n-tiles warp, warp + 4, warp + 8, ... two at a time (an A fragment feeds two MMAs);
  // the B fragments of all k-steps of a digit pair are loaded before its MMAs
  for (int base = warp; base < n_nt; base += 8) {
    const int nt[2] = {base, base + 4};
    const bool two = nt[1] < n_nt;
    df32 acc[2][kMt][4];
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
      for (int mt = 0; mt < kMt; mt++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[u][mt][q] = df32(0.0f, 0.0f);
    for (int k0 = 0; k0 < Kp; k0 += kKc) {
      const int n_ks = min(kKc, Kp - k0) / 16;
      for (int ts = 2; ts <= kDig + 1; ts++) {
        float cs[2][kMt][4];
#pragma unroll
        for (int u = 0; u < 2; u++)
#pragma unroll
          for (int mt = 0; mt < kMt; mt++)
#pragma unroll
            for (int q = 0; q < 4; q++) cs[u][mt][q] = 0.0f;
        for (int i = max(1, ts - kDig); i <= min(kDig, ts - 1); i++) {
          uint32_t bf[2][kKc / 16][2];
#pragma unroll
          for (int u = 0; u < 2; u++) {
            const uint16_t* Bj = P.B_dig + ((size_t)(ts - i - 1) * Mp + nt[two ? u : 0] * 8 + g) * Kp + k0 + 2 * c4;
#pragma unroll
            for (int ks = 0; ks < kKc / 16; ks++)
              if (ks < n_ks) {
                bf[u][ks][0] = __ldg(reinterpret_cast<const unsigned int*>(Bj + ks * 16));
                bf[u][ks][1] = __ldg(reinterpret_cast<const unsigned int*>(Bj + ks * 16 + 8));
              }
          }
          const uint16_t* Ai = Xd + ((size_t)(i - 1) * kRowsP + g) * Sx + k0 + 2 * c4;
#pragma unroll
          for (int ks = 0; ks < kKc / 16; ks++)
            if (ks < n_ks) {
#pragma unroll
              for (int mt = 0; mt < kMt; mt++) {
                const uint16_t* a0 = Ai + (size_t)mt * 16 * Sx + ks * 16;
                const uint32_t a[4] = {ld_pair(a0), ld_pair(a0 + 8 * Sx), ld_pair(a0 + 8), ld_pair(a0 + 8 * Sx + 8)};
                mma_bf16_16816(cs[0][mt], a, bf[0][ks]);
                mma_bf16_16816(cs[1][mt], a, bf[1][ks]);
              }
            }
        }
        // the exact group sums of order ts, weighted 2^(-8 ts)
#pragma unroll
        for (int u = 0; u < 2; u++)
#pragma unroll
          for (int mt = 0; mt < kMt; mt++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[u][mt][q] = acc[u][mt][q] + df32(ldexpf(cs[u][mt][q], -8 * ts), 0.0f);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
      if (u == 1 && !two) break;
#pragma unroll
      for (int mt = 0; mt < kMt; mt++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int row = mt * 16 + g + (q >= 2 ? 8 : 0), col = nt[u] * 8 + 2 * c4 + (q & 1);
          if (row >= kRows || col >= M) continue;
          const int cc = row / kECm, e = row - cc * kECm;
          if (e >= ne) continue;
          const int E = er[row] + P.B_exp[col];
          phi[((w * 5 + cc) * N + e_begin + e) * M + col] = make_float2(ldexpf(acc[u][mt][q].hi, E), ldexpf(acc[u][mt][q].lo, E));
        }
    }
  }
}

// Ratios r_I = eps_I det M_I in double-float from the table pairs. Same launch
// shape as the FP64 ratio kernel: lanes are walkers, each warp 8 determinants.
__global__ void __launch_bounds__(128) k_ratio_df(DevProblem P, DevScratch S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.y * 32 + lane;
  const int nu_det = P.n_det_sp[0], ntot = nu_det + P.n_det_sp[1];
  const int M = P.n_mo;
  const int64_t wp = S.wp;
  for (int q = 0; q < 8; q++) {
    const int t = blockIdx.x * 32 + warp * 8 + q;
    if (t >= ntot) return;
    const int sp = t < nu_det ? 0 : 1;
    const Exc e = P.exc[sp][sp ? t - nu_det : t];
    const float2* T = S.Tdf + (size_t)(sp ? P.n_up * M : 0) * wp;
    df32 m[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const float2 v = (a < e.k && b < e.k) ? T[((size_t)e.h[a] * M + e.p[b]) * wp + w] : make_float2(0.f, 0.f);
        m[a][b] = df32(v.x, v.y);
      }
    const df32 d0 = small_det_dot(e.k, m);
    const df32 dd = e.eps < 0 ? df32(-d0.hi, -d0.lo) : d0;  // the sign on the FP32 words
    S.r[(size_t)t * wp + w] = df_to_double_int(dd);  // the FP64 ratio for the contraction, off the FP64 pipe
    if (S.rdf) S.rdf[(size_t)t * wp + w] = make_float2(dd.hi, dd.lo);
    if (P.split[t]) S.vu[w * ntot + t] = 0.0;  // the contraction adds the pieces of a cut segment
  }
}

// Self-check of the double-float building blocks against FP64 on the device:
// y_df[i] = double-float exp(x_i), y_ref[i] = CUDA's FP64 exp(x_i) (x_i <= 0),
// and prod_df[i] = double-float product x_i * x_{i+1} for comparison with FP64.
__global__ void k_selftest_df(int64_t n, const double* __restrict__ x, double* __restrict__ y_df,
                              double* __restrict__ y_ref, double* __restrict__ prod_df) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const df32 a = df_from_double(x[i]);
  y_df[i] = df_to_double(df_exp_nonpos(a));
  y_ref[i] = exp(x[i]);
  const df32 b = df_from_double(x[(i + 1) % n]);
  prod_df[i] = df_to_double(a * b + a);
}

// The Coulomb sums' reciprocal square root against CUDA's FP64 1 / sqrt on the device:
// y_nr[i] = coulomb_inv_r(x_i), y_ref[i] = 1.0 / sqrt(x_i).
__global__ void k_selftest_inv_r(int64_t n, const double* __restrict__ x, double* __restrict__ y_nr,
                                 double* __restrict__ y_ref) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y_nr[i] = coulomb_inv_r(x[i]);
  y_ref[i] = 1.0 / sqrt(x[i]);
}

}  // namespace

template <int EC>
static cudaError_t launch_mo_mixed_ec(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                                     cudaStream_t st) {
  const size_t smem = sizeof(float) * 2 * 5 * EC * P.n_ao;
  static SmemOptIn opt;  // dynamic shared memory (static arrays come on top)
  cudaError_t e = opt.ensure(k_mo_mixed<EC>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)n_walk, (P.n_elec + EC - 1) / EC);
  k_mo_mixed<EC><<<grid, 128, smem, st>>>(P, reinterpret_cast<float2*>(S.phi), R);
  return cudaGetLastError();
}

size_t mo_tc_smem_bytes(const DevProblem& P, int ec) {
  const int rows = 5 * ec, rows_p = (rows + 15) / 16 * 16;
  return sizeof(float) * 2 * rows * P.n_ao + sizeof(uint16_t) * (size_t)kDig * rows_p * P.tc_sx;
}

template <int EC>
static cudaError_t launch_mo_tc_ec(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                                   cudaStream_t st) {
  const size_t smem = mo_tc_smem_bytes(P, EC);
  static SmemOptIn opt;
  cudaError_t e = opt.ensure(k_mo_tc<EC>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)n_walk, (P.n_elec + EC - 1) / EC);
  k_mo_tc<EC><<<grid, 128, smem, st>>>(P, reinterpret_cast<float2*>(S.phi), R);
  return cudaGetLastError();
}

cudaError_t launch_mo_mixed(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                            cudaStream_t st) {
  // tcgen05 digit products by default; warp-level MMA digits (mo_impl 0) or the compensated
  // CUDA-core product when asked for, or when the problem exceeds what the tcgen05 kernel holds
  if (P.mo_impl == 2 && mo_umma_supported(P)) return launch_mo_umma(P, S, n_walk, R, P.n_sm, st);
  const size_t kSmemMax = 200 * 1024;
  if (P.mo_impl == 0 && P.B_dig && mo_tc_smem_bytes(P, P.mo_ec) <= kSmemMax) {
    switch (P.mo_ec) {
      case 4: return launch_mo_tc_ec<4>(P, S, n_walk, R, st);
      case 8: return launch_mo_tc_ec<8>(P, S, n_walk, R, st);
      default: return launch_mo_tc_ec<6>(P, S, n_walk, R, st);
    }
  }
  switch (P.mo_ec) {
    case 4: return launch_mo_mixed_ec<4>(P, S, n_walk, R, st);
    case 8: return launch_mo_mixed_ec<8>(P, S, n_walk, R, st);
    default: return launch_mo_mixed_ec<6>(P, S, n_walk, R, st);
  }
}

cudaError_t launch_selftest_df(int64_t n, const double* x, double* y_df, double* y_ref, double* prod_df,
                               cudaStream_t st) {
  k_selftest_df<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y_df, y_ref, prod_df);
  return cudaGetLastError();
}

cudaError_t launch_selftest_inv_r(int64_t n, const double* x, double* y_nr, double* y_ref, cudaStream_t st) {
  k_selftest_inv_r<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y_nr, y_ref);
  return cudaGetLastError();
}

cudaError_t launch_ratios_mixed(const DevProblem& P, const DevScratch& S, int64_t n_walk, cudaStream_t st) {
  const int ntot = P.n_det_sp[0] + P.n_det_sp[1];
  const int64_t wpad = (n_walk + 31) / 32 * 32;
  dim3 grid((ntot + 31) / 32, (unsigned)(wpad / 32));
  k_ratio_df<<<grid, 128, 0, st>>>(P, S);
  return cudaGetLastError();
}

}  // namespace mdet

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
// inputs). Phi = s + c is stored in FP64.
template <int kECm>
__global__ void __launch_bounds__(128) k_mo_mixed(DevProblem P, double* __restrict__ phi,
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
        if (e < ne) phi[((w * 5 + cc) * N + e_begin + e) * M + m] = (double)s[cc * kECm + e] + (double)c[cc * kECm + e];
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
    const double d = df_to_double(small_det(e.k, m));
    S.r[(size_t)t * wp + w] = e.eps < 0 ? -d : d;
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

}  // namespace

template <int EC>
static cudaError_t launch_mo_mixed_ec(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                                     cudaStream_t st) {
  const size_t smem = sizeof(float) * 2 * 5 * EC * P.n_ao;
  static size_t attr_bytes = 0;  // dynamic shared memory opted in so far (static arrays come on top)
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_mo_mixed<EC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  dim3 grid((unsigned)n_walk, (P.n_elec + EC - 1) / EC);
  k_mo_mixed<EC><<<grid, 128, smem, st>>>(P, S.phi, R);
  return cudaGetLastError();
}

cudaError_t launch_mo_mixed(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                            cudaStream_t st) {
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

cudaError_t launch_ratios_mixed(const DevProblem& P, const DevScratch& S, int64_t n_walk, cudaStream_t st) {
  const int ntot = P.n_det_sp[0] + P.n_det_sp[1];
  const int64_t wpad = (n_walk + 31) / 32 * 32;
  dim3 grid((ntot + 31) / 32, (unsigned)(wpad / 32));
  k_ratio_df<<<grid, 128, 0, st>>>(P, S);
  return cudaGetLastError();
}

}  // namespace mdet

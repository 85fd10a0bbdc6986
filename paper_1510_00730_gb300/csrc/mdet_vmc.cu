// Variational Monte Carlo moves and the learned proposal (include/mdet_vmc.h).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit
// multiplications by 0xD2511F53 and 0xCD9E8D57, with the key bumped by the
// Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds. Counter layout:
// (group of 4 coordinates, walker, step low, step high / purpose), key = seed.
// Normal variates by the Box-Muller transform of two uniforms in (0, 1).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mdet_vmc.h"
#include "mdet_internal.h"

using mdet::GemmEpilogue;
using mdet::GemmOperand;
using mdet::kEpiAtomic;
using mdet::kEpiBias;
using mdet::kEpiDtanh;
using mdet::kEpiTanhBias;
using mdet::launch_gemm_bf16;

namespace {

__host__ __device__ inline void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       uint32_t out[4]) {
  for (int r = 0; r < 10; r++) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

constexpr uint32_t kPurposeNoise = 0u, kPurposeAccept = 1u << 31;

// Four standard normal variates for (walker, group of 4 coordinates).
__device__ inline void normal4(uint64_t seed, uint64_t step, int64_t w, int grp, float z[4]) {
  uint32_t x[4];
  philox((uint32_t)grp, (uint32_t)w, (uint32_t)step, (uint32_t)(step >> 32) ^ kPurposeNoise, (uint32_t)seed,
         (uint32_t)(seed >> 32), x);
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const float u1 = ((float)x[2 * q] + 0.5f) * 0x1p-32f;
    const float u2 = ((float)x[2 * q + 1] + 0.5f) * 0x1p-32f;
    const float rr = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    z[2 * q] = rr * cs;
    z[2 * q + 1] = rr * sn;
  }
}

__device__ inline double uniform_accept(uint64_t seed, uint64_t step, int64_t w) {
  uint32_t x[4];
  philox(0u, (uint32_t)w, (uint32_t)step, (uint32_t)(step >> 32) ^ kPurposeAccept, (uint32_t)seed,
         (uint32_t)(seed >> 32), x);
  return ((double)x[0] + 0.5) * 0x1p-32;  // in (0, 1)
}

__global__ void k_propose_drift(int64_t n_walk, int n3, const double* __restrict__ R, const double* __restrict__ F,
                                double tau, uint64_t seed, uint64_t step, double* __restrict__ Rn,
                                double* __restrict__ lq) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  const double st = sqrt(tau);
  double acc = 0.0;
  for (int g = 0; g < (n3 + 3) / 4; g++) {
    float z[4];
    normal4(seed, step, w, g, z);
    for (int q = 0; q < 4 && 4 * g + q < n3; q++) {
      const int64_t i = w * n3 + 4 * g + q;
      const double mean = R[i] + tau * F[i];
      const double rn = mean + st * (double)z[q];
      Rn[i] = rn;
      const double d = rn - mean;
      acc += d * d;
    }
  }
  lq[w] = -acc / (2.0 * tau);
}

__global__ void k_reverse_drift(int64_t n_walk, int n3, const double* __restrict__ R, const double* __restrict__ Rn,
                                const double* __restrict__ Fn, double tau, double* __restrict__ lq) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  double acc = 0.0;
  for (int c = 0; c < n3; c++) {
    const int64_t i = w * n3 + c;
    const double d = R[i] - (Rn[i] + tau * Fn[i]);
    acc += d * d;
  }
  lq[w] = -acc / (2.0 * tau);
}

__global__ void k_accept(int64_t n_walk, int N, uint64_t seed, uint64_t step, const double* __restrict__ lqf,
                         const double* __restrict__ lqr, double* R, double* lp, int8_t* sg, double* grad, double* lap,
                         double* el, const double* __restrict__ Rn, const double* __restrict__ lpn,
                         const int8_t* __restrict__ sgn, const double* __restrict__ gradn,
                         const double* __restrict__ lapn, const double* __restrict__ eln, int32_t* acc_out,
                         uint32_t* n_acc) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  const double la = 2.0 * (lpn[w] - lp[w]) + lqr[w] - lqf[w];
  const double u = uniform_accept(seed, step, w);
  // la = +inf (the current state has |Psi| = 0 or underflowed) accepts any
  // finite proposal; a proposal with a non-finite state is never taken.
  bool ok = sgn[w] != 0 && isfinite(lpn[w]) && !isnan(la) && log(u) < la;
  for (int c = 0; c < 3 * N && ok; c++) ok = isfinite(gradn[w * 3 * N + c]);
  if (acc_out) acc_out[w] = ok ? 1 : 0;
  if (!ok) return;
  for (int c = 0; c < 3 * N; c++) {
    R[w * 3 * N + c] = Rn[w * 3 * N + c];
    grad[w * 3 * N + c] = gradn[w * 3 * N + c];
  }
  for (int i = 0; i < N; i++) lap[w * N + i] = lapn[w * N + i];
  lp[w] = lpn[w];
  sg[w] = sgn[w];
  if (el) el[w] = eln[w];
  if (n_acc) atomicAdd(n_acc, 1u);
}

// Drift limiting of Umrigar, Nightingale and Runge (J. Chem. Phys. 99, 2865
// (1993)) per electron: Fbar_i = F_i (-1 + sqrt(1 + 2 a tau |F_i|^2)) / (a tau |F_i|^2),
// written as F_i * 2 / (1 + sqrt(1 + 2 a tau |F_i|^2)) (no cancellation at small |F_i|).
__global__ void k_limit_drift(int64_t n_walk, int N, const double* __restrict__ F, double tau, double a,
                              double* __restrict__ Fb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_walk * N) return;
  const double fx = F[3 * i], fy = F[3 * i + 1], fz = F[3 * i + 2];
  const double f2 = fx * fx + fy * fy + fz * fz;
  const double k = a > 0.0 ? 2.0 / (1.0 + sqrt(1.0 + 2.0 * a * tau * f2)) : 1.0;
  Fb[3 * i] = k * fx;
  Fb[3 * i + 1] = k * fy;
  Fb[3 * i + 2] = k * fz;
}

__global__ void k_select_rows(int64_t n_walk, int width, const int32_t* __restrict__ take,
                              const float* __restrict__ src, float* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_walk * width) return;
  if (take[i / width]) dst[i] = src[i];
}

__global__ void k_r2(int64_t n_walk, int N, const double* __restrict__ R, double* __restrict__ r2) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  double s = 0.0;
  for (int c = 0; c < 3 * N; c++) s += R[w * 3 * N + c] * R[w * 3 * N + c];
  r2[w] = s;
}

}  // namespace

// ---------------------------------------------------------------------------
// The perceptron
struct mdet_mlp {
  int device = 0;
  int n_elec = 0, n_in = 0, H = 0, n_out = 0;
  double mu_max = 1.0, s0 = -1.0, s_span = 2.0, coord_scale = 2.0;
  int64_t n_params = 0;
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16* pb = nullptr;
  int64_t cap = 0;
  // per walker: input, hidden activations (FP32, kept for the backward pass) and the
  // back-propagated deltas of the two hidden layers
  float *x = nullptr, *h1 = nullptr, *h2 = nullptr, *d1 = nullptr, *d2 = nullptr;
};

namespace {

constexpr int kCapRound = 128;  // scratch rows are allocated in multiples of one GEMM tile

// x = R / coord_scale in FP32, the network's input, kept for the backward pass.
__global__ void k_mlp_input(int64_t n, const double* __restrict__ R, float inv_scale, float* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (float)R[i] * inv_scale;
}

// Bias gradients: gb[n] += sum over walkers of d[w][n] for up to three (d, width, gb) jobs
// (blockIdx.z); each thread sums one column over a slice of the walkers.
struct ColSumJob {
  const float* d;
  int width;
  float* gb;
};
struct ColSumJobs {
  ColSumJob j[3];
};
__global__ void k_bias_grad(ColSumJobs jobs, int64_t n_walk, int64_t per) {
  const ColSumJob J = jobs.j[blockIdx.z];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= J.width) return;
  const int64_t w0 = (int64_t)blockIdx.y * per, w1 = min(n_walk, w0 + per);
  float s = 0.0f;
  for (int64_t w = w0; w < w1; w++) s += J.d[w * J.width + n];
  if (s != 0.0f) atomicAdd(J.gb + n, s);
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, __nv_bfloat16* __restrict__ pb, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  const float v = p[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
  p[i] = v;
  pb[i] = __float2bfloat16_rn(v);
}

struct Head {
  int N;
  double mu_max, s0, s_span;
};

// Head of the network for electron e, coordinate c: log-scale
// s_e = s0 + s_span tanh(out[3N + e]), sigma_e = exp(s_e), and mean offset
// mu_c = sigma_e mu_max tanh(out[c]) (in units of the electron's own step).

// Gaussian negative log-likelihood of R0 -> R1 per walker and its gradient
// with respect to the raw outputs (mean over walkers):
//   NLL = sum_c d_c^2 / (2 sigma_e^2) + 3 sum_e s_e,  d_c = R1_c - R0_c - mu_c,
//   dNLL/dmu_c = -d_c / sigma_e^2,  dNLL/ds_e = 3 - sum_c (d_c^2 + d_c mu_c) / sigma_e^2.
__global__ void k_nll(Head hd, int64_t n_walk, const double* __restrict__ R0, const double* __restrict__ R1,
                      const float* __restrict__ out, float* __restrict__ dout, double* __restrict__ loss) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (w < n_walk) {
    const int N = hd.N, no = 4 * N;
    const float invB = 1.0f / (float)n_walk;
    for (int e = 0; e < N; e++) {
      const float ts = tanhf(out[w * no + 3 * N + e]);
      const float s = (float)hd.s0 + (float)hd.s_span * ts;
      const float sig = expf(s), iv = expf(-2.0f * s);
      float d2 = 0.0f, dmu = 0.0f;
      for (int c = 0; c < 3; c++) {
        const float tm = tanhf(out[w * no + 3 * e + c]);
        const float mu = sig * (float)hd.mu_max * tm;
        const float d = (float)(R1[w * 3 * N + 3 * e + c] - R0[w * 3 * N + 3 * e + c]) - mu;
        d2 += d * d;
        dmu += d * mu;
        dout[w * no + 3 * e + c] = invB * (-d * iv) * sig * (float)hd.mu_max * (1.0f - tm * tm);
      }
      l += 0.5 * d2 * iv + 3.0 * s;
      dout[w * no + 3 * N + e] = invB * (3.0f - (d2 + dmu) * iv) * (float)hd.s_span * (1.0f - ts * ts);
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l / (double)n_walk);
}

// The learned move of electron e, coordinate c: mean R_c + mu_c + sigma_e^2 F_c
// (F = grad Psi / Psi at R, or 0 without the Langevin term), scale sigma_e.
__global__ void k_propose_mlp(Head hd, int64_t n_walk, const double* __restrict__ R, const float* __restrict__ out,
                              const double* __restrict__ F, uint64_t seed, uint64_t step, double* __restrict__ Rn,
                              double* __restrict__ lq) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  const int N = hd.N, n3 = 3 * N, no = 4 * N;
  double acc = 0.0;
  for (int g = 0; g < (n3 + 3) / 4; g++) {
    float z[4];
    normal4(seed, step, w, g, z);
    for (int q = 0; q < 4 && 4 * g + q < n3; q++) {
      const int c = 4 * g + q, e = c / 3;
      const double s = hd.s0 + hd.s_span * tanh((double)out[w * no + n3 + e]);
      const double sig = exp(s);
      const double mu = sig * hd.mu_max * tanh((double)out[w * no + c]);
      const double mean = R[w * n3 + c] + mu + (F ? sig * sig * F[w * n3 + c] : 0.0);
      const double rn = mean + sig * (double)z[q];
      Rn[w * n3 + c] = rn;
      const double d = (rn - mean) / sig;
      acc += -0.5 * d * d - s;
    }
  }
  lq[w] = acc;
}

__global__ void k_reverse_mlp(Head hd, int64_t n_walk, const double* __restrict__ R, const double* __restrict__ Rn,
                              const float* __restrict__ out_n, const double* __restrict__ Fn,
                              double* __restrict__ lq) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  const int N = hd.N, n3 = 3 * N, no = 4 * N;
  double acc = 0.0;
  for (int c = 0; c < n3; c++) {
    const int e = c / 3;
    const double s = hd.s0 + hd.s_span * tanh((double)out_n[w * no + n3 + e]);
    const double sig = exp(s);
    const double mu = sig * hd.mu_max * tanh((double)out_n[w * no + c]);
    const double d = (R[w * n3 + c] - (Rn[w * n3 + c] + mu + (Fn ? sig * sig * Fn[w * n3 + c] : 0.0))) / sig;
    acc += -0.5 * d * d - s;
  }
  lq[w] = acc;
}

// Training objectives of the learned move (see mdet_vmc.h), per walker:
//   ESJD  J = A D2,  A = min(1, alpha), D2 = sum_e w_e |R'_e - R_e|^2;
//   speed J = min(0, log alpha) + beta * 3 sum_e s_e  (beta > 0).
// With the noise chi held fixed, R'_c = R_c + mu_c + sigma_e^2 F_c + sigma_e chi_c, so
//   dR'_c/dmu_c = 1,  dR'_c/ds_e = 2 sigma_e^2 F_c + sigma_e chi_c + mu_c  (mu_c scales with sigma_e),
// log q(R'|R) = -|chi|^2/2 - 3 sum_e s_e depends on the parameters through s only,
// and with a_c = R_c - R'_c - mu'_c - sigma'^2_e F'_c (F' held fixed)
//   log q(R|R') = -sum_c a_c^2 / (2 sigma'^2_e) - 3 sum_e s'_e,
//   d log alpha / dR'_c = 2 G'_c + a_c / sigma'^2_e  (G' = grad log|Psi| at R'; F' = G' unless limited),
//   d log alpha / dmu'_c = a_c / sigma'^2_e,
//   d log alpha / ds'_e = sum_c (a_c^2 + a_c (mu'_c + 2 sigma'^2_e F'_c)) / sigma'^2_e - 3.
// The jump of electron e is weighted by w_e = 1 / (|R_e|^2 + len2) (len2 > 0) or 1.
// obj[0] += mean J, obj[1] += mean A.
__global__ void k_esjd(Head hd, int64_t n_walk, const double* __restrict__ R, const double* __restrict__ Rn,
                       const float* __restrict__ out, const float* __restrict__ outn, const double* __restrict__ lp,
                       const double* __restrict__ lpn, const int8_t* __restrict__ sgn, const double* __restrict__ F,
                       const double* __restrict__ Fn, const double* __restrict__ Gn, bool langevin, double len2,
                       double beta, float* __restrict__ dout, float* __restrict__ doutn, double* __restrict__ obj) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double J = 0.0, Aw = 0.0;
  if (w < n_walk) {
    const int N = hd.N, n3 = 3 * N, no = 4 * N;
    const double invB = 1.0 / (double)n_walk;
    const double kl = langevin ? 1.0 : 0.0, mm = hd.mu_max;
    const bool speed = beta > 0.0;
    // log alpha, the weighted |dR|^2 and the sum of log-scales
    double lqf = 0.0, lqr = 0.0, D2 = 0.0, S = 0.0;
    for (int e = 0; e < N; e++) {
      const double s = hd.s0 + hd.s_span * tanh((double)out[w * no + n3 + e]);
      const double sn = hd.s0 + hd.s_span * tanh((double)outn[w * no + n3 + e]);
      const double sig = exp(s), sign = exp(sn);
      double r2 = 0.0, j2 = 0.0;
      for (int d = 0; d < 3; d++) {
        const int c = 3 * e + d;
        const double mu = sig * mm * tanh((double)out[w * no + c]);
        const double mun = sign * mm * tanh((double)outn[w * no + c]);
        const double dR = Rn[w * n3 + c] - R[w * n3 + c];
        const double chi = (dR - mu - kl * sig * sig * F[w * n3 + c]) / sig;
        const double a = -dR - mun - kl * sign * sign * Fn[w * n3 + c];
        lqf += -0.5 * chi * chi;
        lqr += -0.5 * a * a / (sign * sign);
        j2 += dR * dR;
        r2 += R[w * n3 + c] * R[w * n3 + c];
      }
      lqf -= 3.0 * s;
      lqr -= 3.0 * sn;
      S += s;
      D2 += (len2 > 0.0 ? 1.0 / (r2 + len2) : 1.0) * j2;
    }
    const double la = 2.0 * (lpn[w] - lp[w]) + lqr - lqf;
    bool valid = sgn[w] != 0 && isfinite(la) && isfinite(D2);
    for (int c = 0; c < n3 && valid; c++)
      valid = isfinite(Fn[w * n3 + c]) && isfinite(F[w * n3 + c]) && isfinite(Gn[w * n3 + c]);
    const double A = valid ? (la < 0.0 ? exp(la) : 1.0) : 0.0;
    const bool act = valid && la < 0.0;  // acceptance below 1 depends on the parameters
    // dJ = cA d(log alpha) + cD d(D2) + cH d(sum_e s_e)
    const double cA = act ? (speed ? 1.0 : A * D2) : 0.0;
    const double cD = speed ? 0.0 : A;
    const double cH = speed ? 3.0 * beta : 0.0;
    Aw = A;
    J = valid ? (speed ? fmin(la, 0.0) + beta * 3.0 * S : A * D2) : 0.0;
    if (!valid) {  // a rejected move (node, non-finite state): no contribution to J or its gradient
      for (int c = 0; c < no; c++) dout[w * no + c] = doutn[w * no + c] = 0.0f;
    }
    for (int e = 0; e < N && valid; e++) {
      const double ts = tanh((double)out[w * no + n3 + e]);
      const double sig = exp(hd.s0 + hd.s_span * ts);
      const double tsn = tanh((double)outn[w * no + n3 + e]);
      const double sign = exp(hd.s0 + hd.s_span * tsn), ivn = 1.0 / (sign * sign);
      double r2 = 0.0;
      for (int d = 0; d < 3; d++) r2 += R[w * n3 + 3 * e + d] * R[w * n3 + 3 * e + d];
      const double we = len2 > 0.0 ? 1.0 / (r2 + len2) : 1.0;
      double dJ_ds = cH, dla_dsn = -3.0;
      for (int d = 0; d < 3; d++) {
        const int c = 3 * e + d;
        const double tm = tanh((double)out[w * no + c]), mu = sig * mm * tm;
        const double tmn = tanh((double)outn[w * no + c]), mun = sign * mm * tmn;
        const double f = kl * F[w * n3 + c], fn = kl * Fn[w * n3 + c];
        const double dR = Rn[w * n3 + c] - R[w * n3 + c];
        const double chi = (dR - mu - sig * sig * f) / sig;
        const double a = -dR - mun - sign * sign * fn;
        const double gR = 2.0 * Gn[w * n3 + c] + a * ivn;  // d log alpha / dR'
        const double gJ = cA * gR + cD * 2.0 * we * dR;    // dJ / dR'
        const double dRds = 2.0 * sig * sig * f + sig * chi + mu;
        dJ_ds += gJ * dRds;
        dla_dsn += (a * a + a * (mun + 2.0 * sign * sign * fn)) * ivn;
        dout[w * no + c] = (float)(-invB * gJ * sig * mm * (1.0 - tm * tm));
        doutn[w * no + c] = (float)(-invB * cA * a * ivn * sign * mm * (1.0 - tmn * tmn));
      }
      dJ_ds += cA * 3.0;  // -log q(R'|R) contributes +3 per electron to d log alpha / d s
      dout[w * no + n3 + e] = (float)(-invB * dJ_ds * hd.s_span * (1.0 - ts * ts));
      doutn[w * no + n3 + e] = (float)(-invB * cA * dla_dsn * hd.s_span * (1.0 - tsn * tsn));
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    J += __shfl_xor_sync(0xffffffffu, J, off);
    Aw += __shfl_xor_sync(0xffffffffu, Aw, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (J != 0.0) atomicAdd(obj, J / (double)n_walk);
    if (Aw != 0.0) atomicAdd(obj + 1, Aw / (double)n_walk);
  }
}

Head head(const mdet_mlp* m) {
  return Head{m->n_elec, m->mu_max, m->s0, m->s_span};
}

mdet_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MDET_OK : MDET_E_CUDA; }

unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

mdet_status ensure_mlp_scratch(mdet_mlp* m, int64_t n_walk) {
  if (n_walk <= m->cap) return MDET_OK;
  cudaFree(m->x);
  cudaFree(m->h1);
  cudaFree(m->h2);
  cudaFree(m->d1);
  cudaFree(m->d2);
  m->x = m->h1 = m->h2 = m->d1 = m->d2 = nullptr;
  m->cap = 0;
  const int64_t cap = (n_walk + kCapRound - 1) / kCapRound * kCapRound;
  if (cudaMalloc((void**)&m->x, sizeof(float) * cap * m->n_in) != cudaSuccess ||
      cudaMalloc((void**)&m->h1, sizeof(float) * cap * m->H) != cudaSuccess ||
      cudaMalloc((void**)&m->h2, sizeof(float) * cap * m->H) != cudaSuccess ||
      cudaMalloc((void**)&m->d1, sizeof(float) * cap * m->H) != cudaSuccess ||
      cudaMalloc((void**)&m->d2, sizeof(float) * cap * m->H) != cudaSuccess)
    return MDET_E_OOM;
  m->cap = cap;
  return MDET_OK;
}

}  // namespace

extern "C" {

void mdet_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1], out);
}

mdet_status mdet_vmc_propose_drift(int64_t n_walk, int n_elec, const double* R, const double* grad, double tau,
                                   uint64_t seed, uint64_t step, double* R_new, double* log_q_fwd, void* stream) {
  if (n_walk < 0 || n_elec < 1 || !(tau > 0.0)) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  k_propose_drift<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(n_walk, 3 * n_elec, R, grad, tau, seed,
                                                                          step, R_new, log_q_fwd);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_reverse_drift(int64_t n_walk, int n_elec, const double* R, const double* R_new,
                                   const double* grad_new, double tau, double* log_q_rev, void* stream) {
  if (n_walk < 0 || n_elec < 1 || !(tau > 0.0)) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  k_reverse_drift<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(n_walk, 3 * n_elec, R, R_new, grad_new,
                                                                          tau, log_q_rev);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_accept(int64_t n_walk, int n_elec, uint64_t seed, uint64_t step, const double* log_q_fwd,
                            const double* log_q_rev, double* R, double* log_abs_psi, int8_t* sign, double* grad,
                            double* lap, double* e_local, const double* R_new, const double* log_abs_psi_new,
                            const int8_t* sign_new, const double* grad_new, const double* lap_new,
                            const double* e_local_new, int32_t* accept, uint32_t* n_accept, void* stream) {
  if (n_walk < 0 || n_elec < 1) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  k_accept<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(
      n_walk, n_elec, seed, step, log_q_fwd, log_q_rev, R, log_abs_psi, sign, grad, lap, e_local, R_new,
      log_abs_psi_new, sign_new, grad_new, lap_new, e_local_new, accept, n_accept);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_limit_drift(int64_t n_walk, int n_elec, const double* F, double tau, double a, double* F_bar,
                                 void* stream) {
  if (n_walk < 0 || n_elec < 0 || !(tau > 0.0) || a < 0.0) return MDET_E_ARG;
  if (n_walk == 0 || n_elec == 0) return MDET_OK;
  if (!F || !F_bar) return MDET_E_ARG;
  k_limit_drift<<<blocks(n_walk * n_elec, 256), 256, 0, (cudaStream_t)stream>>>(n_walk, n_elec, F, tau, a, F_bar);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_select_rows(int64_t n_walk, int width, const int32_t* take, const float* src, float* dst,
                                 void* stream) {
  if (n_walk < 0 || width < 0) return MDET_E_ARG;
  if (n_walk == 0 || width == 0) return MDET_OK;
  if (!take || !src || !dst) return MDET_E_ARG;
  k_select_rows<<<blocks(n_walk * width, 256), 256, 0, (cudaStream_t)stream>>>(n_walk, width, take, src, dst);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_r2(int64_t n_walk, int n_elec, const double* R, double* r2, void* stream) {
  if (n_walk < 0 || n_elec < 1) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  k_r2<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(n_walk, n_elec, R, r2);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_mlp_create(mdet_mlp** out, int device, int n_elec, int hidden, uint64_t seed, double mu_max,
                            double s0, double s_span, double coord_scale) {
  if (!out || n_elec < 1 || hidden < 1 || hidden > 1024 || !(coord_scale > 0)) return MDET_E_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return MDET_E_CUDA;
  mdet_mlp* m = new (std::nothrow) mdet_mlp();
  if (!m) return MDET_E_OOM;
  m->device = device;
  m->n_elec = n_elec;
  m->n_in = 3 * n_elec;
  m->H = hidden;
  m->n_out = 4 * n_elec;
  m->mu_max = mu_max;
  m->s0 = s0;
  m->s_span = s_span;
  m->coord_scale = coord_scale;
  const int64_t ni = m->n_in, H = m->H, no = m->n_out;
  m->oW1 = 0;
  m->ob1 = ni * H;
  m->oW2 = m->ob1 + H;
  m->ob2 = m->oW2 + H * H;
  m->oW3 = m->ob2 + H;
  m->ob3 = m->oW3 + H * no;
  m->n_params = m->ob3 + no;
  std::vector<float> p(m->n_params, 0.0f);
  // Glorot-uniform weights from Philox (counter = parameter index, key = seed)
  auto fill = [&](int64_t off, int64_t fan_in, int64_t fan_out) {
    const double a = std::sqrt(6.0 / (double)(fan_in + fan_out));
    for (int64_t i = 0; i < fan_in * fan_out; i++) {
      uint32_t x[4];
      philox((uint32_t)i, (uint32_t)(off >> 32) ^ 0x4d4c50u, (uint32_t)off, 0u, (uint32_t)seed, (uint32_t)(seed >> 32),
             x);
      const double u = ((double)x[0] + 0.5) * 0x1p-32;
      p[off + i] = (float)(a * (2.0 * u - 1.0));
    }
  };
  fill(m->oW1, ni, H);
  fill(m->oW2, H, H);
  fill(m->oW3, H, no);
  const size_t bytes = sizeof(float) * m->n_params;
  if (cudaMalloc((void**)&m->p, bytes) != cudaSuccess || cudaMalloc((void**)&m->g, bytes) != cudaSuccess ||
      cudaMalloc((void**)&m->m1, bytes) != cudaSuccess || cudaMalloc((void**)&m->m2, bytes) != cudaSuccess ||
      cudaMalloc((void**)&m->pb, sizeof(__nv_bfloat16) * m->n_params) != cudaSuccess) {
    mdet_mlp_destroy(m);
    return MDET_E_OOM;
  }
  cudaMemset(m->g, 0, bytes);
  cudaMemset(m->m1, 0, bytes);
  cudaMemset(m->m2, 0, bytes);
  mdet_status s = mdet_mlp_set_params(m, p.data());
  if (s != MDET_OK) {
    mdet_mlp_destroy(m);
    return s;
  }
  *out = m;
  return MDET_OK;
}

void mdet_mlp_destroy(mdet_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->p);
  cudaFree(m->g);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->pb);
  cudaFree(m->x);
  cudaFree(m->h1);
  cudaFree(m->h2);
  cudaFree(m->d1);
  cudaFree(m->d2);
  delete m;
}

int64_t mdet_mlp_n_params(const mdet_mlp* m) { return m ? m->n_params : 0; }

mdet_status mdet_mlp_get_params(const mdet_mlp* m, float* host) {
  if (!m || !host) return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MDET_E_CUDA;
  return cuda_status(cudaMemcpy(host, m->p, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
}

mdet_status mdet_mlp_get_grads(const mdet_mlp* m, float* host) {
  if (!m || !host) return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MDET_E_CUDA;
  return cuda_status(cudaMemcpy(host, m->g, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
}

mdet_status mdet_mlp_set_params(mdet_mlp* m, const float* host) {
  if (!m || !host) return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MDET_E_CUDA;
  std::vector<__nv_bfloat16> b(m->n_params);
  for (int64_t i = 0; i < m->n_params; i++) b[i] = __float2bfloat16_rn(host[i]);
  if (cudaMemcpy(m->p, host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->pb, b.data(), sizeof(__nv_bfloat16) * m->n_params, cudaMemcpyHostToDevice) != cudaSuccess)
    return MDET_E_CUDA;
  return MDET_OK;
}

mdet_status mdet_mlp_forward(mdet_mlp* m, int64_t n_walk, const double* R, float* out, void* stream) {
  if (!m || n_walk < 0 || !R || !out) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  if (cudaSetDevice(m->device) != cudaSuccess) return MDET_E_CUDA;
  mdet_status s = ensure_mlp_scratch(m, n_walk);
  if (s != MDET_OK) return s;
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t ni = m->n_in, H = m->H, no = m->n_out;
  k_mlp_input<<<blocks(n_walk * ni, 256), 256, 0, st>>>(n_walk * ni, R, (float)(1.0 / m->coord_scale), m->x);
  cudaError_t e = cudaGetLastError();
  // layer l: A = the walkers' activations [n_walk][K], B = W_l^T read from the BF16 copy
  // W_l[K][width] (row n of B is column n of W_l)
  const __nv_bfloat16* pb = m->pb;
  auto layer = [&](const float* a, int64_t K, int64_t oW, int64_t width, int kind, int64_t ob, float* o) {
    const GemmOperand A{a, K, 1, n_walk, K, 0};
    const GemmOperand B{pb + oW, 1, width, width, K, 1};
    const GemmEpilogue E{kind, o, width, 1, m->p + ob, nullptr, 0};
    return launch_gemm_bf16(A, B, K, E, st);
  };
  if (e == cudaSuccess) e = layer(m->x, ni, m->oW1, H, kEpiTanhBias, m->ob1, m->h1);
  if (e == cudaSuccess) e = layer(m->h1, H, m->oW2, H, kEpiTanhBias, m->ob2, m->h2);
  if (e == cudaSuccess) e = layer(m->h2, H, m->oW3, no, kEpiBias, m->ob3, out);
  return cuda_status(e);
}

mdet_status mdet_mlp_backward(mdet_mlp* m, int64_t n_walk, const float* dout, void* stream) {
  if (!m || n_walk < 0 || !dout || n_walk > m->cap) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  if (cudaSetDevice(m->device) != cudaSuccess) return MDET_E_CUDA;
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t ni = m->n_in, H = m->H, no = m->n_out;
  const __nv_bfloat16* pb = m->pb;
  // deltas: d2 = (dout W3^T) (1 - h2^2), d1 = (d2 W2^T) (1 - h1^2); B = W_l itself, row n of
  // W_l[n][.] over its width
  const GemmOperand Dout{dout, no, 1, n_walk, no, 0};
  cudaError_t e = launch_gemm_bf16(Dout, GemmOperand{pb + m->oW3, no, 1, H, no, 1}, no,
                                   GemmEpilogue{kEpiDtanh, m->d2, H, 1, nullptr, m->h2, H}, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(GemmOperand{m->d2, H, 1, n_walk, H, 0}, GemmOperand{pb + m->oW2, H, 1, H, H, 1}, H,
                         GemmEpilogue{kEpiDtanh, m->d1, H, 1, nullptr, m->h1, H}, st);
  // weight gradients, summed over the walkers (the GEMMs' K), 1,024 walkers per CTA:
  // gW3[k][j] = sum_w h2[w][k] dout[w][j], gW2[k][j] = sum_w h1[w][k] d2[w][j],
  // gW1[i][j] = sum_w x[w][i] d1[w][j] (computed as its transpose: rows j, columns i)
  const int64_t kpc = 1024;
  if (e == cudaSuccess)
    e = launch_gemm_bf16(GemmOperand{m->h2, 1, H, H, n_walk, 0}, GemmOperand{dout, 1, no, no, n_walk, 0}, kpc,
                         GemmEpilogue{kEpiAtomic, m->g + m->oW3, no, 1, nullptr, nullptr, 0}, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(GemmOperand{m->h1, 1, H, H, n_walk, 0}, GemmOperand{m->d2, 1, H, H, n_walk, 0}, kpc,
                         GemmEpilogue{kEpiAtomic, m->g + m->oW2, H, 1, nullptr, nullptr, 0}, st);
  if (e == cudaSuccess)
    e = launch_gemm_bf16(GemmOperand{m->d1, 1, H, H, n_walk, 0}, GemmOperand{m->x, 1, ni, ni, n_walk, 0}, kpc,
                         GemmEpilogue{kEpiAtomic, m->g + m->oW1, 1, H, nullptr, nullptr, 0}, st);
  if (e != cudaSuccess) return cuda_status(e);
  // bias gradients from the unrounded deltas
  const ColSumJobs jobs{{{dout, (int)no, m->g + m->ob3}, {m->d2, (int)H, m->g + m->ob2}, {m->d1, (int)H, m->g + m->ob1}}};
  const int64_t per = 256;
  const dim3 grid(blocks(std::max(no, H), 128), (unsigned)((n_walk + per - 1) / per), 3);
  k_bias_grad<<<grid, 128, 0, st>>>(jobs, n_walk, per);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_mlp_zero_grad(mdet_mlp* m, void* stream) {
  if (!m) return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return MDET_E_CUDA;
  return cuda_status(cudaMemsetAsync(m->g, 0, sizeof(float) * m->n_params, (cudaStream_t)stream));
}

mdet_status mdet_mlp_adam(mdet_mlp* m, double lr, double beta1, double beta2, double eps, int64_t t, void* stream) {
  if (!m || t < 1) return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return MDET_E_CUDA;
  const float c1 = (float)(1.0 - std::pow(beta1, (double)t)), c2 = (float)(1.0 - std::pow(beta2, (double)t));
  k_adam<<<blocks(m->n_params, 256), 256, 0, (cudaStream_t)stream>>>(m->n_params, m->p, m->g, m->m1, m->m2, m->pb,
                                                                      (float)lr, (float)beta1, (float)beta2,
                                                                      (float)eps, c1, c2);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_mlp_nll_grad(const mdet_mlp* m, int64_t n_walk, const double* R0, const double* R1, const float* out,
                              float* dout, double* loss, void* stream) {
  if (!m || n_walk < 1 || !R0 || !R1 || !out || !dout || !loss) return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return MDET_E_CUDA;
  if (cudaMemsetAsync(loss, 0, sizeof(double), (cudaStream_t)stream) != cudaSuccess) return MDET_E_CUDA;
  k_nll<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(head(m), n_walk, R0, R1, out, dout, loss);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_mlp_esjd_grad(const mdet_mlp* m, int64_t n_walk, const double* R, const double* R_new,
                               const float* out, const float* out_new, const double* log_abs_psi,
                               const double* log_abs_psi_new, const int8_t* sign_new, const double* drift,
                               const double* drift_new, const double* grad_new, int langevin, double jump_len2,
                               double speed_beta, float* dout, float* dout_new, double* objective, void* stream) {
  if (!m || n_walk < 1 || !R || !R_new || !out || !out_new || !log_abs_psi || !log_abs_psi_new || !sign_new ||
      !grad_new || !dout || !dout_new || !objective || (langevin && (!drift || !drift_new)))
    return MDET_E_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return MDET_E_CUDA;
  if (cudaMemsetAsync(objective, 0, 2 * sizeof(double), (cudaStream_t)stream) != cudaSuccess) return MDET_E_CUDA;
  k_esjd<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(
      head(m), n_walk, R, R_new, out, out_new, log_abs_psi, log_abs_psi_new, sign_new, langevin ? drift : grad_new,
      langevin ? drift_new : grad_new, grad_new, langevin != 0, jump_len2, speed_beta, dout, dout_new, objective);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_propose_mlp(const mdet_mlp* m, int64_t n_walk, const double* R, const float* out,
                                 const double* drift, uint64_t seed, uint64_t step, double* R_new, double* log_q_fwd,
                                 void* stream) {
  if (!m || n_walk < 0) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  if (!R || !out || !R_new || !log_q_fwd) return MDET_E_ARG;
  k_propose_mlp<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(head(m), n_walk, R, out, drift, seed, step,
                                                                        R_new, log_q_fwd);
  return cuda_status(cudaGetLastError());
}

mdet_status mdet_vmc_reverse_mlp(const mdet_mlp* m, int64_t n_walk, const double* R, const double* R_new,
                                 const float* out_new, const double* drift_new, double* log_q_rev, void* stream) {
  if (!m || n_walk < 0) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  if (!R || !R_new || !out_new || !log_q_rev) return MDET_E_ARG;
  k_reverse_mlp<<<blocks(n_walk, 128), 128, 0, (cudaStream_t)stream>>>(head(m), n_walk, R, R_new, out_new,
                                                                        drift_new, log_q_rev);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"

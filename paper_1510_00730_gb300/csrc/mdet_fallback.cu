// Stability fallback: walkers whose reference Slater matrix is too
// ill-conditioned for the reference-relative ratio table are re-evaluated by
// the plain cubic method (LU of every distinct determinant, the paper's
// "no Sherman-Morrison" mode of Table 2, and its O(N^3) fallback of Sec. 2.2),
// in FP64, followed by their own contraction and epilogue (Eqs. 2, 5-8).
//
//   k_fb_list    compacts the flagged walkers into a device list (no host sync)
//   k_fb_dets    one thread per (determinant, flagged walker): in-place
//                Gauss-Jordan inversion with partial pivoting of the Slater
//                matrix, D as a signed mantissa times 2^e, and (d_{i mu} D)/D = sum_a d_mu phi_{o_a}(r_i) (S^-1)_{a i}
//   k_fb_scale   per flagged walker: common power-of-two scale of its determinant values
//   k_fb_rows    fixed grid over (walker, 64 rows) items, a warp per row: v = C d_dn, u = C^T d_up, Psi, gradient
//                and Laplacian sums, reduced per block then with atomics
//   k_fb_out     per flagged walker: potential energy and outputs
//
// Mixed precision first escalates: the flagged walkers (at most the cap) are
// gathered (k_esc_gather), evaluated again by the FP64 ratio-table kernels on a
// scratch of their own, and only those whose FP64 estimate still exceeds the
// tolerance go through the full-LU path above; k_esc_scatter writes the results
// back to the walkers' slots.
#include <algorithm>
#include <climits>
#include <cfloat>
#include <cmath>

#include "mdet_internal.h"

namespace mdet {

namespace {

constexpr int kFbMax = MDET_FALLBACK_MAX_SPIN;

__global__ void k_fb_list(const DevProblem P, uint32_t* __restrict__ wstat, uint32_t* __restrict__ status,
                          int64_t n_walk, int* __restrict__ list) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  const uint32_t st = wstat[w];
  if (!(st & MDET_WS_FALLBACK)) return;
  const int i = atomicAdd(list, 1);
  if (i < P.fallback_cap) {
    list[1 + i] = (int)w;
  } else {  // beyond the fallback capacity: keep the table result, flagged
    const uint32_t s2 = (st & ~MDET_WS_FALLBACK) | MDET_WS_REF_ILLCOND;
    wstat[w] = s2;
    if (status) status[w] = s2;
  }
}

__global__ void __launch_bounds__(64) k_fb_dets(DevProblem P, DevScratch S) {
  const int slot = blockIdx.y;
  const int count = min(S.fb_list[0], P.fallback_cap);
  if (slot >= count) return;
  const int64_t w = S.fb_list[1 + slot];
  extern __shared__ double fsm[];
  const int nu = P.n_up, nd = P.n_dn, N = nu + nd, M = P.n_mo, nmax = max(nu, nd);
  const int nu_det = P.n_det_sp[0], ntot = nu_det + P.n_det_sp[1];
  const int stride = 2 + 4 * nmax;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntot) return;
  const int sp = t < nu_det ? 0 : 1;
  const int n = sp ? nd : nu, e0 = sp ? nu : 0;
  const Exc e = P.exc[sp][sp ? t - nu_det : t];
  int cols[kFbMax];
  const int* occ = P.ref_occ + sp * kMaxSpin;
  for (int a = 0; a < n; a++) cols[a] = occ[a];
  for (int q = 0; q < e.k; q++) cols[e.h[q]] = e.p[q];
  double* A = fsm + threadIdx.x * nmax * nmax;  // n x n, row-major, stride n
  const double* ph = S.phi + (size_t)w * 5 * N * M;
  for (int i = 0; i < n; i++)
    for (int a = 0; a < n; a++) A[i * n + a] = ph[(size_t)(e0 + i) * M + cols[a]];
  int piv[kFbMax];
  // |D| = pm 2^pe with pm in [0.5, 1), no logarithm; pivots compared by the integer order of
  // their magnitude bits (the order of the magnitudes), the sign kept as a bit, so that the
  // FP64 pipe runs the elimination and not the bookkeeping
  double pm = 1.0;
  int pe = 0, neg = e.eps < 0;
  bool singular = false;
  for (int k = 0; k < n; k++) {
    int p = k;
    unsigned long long best = (unsigned long long)__double_as_longlong(A[k * n + k]) & 0x7fffffffffffffffULL;
    for (int i = k + 1; i < n; i++) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(A[i * n + k]) & 0x7fffffffffffffffULL;
      if (v > best) {
        best = v;
        p = i;
      }
    }
    piv[k] = p;
    if (best == 0ULL || best >= 0x7ff0000000000000ULL) {  // no nonzero pivot, or Inf / NaN: singular
      singular = true;
      break;
    }
    if (p != k) {
      neg ^= 1;
      for (int j = 0; j < n; j++) {
        const double tmp = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = tmp;
      }
    }
    const double d = A[k * n + k];
    {
      const long long b = __double_as_longlong(d);
      neg ^= (int)((unsigned long long)b >> 63);
      int ex = (int)((b >> 52) & 0x7ff);
      long long bn = b;
      if (ex == 0) {  // a subnormal pivot: scaled by 2^64 into the normal range (exact)
        bn = __double_as_longlong(d * 0x1p64);
        ex = (int)((bn >> 52) & 0x7ff) - 64;
      }
      pm *= __longlong_as_double((bn & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
      pe += ex - 1022;
      const long long bm = __double_as_longlong(pm);  // back into [0.5, 1)
      pe += (int)((bm >> 52) & 0x7ff) - 1022;
      pm = __longlong_as_double((bm & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
    }
    const double inv = 1.0 / d;
    A[k * n + k] = 1.0;
    for (int j = 0; j < n; j++) A[k * n + j] *= inv;
    for (int i = 0; i < n; i++) {
      if (i == k) continue;
      const double f = A[i * n + k];
      A[i * n + k] = 0.0;
      if ((__double_as_longlong(f) << 1) != 0)
        for (int j = 0; j < n; j++) A[i * n + j] = fma(-f, A[k * n + j], A[i * n + j]);
    }
  }
  double* rec = S.fb + ((size_t)slot * ntot + t) * stride;
  if (singular) {
    rec[0] = -INFINITY;
    rec[1] = 0.0;
    for (int q = 0; q < 4 * n; q++) rec[2 + q] = 0.0;
    return;
  }
  // (P S)^-1 = S^-1 P^-1: undo the row interchanges on the columns, last first
  for (int k = n - 1; k >= 0; k--)
    if (piv[k] != k)
      for (int i = 0; i < n; i++) {
        const double tmp = A[i * n + k];
        A[i * n + k] = A[i * n + piv[k]];
        A[i * n + piv[k]] = tmp;
      }
  rec[0] = __longlong_as_double((long long)pe);  // the exponent, an integer in the bits
  rec[1] = __longlong_as_double(__double_as_longlong(pm) | ((long long)neg << 63));  // D / 2^pe
  for (int i = 0; i < n; i++)
    for (int mu = 0; mu < 4; mu++) {
      const double* dph = ph + ((size_t)(1 + mu) * N + e0 + i) * M;
      double acc = 0.0;
      for (int a = 0; a < n; a++) acc = fma(dph[cols[a]], A[a * n + i], acc);
      rec[2 + i * 4 + mu] = acc;
    }
}

// threads per flagged walker of k_fb_scale (its exponentials and two block reductions over every
// distinct determinant)
constexpr int kFbScaleThreads = 256;

__device__ __forceinline__ long long block_max_ll(long long v, long long* red) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  long long r = LLONG_MIN;
  for (int q = 0; q < (int)(blockDim.x >> 5); q++) r = max(r, red[q]);
  return r;
}

// Per flagged walker: common scale per spin, 2^L with L the largest exponent of its nonzero
// determinants (each stored as a signed mantissa in [0.5, 1) times 2^e), the scaled values
// d = mantissa 2^(e - L) in place and in a contiguous copy for the gathers (exact, by the
// exponent bits; below 2^-1022 of the largest they are zero), and cleared accumulators.
// acc layout per slot: [0] L_up ln 2, [1] L_dn ln 2, [2] Psi, [3..3+4N) G[i][mu].
__global__ void __launch_bounds__(kFbScaleThreads) k_fb_scale(DevProblem P, DevScratch S) {
  const int slot = blockIdx.x;
  const int count = min(S.fb_list[0], P.fallback_cap);
  if (slot >= count) return;
  const int nu = P.n_up, nd = P.n_dn, N = nu + nd, nmax = max(nu, nd);
  const int nu_det = P.n_det_sp[0], ntot = nu_det + P.n_det_sp[1];
  const int stride = 2 + 4 * nmax;
  double* rec = S.fb + (size_t)slot * ntot * stride;
  double* dv = S.fb + (size_t)P.fallback_cap * ntot * stride + (size_t)slot * ntot;
  double* acc = S.fb_acc + (size_t)slot * (3 + 4 * 2 * kFbMax);
  __shared__ long long red[kFbScaleThreads / 32];
  long long lu = LLONG_MIN, ld = LLONG_MIN;
  for (int t = threadIdx.x; t < ntot; t += blockDim.x)
    if ((__double_as_longlong(rec[(size_t)t * stride + 1]) << 1) != 0) {  // a nonzero determinant
      const long long e = __double_as_longlong(rec[(size_t)t * stride]);
      if (t < nu_det) lu = max(lu, e);
      else ld = max(ld, e);
    }
  long long Lu = block_max_ll(lu, red);
  long long Ld = block_max_ll(ld, red);
  if (Lu == LLONG_MIN) Lu = 0;
  if (Ld == LLONG_MIN) Ld = 0;
  for (int t = threadIdx.x; t < ntot; t += blockDim.x) {
    double* r = rec + (size_t)t * stride;
    const long long m = __double_as_longlong(r[1]);
    double d = 0.0;
    if ((m << 1) != 0) {
      const long long ex = 1022 + __double_as_longlong(r[0]) - (t < nu_det ? Lu : Ld);  // <= 1022
      if (ex >= 1) d = __longlong_as_double((m & ~(0x7ffLL << 52)) | (ex << 52));
    }
    r[0] = d;
    dv[t] = d;
  }
  for (int q = threadIdx.x; q < 1 + 4 * N; q += blockDim.x) acc[2 + q] = 0.0;
  if (threadIdx.x == 0) {
    acc[0] = (double)Lu * 0.69314718055994530942;
    acc[1] = (double)Ld * 0.69314718055994530942;
  }
}

// grid (ceil(ntot / 256), count slots): one thread per up row (v = C d_dn,
// Psi and the up-electron sums) or down column (u = C^T d_up, the
// down-electron sums); block sums in shared memory, then one atomic per value.
// distinct determinants per work item of k_fb_rows, one per warp: the longest rows of C hold
// thousands of nonzeros, and a warp that walked eight of them in turn set the kernel's latency
constexpr int kFbRowsPerItem = 8;

__global__ void __launch_bounds__(256) k_fb_rows(DevProblem P, DevScratch S) {
  const int count = min(S.fb_list[0], P.fallback_cap);
  const int nu = P.n_up, nd = P.n_dn, N = nu + nd, nmax = max(nu, nd);
  const int nu_det = P.n_det_sp[0], ntot = nu_det + P.n_det_sp[1];
  const int stride = 2 + 4 * nmax;
  const int n_rg = (ntot + kFbRowsPerItem - 1) / kFbRowsPerItem;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double G[1 + 4 * 2 * kFbMax];  // Psi, then G
  // work items (flagged walker, group of 64 distinct determinants) over a fixed grid: a batch
  // without flagged walkers costs one small launch
  for (int64_t item = blockIdx.x; item < (int64_t)count * n_rg; item += gridDim.x) {
    const int slot = (int)(item / n_rg), rg = (int)(item - (int64_t)slot * n_rg);
    const double* rec = S.fb + (size_t)slot * ntot * stride;
    const double* dv = S.fb + (size_t)P.fallback_cap * ntot * stride + (size_t)slot * ntot;
    for (int q = threadIdx.x; q < 1 + 4 * N; q += blockDim.x) G[q] = 0.0;
    __syncthreads();
    // one warp per distinct determinant: its row (up) or column (down) of C, whose length
    // varies by orders of magnitude, is split over the lanes and reduced with shuffles
    for (int t = rg * kFbRowsPerItem + warp; t < min(ntot, (rg + 1) * kFbRowsPerItem); t += blockDim.x >> 5) {
      const bool up = t < nu_det;
      double v = 0.0;
      if (up) {
        for (int k = P.csr_ptr[t] + lane; k < P.csr_ptr[t + 1]; k += 32)
          v = fma(P.csr_val[k], dv[nu_det + P.csr_col[k]], v);
      } else {
        const int J = t - nu_det;
        for (int k = P.csc_ptr[J] + lane; k < P.csc_ptr[J + 1]; k += 32) v = fma(P.csc_val[k], dv[P.csc_row[k]], v);
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      const double* r = rec + (size_t)t * stride;
      const double vd = v * r[0];
      if (vd != 0.0) {
        if (up) {
          if (lane == 0) atomicAdd(&G[0], vd);
          for (int q = lane; q < 4 * nu; q += 32) atomicAdd(&G[1 + q], vd * r[2 + q]);
        } else {
          for (int q = lane; q < 4 * nd; q += 32) atomicAdd(&G[1 + 4 * nu + q], vd * r[2 + q]);
        }
      }
    }
    __syncthreads();
    double* acc = S.fb_acc + (size_t)slot * (3 + 4 * 2 * kFbMax);
    for (int q = threadIdx.x; q < 1 + 4 * N; q += blockDim.x)
      if (G[q] != 0.0) atomicAdd(&acc[2 + q], G[q]);
    __syncthreads();
  }
}

// Per flagged walker: potential energy and the outputs.
__global__ void __launch_bounds__(64) k_fb_out(DevProblem P, DevScratch S, const double* __restrict__ R,
                                               double* __restrict__ log_abs_psi, int8_t* __restrict__ sign,
                                               double* __restrict__ grad, double* __restrict__ lap,
                                               double* __restrict__ e_local, uint32_t* __restrict__ status) {
  const int slot = blockIdx.x;
  const int count = min(S.fb_list[0], P.fallback_cap);
  if (slot >= count) return;
  const int64_t w = S.fb_list[1 + slot];
  const int nu = P.n_up, nd = P.n_dn, N = nu + nd;
  const double* acc = S.fb_acc + (size_t)slot * (3 + 4 * 2 * kFbMax);
  const double* G = acc + 3;
  __shared__ double red[2];
  double vp = 0.0;
  const double* rr = R + w * N * 3;
  for (int q = threadIdx.x; q < N * P.n_nuc; q += blockDim.x) {
    const int i = q / P.n_nuc, A = q - i * P.n_nuc;
    const double dx = rr[3 * i] - P.nuc_xyz[3 * A], dy = rr[3 * i + 1] - P.nuc_xyz[3 * A + 1],
                 dz = rr[3 * i + 2] - P.nuc_xyz[3 * A + 2];
    vp -= P.Z[A] / sqrt(dx * dx + dy * dy + dz * dz);
  }
  for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
    const int i = q / N, j = q - i * N;
    if (j <= i) continue;
    const double dx = rr[3 * i] - rr[3 * j], dy = rr[3 * i + 1] - rr[3 * j + 1], dz = rr[3 * i + 2] - rr[3 * j + 2];
    vp += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
  }
  if (threadIdx.x == 0)
    for (int A = 0; A < P.n_nuc; A++)
      for (int B = A + 1; B < P.n_nuc; B++) {
        const double dx = P.nuc_xyz[3 * A] - P.nuc_xyz[3 * B], dy = P.nuc_xyz[3 * A + 1] - P.nuc_xyz[3 * B + 1],
                     dz = P.nuc_xyz[3 * A + 2] - P.nuc_xyz[3 * B + 2];
        vp += P.Z[A] * P.Z[B] / sqrt(dx * dx + dy * dy + dz * dz);
      }
#pragma unroll
  for (int off = 16; off; off >>= 1) vp += __shfl_xor_sync(0xffffffffu, vp, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vp;
  __syncthreads();
  const double Ps = acc[2];
  const double inv = 1.0 / Ps;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    grad[(w * N + i) * 3 + 0] = G[4 * i + 0] * inv;
    grad[(w * N + i) * 3 + 1] = G[4 * i + 1] * inv;
    grad[(w * N + i) * 3 + 2] = G[4 * i + 2] * inv;
    lap[w * N + i] = G[4 * i + 3] * inv;
  }
  if (threadIdx.x == 0) {
    double tl = 0.0;
    for (int i = 0; i < N; i++) tl += G[4 * i + 3];
    const double el = -0.5 * tl * inv + red[0] + red[1];
    const double lg = log(fabs(Ps)) + acc[0] + acc[1];
    log_abs_psi[w] = lg;
    sign[w] = (int8_t)((Ps > 0.0) - (Ps < 0.0));
    if (e_local) e_local[w] = el;
    uint32_t st = (S.wstat[w] & (MDET_WS_REF_SINGULAR | MDET_WS_REF_ILLCOND)) | MDET_WS_FALLBACK;
    if (Ps == 0.0) st |= MDET_WS_PSI_ZERO;
    if (!isfinite(lg) || !isfinite(el)) st |= MDET_WS_NONFINITE;
    S.wstat[w] = st;
    if (status) status[w] = st;
  }
}

// Escalation: the listed walkers (count, then indices; at most cap) are copied to
// the front of Re with their magnitude sums sum |c r r| (psia, from the evaluation
// that flagged them: the conditioning of the CI sum needs no FP64 recomputation),
// and *live receives min(count, cap) for the FP64 kernels.
__global__ void k_esc_gather(const int* __restrict__ list, int cap, int n3, const double* __restrict__ R,
                             double* __restrict__ Re, int* __restrict__ live, const float* __restrict__ psia,
                             float* __restrict__ psia_e) {
  const int count = min(list[0], cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) *live = count;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)count * n3;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n3, q = t - i * n3;
    Re[t] = R[(int64_t)list[1 + i] * n3 + q];
    if (q == 0) psia_e[i] = psia[list[1 + i]];
  }
}

// Without the FP64 table every gathered walker goes to full LU.
__global__ void k_esc_mark(const int* __restrict__ live, uint32_t* __restrict__ wstat, int cap) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cap && i < *live) wstat[i] = MDET_WS_FALLBACK;
}

// Escalation: the results of slot i go back to walker list[1 + i], whose status
// becomes that of its FP64 re-evaluation plus or_bits. grid cap, block 64.
__global__ void __launch_bounds__(64) k_esc_scatter(const int* __restrict__ list, int cap, int N,
                                                    const EscOut e, uint32_t or_bits, double* __restrict__ log_abs_psi,
                                                    int8_t* __restrict__ sign, double* __restrict__ grad,
                                                    double* __restrict__ lap, double* __restrict__ e_local,
                                                    uint32_t* __restrict__ status, uint32_t* __restrict__ wstat) {
  const int count = min(list[0], cap);
  const int i = blockIdx.x;
  if (i >= count) return;
  const int64_t w = list[1 + i];
  for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) grad[w * 3 * N + q] = e.grad[(int64_t)i * 3 * N + q];
  for (int q = threadIdx.x; q < N; q += blockDim.x) lap[w * N + q] = e.lap[(int64_t)i * N + q];
  if (threadIdx.x == 0) {
    log_abs_psi[w] = e.log_abs_psi[i];
    sign[w] = e.sign[i];
    if (e_local) e_local[w] = e.e_local[i];
    const uint32_t st = e.status[i] | or_bits;
    wstat[w] = st;
    if (status) status[w] = st;
  }
}

}  // namespace

cudaError_t launch_fb_list(const DevProblem& P, uint32_t* wstat, uint32_t* status, int64_t n_walk, int* list,
                           cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(list, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_fb_list<<<(unsigned)((n_walk + 255) / 256), 256, 0, st>>>(P, wstat, status, n_walk, list);
  return cudaGetLastError();
}

cudaError_t launch_esc_gather(const int* list, int cap, int n3, const double* R, double* Re, int* live,
                              const float* psia, float* psia_e, cudaStream_t st) {
  const int64_t total = (int64_t)cap * n3;
  k_esc_gather<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 1024)), 256, 0, st>>>(
      list, cap, n3, R, Re, live, psia, psia_e);
  return cudaGetLastError();
}

cudaError_t launch_esc_mark(const int* live, uint32_t* wstat, int cap, cudaStream_t st) {
  k_esc_mark<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(live, wstat, cap);
  return cudaGetLastError();
}

cudaError_t launch_esc_scatter(const int* list, int cap, int N, const EscOut& e, uint32_t or_bits,
                               double* log_abs_psi, int8_t* sign, double* grad, double* lap, double* e_local,
                               uint32_t* status, uint32_t* wstat, cudaStream_t st) {
  k_esc_scatter<<<(unsigned)cap, 64, 0, st>>>(list, cap, N, e, or_bits, log_abs_psi, sign, grad, lap, e_local, status,
                                              wstat);
  return cudaGetLastError();
}

cudaError_t launch_fallback(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                            double* log_abs_psi, int8_t* sign, double* grad, double* lap, double* e_local,
                            uint32_t* status, cudaStream_t st) {
  if (!(P.fallback_tol > 0.0) || !S.fb || P.n_up > kFbMax) return cudaSuccess;
  cudaError_t e = launch_fb_list(P, S.wstat, status, n_walk, S.fb_list, st);
  if (e != cudaSuccess) return e;
  const int nmax = P.n_up > P.n_dn ? P.n_up : P.n_dn;
  const int ntot = P.n_det_sp[0] + P.n_det_sp[1];
  // one thread per determinant, its Slater matrix in shared memory: 32-thread blocks from 12
  // electrons per spin up, so that three blocks (96 threads) fit an SM at 17 instead of one of 64
  const int tpb = nmax >= 12 ? 32 : 64;
  const size_t smem = sizeof(double) * tpb * nmax * nmax;
  static SmemOptIn opt;
  if ((e = opt.ensure(k_fb_dets, smem)) != cudaSuccess) return e;
  dim3 g1((ntot + tpb - 1) / tpb, P.fallback_cap);
  k_fb_dets<<<g1, tpb, smem, st>>>(P, S);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_fb_scale<<<P.fallback_cap, kFbScaleThreads, 0, st>>>(P, S);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  static int n_sm = 0;
  if (!n_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0) n_sm = 132;
  }
  const int64_t items = (int64_t)P.fallback_cap * ((ntot + kFbRowsPerItem - 1) / kFbRowsPerItem);
  k_fb_rows<<<(unsigned)std::min<int64_t>(items, 4 * n_sm), 256, 0, st>>>(P, S);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_fb_out<<<P.fallback_cap, 64, 0, st>>>(P, S, R, log_abs_psi, sign, grad, lap, e_local, status);
  return cudaGetLastError();
}

}  // namespace mdet

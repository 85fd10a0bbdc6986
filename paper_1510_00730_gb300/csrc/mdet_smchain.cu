// mdet_smchain.cu -- the paper's sequential route to the determinant values
// (Sec. 2.2), kept beside the table method for comparison. For each walker and
// spin, the distinct determinants are visited in the order of the key of Eq. 3:
// the first one gets a Gauss-Jordan inverse with partial pivoting, and every
// following one is reached from its predecessor by in-place Sherman-Morrison
// column substitutions (Eq. 4), one column at a time. A substitution whose
// ratio has modulus below 1e-3 is deferred and retried after the others; a
// round of retries that applies none of them cancels the updates, and the
// determinant is recomputed by a full inverse (O(N^3)).
//
// One warp per (walker, spin). The inverse lives in shared memory: lanes own
// its rows (orbital index a) when forming w = S^-1 phi_p, and its columns
// (electron index i) for the rank-one update.

#include <cmath>

#include "mdet_internal.h"

namespace mdet {

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr double kSmMin = 1e-3;  // the paper's threshold on |ratio|

// component 0 (the value) of the orbital array: FP64, or double-float pairs in a mixed context
__device__ __forceinline__ double phi_val(const double* __restrict__ phi, int64_t w, int n_elec, int n_mo, int e,
                                          int m, int df) {
  const size_t ix = ((w * 5 + 0) * n_elec + e) * n_mo + m;
  if (df) {
    const float2 v = reinterpret_cast<const float2*>(phi)[ix];
    return (double)v.x + (double)v.y;
  }
  return phi[ix];
}

// Gauss-Jordan inverse of S[i][a] = phi_{occ[a]}(r_{e0+i}) with partial
// pivoting; A, B: [N][N+1] shared scratch (B = S^-1 on exit, B[a][i]).
// Returns log|det| in *ld and the sign in *sg (0 when singular).
__device__ void full_inverse(const double* __restrict__ phi, int df, int64_t w, int n_elec, int n_mo, int e0, int N,
                             const uint8_t* occ, double* A, double* B, double* ld, double* sg) {
  const int lane = threadIdx.x & 31, P = N + 1;
  if (lane < N) {
    for (int a = 0; a < N; a++) {
      A[lane * P + a] = phi_val(phi, w, n_elec, n_mo, e0 + lane, occ[a], df);
      B[lane * P + a] = lane == a ? 1.0 : 0.0;
    }
  }
  __syncwarp();
  double logd = 0.0, sign = 1.0;
  for (int p = 0; p < N; p++) {
    // pivot: largest |A[row][p]| over rows >= p (lowest row on ties)
    double v = (lane >= p && lane < N) ? fabs(A[lane * P + p]) : -1.0;
    int r = lane;
    for (int off = 16; off; off >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
      const int r2 = __shfl_xor_sync(0xffffffffu, r, off);
      if (v2 > v || (v2 == v && r2 < r)) {
        v = v2;
        r = r2;
      }
    }
    if (!(v > 0.0)) {
      *ld = -INFINITY;
      *sg = 0.0;
      return;
    }
    if (r != p) {
      if (lane < N) {
        double t = A[p * P + lane];
        A[p * P + lane] = A[r * P + lane];
        A[r * P + lane] = t;
        t = B[p * P + lane];
        B[p * P + lane] = B[r * P + lane];
        B[r * P + lane] = t;
      }
      sign = -sign;
    }
    __syncwarp();
    const double piv = A[p * P + p];
    logd += log(fabs(piv));
    if (piv < 0.0) sign = -sign;
    __syncwarp();
    if (lane < N) {
      A[p * P + lane] /= piv;
      B[p * P + lane] /= piv;
    }
    __syncwarp();
    if (lane < N && lane != p) {
      const double f = A[lane * P + p];
      for (int j = 0; j < N; j++) {
        A[lane * P + j] -= f * A[p * P + j];
        B[lane * P + j] -= f * B[p * P + j];
      }
    }
    __syncwarp();
  }
  *ld = logd;
  *sg = sign;
}

// Sign of the permutation that sorts cols[0..N) ascending.
__device__ __forceinline__ double parity(const int* cols, int N) {
  const int lane = threadIdx.x & 31;
  int inv = 0;
  if (lane < N)
    for (int b = lane + 1; b < N; b++) inv += cols[lane] > cols[b];
  for (int off = 16; off; off >>= 1) inv += __shfl_xor_sync(0xffffffffu, inv, off);
  return (inv & 1) ? -1.0 : 1.0;
}

// Shared memory of one warp for matrices of order N: A and B [N][N+1], w [32], cols [32].
__host__ __device__ constexpr int warp_doubles(int N) { return 2 * N * (N + 1) + 32 + 16; }

__global__ void k_sm_chain(DevProblem P, DevScratch S, int spin, const SmStep* __restrict__ steps, int n_steps,
                           int64_t n_walk, double* __restrict__ r, int64_t ld_r, int32_t* __restrict__ n_inv,
                           int32_t* __restrict__ n_subst) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  const int N = spin == 0 ? P.n_up : P.n_dn, e0 = spin == 0 ? 0 : P.n_up, Pd = N + 1;
  double* A = sm + (size_t)warp * warp_doubles(N);
  double* B = A + N * Pd;
  double* wv = B + N * Pd;                // w = S^-1 phi_p, [32]
  int* cols = (int*)(wv + 32);            // current orbital of each column, [32]
  if (w >= n_walk || N == 0) return;
  const double ld0 = S.ld0[w * 2 + spin], sg0 = S.sg0[w * 2 + spin];
  const int r_off = spin == 0 ? 0 : P.n_det_sp[0];
  // the running determinant as dm * 2^de (dm in [0.5, 1) in modulus, with its sign): no FP64 log or exp per
  // substitution; the ratio to D_ref uses 1/D_ref when that is representable
  const bool scaled = fabs(ld0) < 600.0;
  const double inv_ref = scaled ? sg0 * exp(-ld0) : 0.0;
  double logd = 0.0, sign = 0.0, dm = 0.0;
  int de = 0;
  int inv = 0, subst = 0;
  bool fresh = true;  // the next determinant needs a full inverse
  for (int t = 0; t < n_steps; t++) {
    const SmStep st = steps[t];
    bool rebuild = fresh || st.n_sub > kSmMaxSub;
    if (!rebuild) {
      // substitutions hole[s] -> part[s]; pending as a bit mask, retried until none is left
      unsigned pending = (1u << st.n_sub) - 1u;
      while (pending) {
        unsigned failed = 0;
        for (int s = 0; s < st.n_sub; s++) {
          if (!((pending >> s) & 1u)) continue;
          const unsigned hit = __ballot_sync(0xffffffffu, lane < N && cols[lane] == st.hole[s]);
          const int k = __ffs(hit) - 1;
          if (k < 0) {  // not a column of the current matrix (inconsistent records): recompute
            failed |= 1u << s;
            continue;
          }
          // w_a = sum_i S^-1[a][i] phi_part(r_i): one orbital value per lane, broadcast by shuffles
          const double pv = lane < N ? phi_val(S.phi, w, P.n_elec, P.n_mo, e0 + lane, st.part[s], P.phi_df) : 0.0;
          double acc = 0.0;
          for (int i = 0; i < N; i++) acc += (lane < N ? B[lane * Pd + i] : 0.0) * __shfl_sync(0xffffffffu, pv, i);
          if (lane < N) wv[lane] = acc;
          __syncwarp();
          const double wk = wv[k];
          if (!(fabs(wk) >= kSmMin)) {  // Sec. 2.2: deferred (also a NaN ratio)
            failed |= 1u << s;
            __syncwarp();
            continue;
          }
          // in-place column substitution: row k /= wk, rows a != k -= w_a / wk * (old row k); lane = column i
          const double rk = 1.0 / wk;
          if (lane < N) {
            const double bk = B[k * Pd + lane] * rk;
            for (int a = 0; a < N; a++) B[a * Pd + lane] = a == k ? bk : B[a * Pd + lane] - wv[a] * bk;
          }
          __syncwarp();
          if (lane == 0) cols[k] = st.part[s];
          __syncwarp();
          int ex;
          dm = frexp(dm * wk, &ex);
          de += ex;
          subst++;
        }
        if (failed == pending) {  // no progress: cancel and recompute from scratch
          rebuild = true;
          break;
        }
        pending = failed;
      }
    }
    if (rebuild) {
      full_inverse(S.phi, P.phi_df, w, P.n_elec, P.n_mo, e0, N, st.occ, A, B, &logd, &sign);
      if (lane < N) cols[lane] = st.occ[lane];
      __syncwarp();
      inv++;
      // log|D| = logd -> dm 2^de with dm = sign * 2^f, f in [-1, 0)
      if (sign != 0.0) {
        const double l2 = logd * 1.4426950408889634;  // log2(e)
        de = (int)floor(l2) + 1;
        dm = sign * exp2(l2 - (double)de);
      } else {
        dm = 0.0;
        de = 0;
      }
    }
    // determinant with ascending columns = det(current matrix) * parity(cols)
    const double par = parity(cols, N);
    double ratio;
    if (dm == 0.0)
      ratio = 0.0;
    else if (scaled)
      ratio = ldexp(dm * par * inv_ref, de);
    else
      ratio = (dm < 0.0 ? -par : par) * sg0 * exp(log(fabs(dm)) + (double)de * 0.6931471805599453 - ld0);
    if (lane == 0) r[(int64_t)(r_off + st.ctx) * ld_r + w] = ratio;
    fresh = dm == 0.0;  // after a singular determinant the next one starts from scratch
  }
  if (lane == 0) {
    atomicAdd(n_inv + w, inv);
    atomicAdd(n_subst + w, subst);
  }
}

}  // namespace

size_t sm_chain_smem_bytes(int n) { return (size_t)kWarpsPerBlock * warp_doubles(n) * sizeof(double); }

cudaError_t launch_sm_chain(const DevProblem& P, const DevScratch& S, int spin, const SmStep* steps, int n_steps,
                            int64_t n_walk, double* r, int64_t ld_r, int32_t* n_inv, int32_t* n_subst,
                            cudaStream_t st) {
  if (n_walk <= 0 || n_steps <= 0) return cudaSuccess;
  const size_t smem = sm_chain_smem_bytes(spin == 0 ? P.n_up : P.n_dn);
  cudaError_t e = cudaFuncSetAttribute(k_sm_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((n_walk + kWarpsPerBlock - 1) / kWarpsPerBlock);
  k_sm_chain<<<grid, 32 * kWarpsPerBlock, smem, st>>>(P, S, spin, steps, n_steps, n_walk, r, ld_r, n_inv, n_subst);
  return cudaGetLastError();
}

}  // namespace mdet

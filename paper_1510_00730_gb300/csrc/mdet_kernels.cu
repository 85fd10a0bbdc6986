// FP64 kernels of one evaluation (Sec. 2.2-2.4), in launch order:
//   k_mo_f64         orbitals and their derivatives at every electron (Sec. 2)
//   k_ref            LU with partial pivoting of each reference Slater matrix,
//                    its inverse A, log|D_ref|, the table T = A Phi and the
//                    single-determinant derivatives g (Sec. 2.2; Sec. 5 Table method)
//   k_ratio_f64      D_I / D_ref = eps_I det T[h_I, p_I] for every distinct
//                    spin determinant (k x k, k <= 4)
//   k_spmm_wm        v = C r_dn (plus Psi~ = r_up . v) and u = C^T r_up (Sec. 2.4),
//                    8 walkers per lane, walker-major output (k_spmm_df: the
//                    double-float option of the mixed path; k_spmm_f64: the
//                    walker-minor form used by the allocation-free entry point)
//   k_final          derivative aggregation and the per-walker epilogue (Eqs. 5-8)
// k_ref and k_final take a MIXED flag: the mixed-precision variants (and the
// mixed orbital and ratio kernels of mdet_kernels_mixed.cu) run the
// per-determinant work in double-float on the FP32 pipe; see df32.cuh.
//
// Notation. For spin s with n electrons (rows i) and reference occupied MOs
// o_1 < ... < o_n (columns a): S_ref[i][a] = phi_{o_a}(r_i), A = S_ref^-1
// (A[a][i]), T[a][m] = sum_i A[a][i] phi_m(r_i). A determinant I that replaces
// reference columns h_1..h_k by MOs p_1..p_k has
//   D_I / D_ref = eps_I det M_I,    M_I[alpha][beta] = T[h_alpha][p_beta]
// (generalised matrix-determinant lemma; eps_I reorders the columns ascending).
// Since row i of every Slater matrix depends on r_i only, the derivative
// d_{i mu} D_I / D_ref (mu = x, y, z, Laplacian) is the same ratio for the
// matrices with row i replaced by d_mu phi(r_i), which gives
//   d_{i mu} D_I / D_ref = eps_I [ g_{i mu} det M_I + sum_{alpha beta}
//                          cof(M_I)[alpha][beta] Y_{i mu}[p_beta] A[h_alpha][i] ]
//   g_{i mu} = sum_a A[a][i] d_mu phi_{o_a}(r_i),
//   Y_{i mu}[m] = d_mu phi_m(r_i) - sum_b d_mu phi_{o_b}(r_i) T[b][m].
// Summed against the contraction weights w_I (v for up, u for down) this is
//   sum_I w_I d_{i mu} D_I / D_ref = g_{i mu} Psi~ + sum_{a,m} A[a][i] Y_{i mu}[m] W[a][m],
//   W[a][m] = sum_I w_I eps_I cof(M_I)[alpha][beta] over (h_alpha, p_beta) = (a, m),
// so the per-determinant derivative vectors are never stored.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "df32.cuh"
#include "mdet_device.cuh"
#include "mdet_internal.h"

namespace mdet {

namespace {


// ---------------------------------------------------------------------------
// K1: orbitals. grid (n_walk, ceil(n_elec / kEC)); smem X[5][kEC][n_ao]; kEC (electrons
// per CTA) is a tuning parameter.
// AO chi = P(x, y, z) f(r^2), P = x^a y^b z^c (degree l), f(s) = sum_p c_p e^{-alpha_p s}:
//   d_x chi = P_x f + 2 x P f',   Lap chi = (Lap P) f + P ((4 l + 6) f' + 4 s f'')
// (Euler: x P_x + y P_y + z P_z = l P). Then Phi[c][e][m] = sum_mu X[c][e][mu] B[mu][m].
template <int kEC>
__global__ void __launch_bounds__(128) k_mo_f64(DevProblem P, double* __restrict__ phi,
                                                const double* __restrict__ R, const int* __restrict__ live) {
  extern __shared__ double smem[];
  const int K = P.n_ao, M = P.n_mo, N = P.n_elec;
  const int64_t w = blockIdx.x;
  if (live && w >= *live) return;
  const int e_begin = blockIdx.y * kEC;
  const int ne = min(kEC, N - e_begin);
  double* X = smem;  // X[(c * kEC + e) * K + mu]
  for (int t = threadIdx.x; t < kEC * P.n_shell; t += blockDim.x) {
    const int e = t / P.n_shell, s = t - e * P.n_shell;
    const int l = P.shell_l[s], ao0 = P.shell_ao0[s], nc = (l + 1) * (l + 2) / 2;
    if (e >= ne) {
      for (int c = 0; c < 5; c++)
        for (int q = 0; q < nc; q++) X[(c * kEC + e) * K + ao0 + q] = 0.0;
      continue;
    }
    const double* r = R + (w * N + e_begin + e) * 3;
    ao_shell_values(P, s, r, [&](int c, int q, double v) { X[(c * kEC + e) * K + ao0 + q] = v; });
  }
  __syncthreads();
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double acc[5 * kEC];
#pragma unroll
    for (int q = 0; q < 5 * kEC; q++) acc[q] = 0.0;
    for (int mu = 0; mu < K; mu++) {
      const double b = __ldg(P.B + (size_t)mu * M + m);
#pragma unroll
      for (int q = 0; q < 5 * kEC; q++) acc[q] = fma(X[q * K + mu], b, acc[q]);
    }
#pragma unroll
    for (int c = 0; c < 5; c++)
#pragma unroll
      for (int e = 0; e < kEC; e++)
        if (e < ne) phi[((w * 5 + c) * N + e_begin + e) * M + m] = acc[c * kEC + e];
  }
}

// ---------------------------------------------------------------------------
// K2+K3: reference inverse and tables. grid n_walk, block 64: warp s factorises
// spin s by Gauss-Jordan elimination with partial pivoting on [S | I] (rows
// stay in their lanes; the pivot order is a permutation whose parity enters
// the sign of the determinant). Then every thread computes T and g.
// MIXED: the orbitals arrive as double-float pairs; the elimination and log|D_ref|
// stay FP64, while A is rounded to double-float pairs (written to Ainv as pairs),
// and T = A Phi and g are formed in double-float on the FP32 pipe (written to Tdf
// and, as pairs, to g); the FP64 table is not written.
template <bool MIXED>
__global__ void __launch_bounds__(64) k_ref(DevProblem P, DevScratch S) {
  __shared__ double aug[2][kMaxSpin][2 * kMaxSpin];
  __shared__ int rowof[2][kMaxSpin];  // pivot row of column a: the row of R that holds row a of A
  __shared__ int bad[2];
  __shared__ uint32_t stf[2];
  const int64_t w = blockIdx.x;
  if (S.live && w >= *S.live) return;
  const int N = P.n_elec, M = P.n_mo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    // Gauss-Jordan elimination on [S | I] with partial pivoting, lanes owning columns: for
    // column j the pivot row p_j is the unused row of largest |S[i][j]|, row p_j is scaled
    // by 1/pivot and column j is eliminated from every other row. Rows stay in place, so
    // at the end the left half is the permutation L[p_j][j] = 1, the right half R = L S^-1,
    // row a of A = S^-1 is row p_a of R, and det S = sgn(j -> p_j) * prod of the pivots.
    // Pivot magnitudes are compared in FP32 from the FP64 bits, and |prod of pivots| is
    // carried as mantissa * 2^exponent with one log at the end, so the FP64 pipe only sees
    // the elimination itself (n FMAs per lane and column step), one reciprocal per pivot
    // and one product per pivot.
    const int sp = warp;
    const int n = sp ? P.n_dn : P.n_up, e0 = sp ? P.n_up : 0;
    const int* occ = P.ref_occ + sp * kMaxSpin;
    for (int c = lane; c < 2 * n; c += 32)
      for (int i = 0; i < n; i++) {
        double v = (c - n == i) ? 1.0 : 0.0;
        if (c < n) {
          const size_t ix = ((w * 5 + 0) * N + e0 + i) * M + occ[c];
          if (MIXED) {
            const float2 f = reinterpret_cast<const float2*>(S.phi)[ix];
            v = df_to_double_int(df32(f.x, f.y));
          } else {
            v = S.phi[ix];
          }
        }
        aug[sp][i][c] = v;
      }
    __syncwarp();
    // |S|_1: the largest column sum (FP32 magnitudes suffice for a conditioning estimate)
    float cs = 0.0f;
    for (int c = lane; c < n; c += 32) {
      float s = 0.0f;
      for (int i = 0; i < n; i++) s += abs_f32_of(aug[sp][i][c]);
      cs = fmaxf(cs, s);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) cs = fmaxf(cs, __shfl_xor_sync(0xffffffffu, cs, off));
    const float normS = cs;
    uint32_t used = 0u;
    double pm = 1.0;  // |prod of pivots| = pm 2^pe, pm in [0.5, 1)
    int pe = 0, negs = 0, singular = 0;
    float pmax = 0.0f, pmin = FLT_MAX;
    for (int j = 0; j < n; j++) {
      int p = -1;
      if (lane == (j & 31)) {
        float best = 0.0f;
        for (int i = 0; i < n; i++) {  // integer and FP32 tests only
          const long long xb = __double_as_longlong(aug[sp][i][j]);
          const float v = abs_f32_of(aug[sp][i][j]);
          if (!((used >> i) & 1u) && (v > best || (p < 0 && (xb << 1) != 0))) {
            best = v;
            p = i;
          }
        }
        if (p >= 0 && ((__double_as_longlong(aug[sp][p][j]) >> 52) & 0x7ff) == 0x7ff) p = -1;  // Inf or NaN
      }
      p = __shfl_sync(0xffffffffu, p, j & 31);
      if (p < 0) {  // no nonzero pivot (or a NaN input): singular reference
        singular = 1;
        break;
      }
      used |= 1u << p;
      if (lane == 0) rowof[sp][j] = p;
      const double piv = aug[sp][p][j];
      {
        const long long b = __double_as_longlong(piv);
        negs += (int)((unsigned long long)b >> 63);
        const int ex = (int)((b >> 52) & 0x7ff);
        // |piv| = m 2^(ex - 1022), m in [0.5, 1) (normal pivots; a subnormal one counts as tiny)
        const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
        pm *= m;
        pe += ex - 1022;
        const long long bm = __double_as_longlong(pm);  // back into [0.5, 1)
        pe += (int)((bm >> 52) & 0x7ff) - 1022;
        pm = __longlong_as_double((bm & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
        const float a = abs_f32_of(piv);
        pmax = fmaxf(pmax, a);
        pmin = fminf(pmin, a);
      }
      const double inv = 1.0 / piv;
      __syncwarp();
      for (int c = lane; c < 2 * n; c += 32) {
        if (c == j) continue;
        const double apc = aug[sp][p][c] * inv;
        aug[sp][p][c] = apc;
        for (int i = 0; i < n; i++)
          if (i != p) aug[sp][i][c] = fma(-aug[sp][i][j], apc, aug[sp][i][c]);
      }
      __syncwarp();
      if (lane == (j & 31))
        for (int i = 0; i < n; i++) aug[sp][i][j] = (i == p) ? 1.0 : 0.0;
      __syncwarp();
    }
    // sign: pivots' signs times the parity of j -> p_j (inversions counted by lane j)
    int inv_cnt = 0;
    if (!singular)
      for (int j = lane; j < n; j += 32)
        for (int k = j + 1; k < n; k++) inv_cnt += rowof[sp][k] < rowof[sp][j];
#pragma unroll
    for (int off = 16; off; off >>= 1) inv_cnt += __shfl_xor_sync(0xffffffffu, inv_cnt, off);
    const double sgn = ((negs + inv_cnt) & 1) ? -1.0 : 1.0;
    // |A|_1: column sums of R (a row permutation of A)
    float ca = 0.0f;
    if (!singular)
      for (int c = lane; c < n; c += 32) {
        float s = 0.0f;
        for (int i = 0; i < n; i++) s += abs_f32_of(aug[sp][i][n + c]);
        ca = fmaxf(ca, s);
      }
#pragma unroll
    for (int off = 16; off; off >>= 1) ca = fmaxf(ca, __shfl_xor_sync(0xffffffffu, ca, off));
    const double kappa1 = (double)normS * (double)ca;
    if (lane == 0) {
      bad[sp] = singular;
      S.ld0[w * 2 + sp] = singular ? -INFINITY : log(pm) + pe * 0.69314718055994530942;
      S.sg0[w * 2 + sp] = singular ? 0.0 : sgn;
      uint32_t st = singular ? MDET_WS_REF_SINGULAR : 0u;
      if (!singular && pmin < 1e-13f * pmax) st |= MDET_WS_REF_ILLCOND;
      S.kap[w * 2 + sp] = singular ? INFINITY : kappa1;
      if (P.fallback_tol > 0.0 && P.n_up <= MDET_FALLBACK_MAX_SPIN && singular) st |= MDET_WS_FALLBACK;
      stf[sp] = st;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S.wstat[w] = stf[0] | stf[1];
    // the contraction accumulates Psi~ and, except for an escalated re-evaluation (live count
    // set: it keeps the magnitude sum of the evaluation that flagged it), sum |c r r|
    S.psit[w] = 0.0;
    if (!S.live) S.psia[w] = 0.0f;
  }
  const int nu = P.n_up, nd = P.n_dn;
  if (MIXED) {
    // each row of A (the right half of its lane's row) as double-float pairs in the left half,
    // which the elimination no longer needs
    const int t = threadIdx.x, sp = t >> 5, lane = t & 31;
    const int n = sp ? nd : nu;
    if (lane < n && !bad[sp]) {
      float2* dst = reinterpret_cast<float2*>(&aug[sp][lane][0]);
      for (int i = 0; i < n; i++) {
        const df32 d = df_from_bits(__double_as_longlong(aug[sp][lane][n + i]));
        dst[i] = make_float2(d.hi, d.lo);
      }
    }
    __syncthreads();
    auto Adf = [&](int sp, int a, int i) {
      const float2 v = reinterpret_cast<const float2*>(&aug[sp][rowof[sp][a]][0])[i];
      return df32(v.x, v.y);
    };
    const float2* phi2 = reinterpret_cast<const float2*>(S.phi);
    float2* Ag2 = reinterpret_cast<float2*>(S.Ainv) + w * (nu * nu + nd * nd);
    const float2 fnan = make_float2(__int_as_float(0x7fc00000), 0.0f);
    for (int t2 = threadIdx.x; t2 < nu * nu + nd * nd; t2 += blockDim.x) {
      const int sp2 = t2 < nu * nu ? 0 : 1;
      const int n2 = sp2 ? nd : nu;
      const int tt = sp2 ? t2 - nu * nu : t2;
      const df32 v = bad[sp2] ? df32(0.0f, 0.0f) : Adf(sp2, tt / n2, tt % n2);
      Ag2[t2] = bad[sp2] ? fnan : make_float2(v.hi, v.lo);
    }
    for (int t2 = threadIdx.x; t2 < N * M; t2 += blockDim.x) {
      const int row = t2 / M, m = t2 - row * M;
      const int sp2 = row < nu ? 0 : 1;
      const int n2 = sp2 ? nd : nu, e0 = sp2 ? nu : 0, a = row - e0;
      df32 acc(0.0f, 0.0f);
      if (!bad[sp2])
        for (int i = 0; i < n2; i++) {
          const float2 pv = phi2[((w * 5 + 0) * N + e0 + i) * M + m];
          acc = acc + Adf(sp2, a, i) * df32(pv.x, pv.y);
        }
      S.Tdf[(size_t)t2 * S.wp + w] = bad[sp2] ? fnan : make_float2(acc.hi, acc.lo);
    }
    float2* g2 = reinterpret_cast<float2*>(S.g);
    for (int t2 = threadIdx.x; t2 < N * 4; t2 += blockDim.x) {
      const int e = t2 >> 2, mu = t2 & 3;
      const int sp2 = e < nu ? 0 : 1;
      const int n2 = sp2 ? nd : nu, e0 = sp2 ? nu : 0, i = e - e0;
      const int* occ = P.ref_occ + sp2 * kMaxSpin;
      df32 acc(0.0f, 0.0f);
      if (!bad[sp2])
        for (int a = 0; a < n2; a++) {
          const float2 pv = phi2[((w * 5 + 1 + mu) * N + e) * M + occ[a]];
          acc = acc + Adf(sp2, a, i) * df32(pv.x, pv.y);
        }
      g2[(w * N + e) * 4 + mu] = bad[sp2] ? fnan : make_float2(acc.hi, acc.lo);
    }
    return;
  }
  // A to global, T = A Phi (walker-minor), g
  // A[a][i] of spin sp
  auto Aat = [&](int sp, int a, int i) { return aug[sp][rowof[sp][a]][(sp ? nd : nu) + i]; };
  double* Ag = S.Ainv + w * (nu * nu + nd * nd);
  for (int t = threadIdx.x; t < nu * nu + nd * nd; t += blockDim.x) {
    const int sp = t < nu * nu ? 0 : 1;
    const int n = sp ? nd : nu;
    const int tt = sp ? t - nu * nu : t;
    Ag[t] = bad[sp] ? NAN : Aat(sp, tt / n, tt % n);
  }
  for (int t = threadIdx.x; t < N * M; t += blockDim.x) {
    const int row = t / M, m = t - row * M;  // row indexes the table rows of both spins
    const int sp = row < nu ? 0 : 1;
    const int n = sp ? nd : nu, e0 = sp ? nu : 0, a = row - e0;
    double acc = 0.0;
    if (!bad[sp])
      for (int i = 0; i < n; i++) acc = fma(Aat(sp, a, i), S.phi[((w * 5 + 0) * N + e0 + i) * M + m], acc);
    if (bad[sp]) acc = NAN;
    S.T[(size_t)t * S.wp + w] = acc;
  }
  for (int t = threadIdx.x; t < N * 4; t += blockDim.x) {
    const int e = t >> 2, mu = t & 3;
    const int sp = e < nu ? 0 : 1;
    const int n = sp ? nd : nu, e0 = sp ? nu : 0, i = e - e0;
    const int* occ = P.ref_occ + sp * kMaxSpin;
    double acc = 0.0;
    if (!bad[sp])
      for (int a = 0; a < n; a++) acc = fma(Aat(sp, a, i), S.phi[((w * 5 + 1 + mu) * N + e) * M + occ[a]], acc);
    S.g[(w * N + e) * 4 + mu] = bad[sp] ? NAN : acc;
  }
}

// ---------------------------------------------------------------------------
// K4: ratios r_I = eps_I det M_I. grid (ceil(n_det_total / 32), wpad / 32),
// block 128 = 4 warps; lanes are walkers, each warp takes 8 determinants.
__global__ void __launch_bounds__(128) k_ratio_f64(DevProblem P, DevScratch S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (S.live && (int64_t)blockIdx.y * 32 >= *S.live) return;
  const int64_t w = (int64_t)blockIdx.y * 32 + lane;
  const int nu_det = P.n_det_sp[0], ntot = nu_det + P.n_det_sp[1];
  const int M = P.n_mo;
  const int64_t wp = S.wp;
  for (int q = 0; q < 8; q++) {
    const int t = blockIdx.x * 32 + warp * 8 + q;
    if (t >= ntot) return;
    const int sp = t < nu_det ? 0 : 1;
    const Exc e = P.exc[sp][sp ? t - nu_det : t];
    const double* T = S.T + (size_t)(sp ? P.n_up * M : 0) * wp;
    double m[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++)
        m[a][b] = (a < e.k && b < e.k) ? T[((size_t)e.h[a] * M + e.p[b]) * wp + w] : 0.0;
    const double d = small_det(e.k, m);
    // the sign by its bit, not by an FP64 instruction
    S.r[(size_t)t * wp + w] = __longlong_as_double(__double_as_longlong(d) ^ ((long long)(e.eps < 0) << 63));
    if (P.split[t]) S.vu[w * ntot + t] = 0.0;  // the contraction adds the pieces of a cut segment
  }
}

// ---------------------------------------------------------------------------
// K5: y[seg][w] += sum_k val_k x[gidx_k][w] over one ordering of C. Each warp
// owns `chunk` consecutive nonzeros and 4 walkers per lane (128 per warp);
// partial sums are flushed with atomics whenever the segment changes. If rdot
// is given, psit[w] += rdot[seg][w] * (partial sum) as well (Psi~ = r_up . v).
__global__ void __launch_bounds__(256) k_spmm_f64(const int* __restrict__ seg, const int* __restrict__ gidx,
                                                  const double* __restrict__ val, int64_t nnz, int chunk,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  int64_t wp, const double* __restrict__ rdot,
                                                  double* __restrict__ psit) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t k0 = gw * chunk;
  if (k0 >= nnz) return;
  const int64_t k1 = min(k0 + (int64_t)chunk, nnz);
  const int64_t wb = (int64_t)blockIdx.y * 128 + lane * 4;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int cur = __ldg(seg + k0);
  auto flush = [&](int s) {
    double* yp = y + (size_t)s * wp + wb;
    atomicAdd(yp + 0, a0);
    atomicAdd(yp + 1, a1);
    atomicAdd(yp + 2, a2);
    atomicAdd(yp + 3, a3);
    if (rdot) {
      const double* rp = rdot + (size_t)s * wp + wb;
      atomicAdd(psit + wb + 0, rp[0] * a0);
      atomicAdd(psit + wb + 1, rp[1] * a1);
      atomicAdd(psit + wb + 2, rp[2] * a2);
      atomicAdd(psit + wb + 3, rp[3] * a3);
    }
  };
  for (int64_t k = k0; k < k1; k++) {
    const int s = __ldg(seg + k);
    if (s != cur) {
      flush(cur);
      cur = s;
      a0 = a1 = a2 = a3 = 0;
    }
    const double c = __ldg(val + k);
    const double2* xp = reinterpret_cast<const double2*>(x + (size_t)__ldg(gidx + k) * wp + wb);
    const double2 u = __ldg(xp), v = __ldg(xp + 1);
    a0 = fma(c, u.x, a0);
    a1 = fma(c, u.y, a1);
    a2 = fma(c, v.x, a2);
    a3 = fma(c, v.y, a3);
  }
  flush(cur);
}


// ---------------------------------------------------------------------------
// K5 (form used by mdet_evaluate): y[seg][w] = sum over segment seg of val_k x[gidx_k][w]
// (v = C r_dn over the rows of the row-major copy of C, u = C^T r_up over the columns of
// the column-major one, Sec. 2.4), x walker-minor with leading dimension wp, y walker-major
// (y[w * ldy + seg_off + seg], the layout the epilogue reads contiguously). A work
// item (`items`, built on the host) is a run of whole segments holding at most `spmm_chunk`
// nonzeros, or one piece of at most that many of a longer segment, for one group of 32 WPL
// walkers, WPL per lane; the nonzero's value and index are uniform across the warp. The sums
// of a whole segment come from exactly one warp and are stored (no clearing, no atomics;
// an item's consecutive segments fill whole sectors of each walker's row); the pieces of a
// cut segment add theirs atomically into entries the ratio kernel cleared. Items run fastest
// within a walker group, so the warps in flight share that group's columns of x in L2.
// QUEUE false: one work item per warp of a full grid. QUEUE true: a persistent grid whose
// warps take the next work item from the counter *queue (zeroed before the launch), so
// blocks that become resident late, while kernels of other streams hold part of the SMs,
// simply take fewer items.
// With rdot: psit[w] += rdot[seg][w] y[seg][w] per segment (Psi~ = r_up . v; atomics on the
// small, L2-resident psit, which keep the registers of a grid that shares every SM with the
// other stages low). ABS: psia[w] += |rdot[seg][w]| sum |c| |x| in FP32 likewise, so that
// psia = sum_ij |c_ij| |r_up,i| |r_dn,j|, the magnitude sum behind Psi~
// (its ratio to |Psi~| is the conditioning of the CI sum, used by the error estimate).
// WPL walkers per lane (8, or 4 for the few walkers of an escalated re-evaluation, where a
// 256-walker group would be mostly padding); walker groups at or beyond the live count are skipped.
// stamp (optional, zeroed before the launch): stamp[0] = ~(global timer at the earliest block
// start), stamp[1] = global timer at the latest warp exit, in ns: the launch's duration on the
// device without events in the stream.
static __device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <bool QUEUE, bool ABS, int WPL>
__global__ void __launch_bounds__(128) k_spmm_seg(const int* __restrict__ seg, const int* __restrict__ gidx,
                                                  const double* __restrict__ val, const int2* __restrict__ items,
                                                  int n_items, int64_t n_groups, const double* __restrict__ x,
                                                  int64_t wp, double* __restrict__ y, int64_t ldy, int seg_off,
                                                  const double* __restrict__ rdot, double* __restrict__ psit,
                                                  float* __restrict__ psia, unsigned long long* __restrict__ queue,
                                                  const int* __restrict__ live, unsigned long long* __restrict__ stamp) {
  constexpr int G = 32 * WPL;
  const int lane = threadIdx.x & 31;
  if (stamp && threadIdx.x == 0) atomicMax(stamp, ~global_timer_ns());
  const int64_t ng = live ? min(n_groups, (int64_t)(*live + G - 1) / G) : n_groups;
  const int64_t n_work = (int64_t)n_items * ng;
  auto next_item = [&]() -> int64_t {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(queue, 1ULL);
    return (int64_t)__shfl_sync(0xffffffffu, t, 0);
  };
  const int64_t first = QUEUE ? next_item() : (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t q = first; q < n_work; q = QUEUE ? next_item() : n_work) {
    const int it = (int)(q % n_items);
    const int64_t grp = q / n_items;
    const int2 r0 = __ldg(items + it);
    const int2 r = make_int2(r0.x, r0.y & 0x7fffffff);
    const bool piece = r0.y < 0;  // one piece of a longer segment: its sums are added, not stored
    const int64_t wb = grp * G + lane * WPL;
    double a[WPL];
    float aa[WPL];  // ABS: sum |c| |x| of the segment
#pragma unroll
    for (int j = 0; j < WPL; j++) {
      a[j] = 0.0;
      aa[j] = 0.0f;
    }
    int cur = __ldg(seg + r.x);
    auto flush = [&](int sg) {
      double* yr = y + wb * ldy + seg_off + sg;
      if (piece) {
#pragma unroll
        for (int j = 0; j < WPL; j++) atomicAdd(yr + j * ldy, a[j]);
      } else {
#pragma unroll
        for (int j = 0; j < WPL; j++) yr[j * ldy] = a[j];
      }
      if (rdot) {
        const double2* rp = reinterpret_cast<const double2*>(rdot + (size_t)sg * wp + wb);
#pragma unroll
        for (int h = 0; h < WPL / 2; h++) {
          const double2 t = __ldg(rp + h);
          atomicAdd(psit + wb + 2 * h, t.x * a[2 * h]);
          atomicAdd(psit + wb + 2 * h + 1, t.y * a[2 * h + 1]);
          if (ABS) {
            atomicAdd(psia + wb + 2 * h, abs_f32_of(t.x) * aa[2 * h]);
            atomicAdd(psia + wb + 2 * h + 1, abs_f32_of(t.y) * aa[2 * h + 1]);
          }
        }
      }
    };
    for (int k = r.x; k < r.y; k++) {
      const int sg = __ldg(seg + k);
      if (sg != cur) {
        flush(cur);
        cur = sg;
#pragma unroll
        for (int j = 0; j < WPL; j++) {
          a[j] = 0.0;
          aa[j] = 0.0f;
        }
      }
      const double c = __ldg(val + k);
      const double2* xp = reinterpret_cast<const double2*>(x + (size_t)__ldg(gidx + k) * wp + wb);
      double xv[WPL];
#pragma unroll
      for (int h = 0; h < WPL / 2; h++) {
        const double2 t = __ldg(xp + h);
        xv[2 * h] = t.x;
        xv[2 * h + 1] = t.y;
      }
#pragma unroll
      for (int j = 0; j < WPL; j++) a[j] = fma(c, xv[j], a[j]);
      if (ABS) {
        const float ca = abs_f32_of(c);
#pragma unroll
        for (int j = 0; j < WPL; j++) aa[j] = fmaf(ca, abs_f32_of(xv[j]), aa[j]);
      }
    }
    flush(cur);
  }
  if (stamp && lane == 0) atomicMax(stamp + 1, global_timer_ns());
}

// The same segmented product with the ratios and C as double-float pairs on
// the FP32 pipe (an option of the mixed path; the default contraction is the
// FP64 kernel above): per walker the compensated dot product of Ogita, Rump and
// Oishi (TwoProd of the leading words, TwoSum into the running sum, cross terms
// and all rounding errors into a second word), about 13 FP32 instructions per
// nonzero instead of one FP64 FMA at 1/54 of the FP32 rate. Segment sums are
// converted to FP64 when stored; work items, layouts and the Psi~ sums as above
// (8 walkers per lane, full grid).
__global__ void __launch_bounds__(128) k_spmm_df(const int* __restrict__ seg, const int* __restrict__ gidx,
                                                 const float2* __restrict__ val, const int2* __restrict__ items,
                                                 int n_items, int64_t n_groups, const float2* __restrict__ x,
                                                 int64_t wp, double* __restrict__ y, int64_t ldy, int seg_off,
                                                 const double* __restrict__ rdot, double* __restrict__ psit,
                                                 float* __restrict__ psia) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < (int64_t)n_items * n_groups;
       q += nwarps) {
    const int it = (int)(q % n_items);
    const int64_t grp = q / n_items;
    const int2 r0 = __ldg(items + it);
    const int2 r = make_int2(r0.x, r0.y & 0x7fffffff);
    const bool piece = r0.y < 0;
    const int64_t wb = grp * 256 + lane * 8;
    float s[8], e[8], aa[8];
#pragma unroll
    for (int j = 0; j < 8; j++) s[j] = e[j] = aa[j] = 0.0f;
    int cur = __ldg(seg + r.x);
    auto flush = [&](int sg) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; j++) v[j] = (double)s[j] + (double)e[j];
      double* yr = y + wb * ldy + seg_off + sg;
      if (piece) {
#pragma unroll
        for (int j = 0; j < 8; j++) atomicAdd(yr + j * ldy, v[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 8; j++) yr[j * ldy] = v[j];
      }
      if (rdot) {
        const double* rp = rdot + (size_t)sg * wp + wb;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          atomicAdd(psit + wb + j, rp[j] * v[j]);
          atomicAdd(psia + wb + j, abs_f32_of(rp[j]) * aa[j]);
        }
      }
    };
    for (int k = r.x; k < r.y; k++) {
      const int sg = __ldg(seg + k);
      if (sg != cur) {
        flush(cur);
        cur = sg;
#pragma unroll
        for (int j = 0; j < 8; j++) s[j] = e[j] = aa[j] = 0.0f;
      }
      const float2 c = __ldg(val + k);
      const float4* xp = reinterpret_cast<const float4*>(x + (size_t)__ldg(gidx + k) * wp + wb);
      float xs[16];
#pragma unroll
      for (int q4 = 0; q4 < 4; q4++) {
        const float4 v = __ldg(xp + q4);
        xs[4 * q4] = v.x;
        xs[4 * q4 + 1] = v.y;
        xs[4 * q4 + 2] = v.z;
        xs[4 * q4 + 3] = v.w;
      }
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const float xh = xs[2 * j], xl = xs[2 * j + 1];
        const float p = __fmul_rn(c.x, xh);
        const float pe = __fmaf_rn(c.x, xh, -p);
        const float cross = __fmaf_rn(c.x, xl, __fmul_rn(c.y, xh));
        float t, err;
        two_sum(s[j], p, t, err);
        s[j] = t;
        e[j] = __fadd_rn(e[j], __fadd_rn(err, __fadd_rn(pe, cross)));
        if (rdot) aa[j] = fmaf(fabsf(c.x), fabsf(xh), aa[j]);
      }
    }
    flush(cur);
  }
}

// Cofactors of one determinant of degree K (compile time) in double-float,
// weighted by w (the FP64 bits of eps_I w_I), added into W: each addition is an
// FP32 shared atomic on the high word whose returned old value gives, by
// TwoSum, the rounding error of that addition, which goes with the low word
// into a second atomic.
template <int K>
__device__ __forceinline__ void scatter_cof_df(const Exc& e, long long wb, const float2* __restrict__ Tdf, int toff,
                                               int Mt, int off, int M, float* Whi, float* Wlo) {
  df32 m[4][4], cof[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const float2 v = (a < K && b < K) ? Tdf[toff + e.h[a] * Mt + e.p[b]] : make_float2(0.f, 0.f);
      m[a][b] = df32(v.x, v.y);
    }
  small_cof_dot<K>(m, cof);
  const df32 wd = df_from_bits(wb);
#pragma unroll
  for (int a = 0; a < K; a++)
#pragma unroll
    for (int b = 0; b < K; b++) {
      const df32 x = cof[a][b] * wd;
      const int slot = off + e.h[a] * M + e.p[b];
      const float old = atomicAdd(Whi + slot, x.hi);
      float s_, err;
      two_sum(old, x.hi, s_, err);
      atomicAdd(Wlo + slot, __fadd_rn(err, x.lo));
    }
}

// ---------------------------------------------------------------------------
// K6: per walker: W scatter over every determinant, Q = A^T W, Pm = T Q^T,
// G_{i mu} = g Psi~ + sum_m d_mu phi[i][m] Q[i][m] - sum_b d_mu phi[i][o_b] Pm[b][i],
// then grad, Laplacian, log|Psi|, sign and E_L. grid n_walk, block 128.
// FP64 variant: cofactors in FP64, W accumulated in three FP32 words with compensated shared
// atomics (acc3_add: more accurate than FP64 accumulation, and off the FP64 pipe, which FP64
// shared-memory atomics occupy), summed into FP64 before Q.
// MIXED variant: cofactors in double-float on the FP32 pipe; W accumulated as
// a compensated pair of FP32 shared atomics: the atomic returns the old value,
// so TwoSum(old, x) recovers the rounding error of the addition it performed,
// which goes into the low word. Q, Pm and G are double-float too (orbitals,
// A and g arrive as pairs), so the FP64 pipe is left to the contraction; the
// sums G are converted to FP64 with integer instructions.
// smem, FP64: T[N][M], W[3][N][M] (FP32), Q[N][M], A blocks, Pm.
// smem, MIXED: W[N][M] as hi/lo FP32 arrays, Q[N][M], A blocks, Pm (all pairs),
//       Tdf[N][M].
template <bool MIXED, int NT>
__global__ void __launch_bounds__(NT, MIXED ? 5 : 1) k_final(DevProblem P, DevScratch S, const double* __restrict__ R,
                                               double* __restrict__ log_abs_psi, int8_t* __restrict__ sign,
                                               double* __restrict__ grad, double* __restrict__ lap,
                                               double* __restrict__ e_local, uint32_t* __restrict__ status) {
  extern __shared__ double sm[];
  const int nu = P.n_up, nd = P.n_dn, N = nu + nd, M = P.n_mo;
  const int NM = N * M;
  const int64_t w = blockIdx.x, wp = S.wp;
  if (S.live && w >= *S.live) return;
  // MIXED keeps T and Q as pairs with rows padded to Mt = M + 1 entries, so that
  // threads reading the same column of different rows hit different banks
  const int Mt = MIXED ? M + 1 : M;
  double* Ts = MIXED ? nullptr : sm;    // [N][M] (FP64 only)
  double* Ws = MIXED ? sm : sm + NM;    // [N][M] (MIXED: hi words, then lo words; FP64: three FP32 words)
  double* Qs = Ws + (MIXED ? NM : (3 * NM + 1) / 2);  // [N][Mt]
  double* As = Qs + N * Mt;             // [nu*nu + nd*nd]
  double* Pm = As + nu * nu + nd * nd;  // [nu*nu + nd*nd]  Pm[b][i] per spin
  float2* Tdf = reinterpret_cast<float2*>(Pm + nu * nu + nd * nd);  // [N][Mt] (MIXED)
  float* Whi = reinterpret_cast<float*>(Ws);                          // MIXED: [N][M] hi words
  float* Wlo = Whi + NM;                                              //        [N][M] lo words
  float* W3 = Wlo + NM;  // FP64: the third word of W (the first two are Whi, Wlo)
  constexpr int NW = NT / 32;  // warps per block
  __shared__ double red[NW];
  __shared__ double Gs[kMaxSpin * 2][4];
  __shared__ float Ga[kMaxSpin * 2][4];
  __shared__ float G2[kMaxSpin * 2][4];
  __shared__ float rmsG[4], estw[2][4];
  for (int t = threadIdx.x; t < NM; t += blockDim.x) {
    if (MIXED) {
      Tdf[(t / M) * Mt + t % M] = S.Tdf[(size_t)t * wp + w];
      Whi[t] = 0.0f;
      Wlo[t] = 0.0f;
    } else {
      Ts[t] = S.T[(size_t)t * wp + w];
      Whi[t] = 0.0f;
      Wlo[t] = 0.0f;
      W3[t] = 0.0f;
    }
  }
  for (int t = threadIdx.x; t < nu * nu + nd * nd; t += blockDim.x) {
    if (MIXED)
      reinterpret_cast<float2*>(As)[t] = reinterpret_cast<const float2*>(S.Ainv)[w * (nu * nu + nd * nd) + t];
    else
      As[t] = S.Ainv[w * (nu * nu + nd * nd) + t];
  }
  __syncthreads();
  const int nu_det = P.n_det_sp[0], ntot = nu_det + P.n_det_sp[1];
  const int tid = threadIdx.x, nth = blockDim.x;
  if constexpr (MIXED) {
    // The determinants of one spin and excitation degree k at a time (the context orders
    // each spin's list by degree), so every lane of a warp runs the same k x k cofactor
    // code; within the group, determinant (q * stride) mod L for q = thread, thread + NT,
    // ... with a prime stride that does not divide L (a permutation), so the lanes of a
    // warp hold determinants far apart in key order, which rarely share a (hole,
    // particle) slot of W, and every thread gets an even share of the group.
    for (int grp = 0; grp < 2 * kMaxExc; grp++) {
      const int sp = grp / kMaxExc, k = grp % kMaxExc + 1;
      const int base = sp ? nu_det : 0;
      const int s0 = P.deg_start[sp][k], L = P.deg_start[sp][k + 1] - s0;
      if (L <= 0) continue;
      const int stride = (L % 7919) ? 7919 : ((L % 7927) ? 7927 : 7933);
      const int step = (int)(((int64_t)nth * stride) % L);
      int tq = (int)(((int64_t)tid * stride) % L);
      const int off = sp ? nu * M : 0;    // W
      const int toff = sp ? nu * Mt : 0;  // the padded pairs of T
      for (int j = tid; j < L; j += nth) {
        const int t = s0 + tq;
        tq += step;
        if (tq >= L) tq -= L;
        const Exc e = P.exc[sp][t];
        // the weight eps_I w_I: sign and zero test on the bits (no FP64 instructions)
        long long wb = __double_as_longlong(S.vu[w * ntot + base + t]);
        if ((wb & 0x7fffffffffffffffLL) == 0) continue;
        if (e.eps < 0) wb ^= (long long)(1ULL << 63);
        switch (k) {
          case 1: scatter_cof_df<1>(e, wb, Tdf, toff, Mt, off, M, Whi, Wlo); break;
          case 2: scatter_cof_df<2>(e, wb, Tdf, toff, Mt, off, M, Whi, Wlo); break;
          case 3: scatter_cof_df<3>(e, wb, Tdf, toff, Mt, off, M, Whi, Wlo); break;
          default: scatter_cof_df<4>(e, wb, Tdf, toff, Mt, off, M, Whi, Wlo); break;
        }
      }
    }
  } else {
    // each thread walks its own contiguous block (sequential loads of records and weights;
    // the FP64 pipe, not the balance, bounds this variant)
    const int per = (ntot + nth - 1) / nth;
    const int n_mine = max(0, min(per, ntot - tid * per));
    for (int j = 0; j < n_mine; j++) {
      const int t = tid * per + j;
      const int sp = t < nu_det ? 0 : 1;
      const Exc e = P.exc[sp][sp ? t - nu_det : t];
      if (e.k == 0) continue;
      long long wb = __double_as_longlong(S.vu[w * ntot + t]);
      if ((wb & 0x7fffffffffffffffLL) == 0) continue;
      if (e.eps < 0) wb ^= (long long)(1ULL << 63);
      const double wgt = __longlong_as_double(wb);
      const int off = sp ? nu * M : 0;
      double m[4][4], cof[4][4];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) m[a][b] = (a < e.k && b < e.k) ? Ts[off + e.h[a] * M + e.p[b]] : 0.0;
      small_cof(e.k, m, cof);
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
          if (a < e.k && b < e.k) {
            const int slot = off + e.h[a] * M + e.p[b];
            acc3_add(Whi + slot, Wlo + slot, W3 + slot, wgt * cof[a][b]);
          }
    }
  }
  __syncthreads();
  const double psit = S.psit[w];
  const double ld = S.ld0[w * 2] + S.ld0[w * 2 + 1];
  const double sg = S.sg0[w * 2] * S.sg0[w * 2 + 1];
  if constexpr (MIXED) {
    // W normalised into (hi, lo) pairs in place
    for (int t = threadIdx.x; t < NM; t += blockDim.x) {
      float hi, lo;
      two_sum(Whi[t], Wlo[t], hi, lo);
      Whi[t] = hi;
      Wlo[t] = lo;
    }
    __syncthreads();
    const float2* A2 = reinterpret_cast<const float2*>(As);
    float2* Q2 = reinterpret_cast<float2*>(Qs);
    float2* P2 = reinterpret_cast<float2*>(Pm);
    // Q[i][m] = sum_a A[a][i] W[a][m] (per spin block)
    for (int t = threadIdx.x; t < NM; t += blockDim.x) {
      const int row = t / M, m = t - row * M;
      const int sp = row < nu ? 0 : 1;
      const int n = sp ? nd : nu, e0 = sp ? nu : 0, i = row - e0;
      const float2* A = A2 + (sp ? nu * nu : 0);
      df32 acc(0.0f, 0.0f);
      for (int a = 0; a < n; a++) {
        const float2 av = A[a * n + i];
        const int wi = (e0 + a) * M + m;
        acc = acc + df32(av.x, av.y) * df32(Whi[wi], Wlo[wi]);
      }
      Q2[row * Mt + m] = make_float2(acc.hi, acc.lo);
    }
    __syncthreads();
    // Pm[b][i] = sum_m T[b][m] Q[i][m]
    for (int t = threadIdx.x; t < nu * nu + nd * nd; t += blockDim.x) {
      const int sp = t < nu * nu ? 0 : 1;
      const int n = sp ? nd : nu, e0 = sp ? nu : 0;
      const int tt = sp ? t - nu * nu : t;
      const int b = tt / n, i = tt - b * n;
      const float2* Tr = Tdf + (e0 + b) * Mt;
      const float2* Qr = Q2 + (e0 + i) * Mt;
      df32 acc(0.0f, 0.0f);
      for (int m = 0; m < M; m++) acc = acc + df32(Tr[m].x, Tr[m].y) * df32(Qr[m].x, Qr[m].y);
      P2[t] = make_float2(acc.hi, acc.lo);
    }
    __syncthreads();
    const df32 psit_df = df_from_bits(__double_as_longlong(psit));
    const float2* phi2 = reinterpret_cast<const float2*>(S.phi);
    const float2* g2 = reinterpret_cast<const float2*>(S.g);
    for (int t = threadIdx.x; t < N * 4; t += blockDim.x) {
      const int e = t >> 2, mu = t & 3;
      const int sp = e < nu ? 0 : 1;
      const int n = sp ? nd : nu, e0 = sp ? nu : 0, i = e - e0;
      const int* occ = P.ref_occ + sp * kMaxSpin;
      const float2* dphi = phi2 + ((w * 5 + 1 + mu) * N + e) * M;
      const float2* Qr = Q2 + e * Mt;
      const float2 gv = g2[(w * N + e) * 4 + mu];
      df32 acc = df32(gv.x, gv.y) * psit_df;
      // magnitudes of the terms, for the error estimate (FP32 is plenty for an estimate)
      float aab = fabsf(acc.hi), aa2 = aab * aab;
      for (int m = 0; m < M; m++) {
        const float2 dv = dphi[m];
        acc = acc + df32(dv.x, dv.y) * df32(Qr[m].x, Qr[m].y);
        const float tm = fabsf(dv.x * Qr[m].x);
        aab += tm;
        aa2 = fmaf(tm, tm, aa2);
      }
      const float2* Pb = P2 + (sp ? nu * nu : 0);
      for (int b = 0; b < n; b++) {
        const float2 dv = dphi[occ[b]], pv = Pb[b * n + i];
        acc = acc - df32(dv.x, dv.y) * df32(pv.x, pv.y);
        const float tm = fabsf(dv.x * pv.x);
        aab += tm;
        aa2 = fmaf(tm, tm, aa2);
      }
      Gs[e][mu] = df_to_double_int(acc);
      Ga[e][mu] = aab;
      G2[e][mu] = sqrtf(aa2);
    }
  } else {
    // W's three words summed into FP64, through Q's space (free until Q is formed), then back
    // over the words
    for (int t = threadIdx.x; t < NM; t += blockDim.x) Qs[t] = ((double)Whi[t] + (double)Wlo[t]) + (double)W3[t];
    __syncthreads();
    double* Wd = Ws;
    for (int t = threadIdx.x; t < NM; t += blockDim.x) Wd[t] = Qs[t];
    __syncthreads();
    // Q[i][m] = sum_a A[a][i] W[a][m] (per spin block)
    for (int t = threadIdx.x; t < NM; t += blockDim.x) {
      const int row = t / M, m = t - row * M;
      const int sp = row < nu ? 0 : 1;
      const int n = sp ? nd : nu, e0 = sp ? nu : 0, i = row - e0;
      const double* A = As + (sp ? nu * nu : 0);
      const double* Wb = Wd + e0 * M;
      double acc = 0.0;
      for (int a = 0; a < n; a++) acc = fma(A[a * n + i], Wb[a * M + m], acc);
      Qs[t] = acc;
    }
    __syncthreads();
    // Pm[b][i] = sum_m T[b][m] Q[i][m]
    for (int t = threadIdx.x; t < nu * nu + nd * nd; t += blockDim.x) {
      const int sp = t < nu * nu ? 0 : 1;
      const int n = sp ? nd : nu, e0 = sp ? nu : 0;
      const int tt = sp ? t - nu * nu : t;
      const int b = tt / n, i = tt - b * n;
      const double* Tr = Ts + (e0 + b) * M;
      const double* Qr = Qs + (e0 + i) * M;
      double acc = 0.0;
      for (int m = 0; m < M; m++) acc = fma(Tr[m], Qr[m], acc);
      Pm[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N * 4; t += blockDim.x) {
      const int e = t >> 2, mu = t & 3;
      const int sp = e < nu ? 0 : 1;
      const int n = sp ? nd : nu, e0 = sp ? nu : 0, i = e - e0;
      const int* occ = P.ref_occ + sp * kMaxSpin;
      const double* dphi = S.phi + ((w * 5 + 1 + mu) * N + e) * M;
      const double* Qr = Qs + e * M;
      double acc = S.g[(w * N + e) * 4 + mu] * psit;
      // magnitudes of the terms, for the error estimate (FP32 is plenty for an estimate)
      float aab = fabsf((float)acc), aa2 = aab * aab;
      for (int m = 0; m < M; m++) {
        acc = fma(dphi[m], Qr[m], acc);
        const float tm = fabsf((float)dphi[m] * (float)Qr[m]);
        aab += tm;
        aa2 = fmaf(tm, tm, aa2);
      }
      const double* Pb = Pm + (sp ? nu * nu : 0);
      for (int b = 0; b < n; b++) {
        acc = fma(-dphi[occ[b]], Pb[b * n + i], acc);
        const float tm = fabsf((float)dphi[occ[b]] * (float)Pb[b * n + i]);
        aab += tm;
        aa2 = fmaf(tm, tm, aa2);
      }
      Gs[e][mu] = acc;
      Ga[e][mu] = aab;
      G2[e][mu] = sqrtf(aa2);
    }
  }
  __syncthreads();
  // potential energy: the electron-electron, electron-nucleus and nucleus-nucleus pairs
  // as one list spread evenly over the block's threads, so that no lane idles on a
  // skipped pair; electron pairs in circulant order, (i, i + d mod N) for d = 1 ..
  // (N - 1) / 2 and then, for even N, (i, i + N / 2) with i < N / 2: each unordered
  // pair once
  double v = 0.0;
  {
    const double* r = R + w * N * 3;
    const int nn = P.n_nuc, H = (N - 1) / 2;
    const int n_ee = N * (N - 1) / 2, n_en = N * nn, n_nn = nn * (nn - 1) / 2;
    for (int t = threadIdx.x; t < n_ee + n_en + n_nn; t += blockDim.x) {
      const double *a, *b;
      double q;
      if (t < n_ee) {
        int i, j;
        if (t < N * H) {
          i = t / H;
          j = i + t % H + 1;
          if (j >= N) j -= N;
        } else {
          i = t - N * H;
          j = i + N / 2;
        }
        a = r + 3 * i;
        b = r + 3 * j;
        q = 1.0;
      } else if (t < n_ee + n_en) {
        const int u = t - n_ee, i = u / nn, A = u - i * nn;
        a = r + 3 * i;
        b = P.nuc_xyz + 3 * A;
        q = -P.Z[A];
      } else {
        int u = t - n_ee - n_en, A = 0;
        while (u >= nn - 1 - A) {
          u -= nn - 1 - A;
          A++;
        }
        const int B = A + 1 + u;
        a = P.nuc_xyz + 3 * A;
        b = P.nuc_xyz + 3 * B;
        q = P.Z[A] * P.Z[B];
      }
      const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
      v = fma(q, coulomb_inv_r(fma(dx, dx, fma(dy, dy, dz * dz))), v);
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const double inv = 1.0 / psit;
  bool finite = true;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const double gx = Gs[t][0] * inv, gy = Gs[t][1] * inv, gz = Gs[t][2] * inv, lp = Gs[t][3] * inv;
    grad[(w * N + t) * 3 + 0] = gx;
    grad[(w * N + t) * 3 + 1] = gy;
    grad[(w * N + t) * 3 + 2] = gz;
    lap[w * N + t] = lp;
    finite &= isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(lp);
  }
  const int all_finite = __syncthreads_and(finite);
  // first-order error estimate of the table result: every determinant ratio
  // carries a relative error ~ u cond_1(S_ref); the derivative sums add terms
  // of the aggregated matrices with cancellation ratio (sum of |terms|) /
  // max(|G|, rms over the walker's electrons), and the aggregation over the
  // expansion cancels like the CI sum itself, kappa_Psi = (sum_ij |c_ij r_i r_j|)
  // / |Psi~|. The estimate is u cond_1 (sum of |terms|) / max(|G|, rms) kappa_Psi
  // (l1 form; the l2 form adds the terms in quadrature). The l1 form decides the
  // fallback.
  const bool fb_on = P.fallback_tol > 0.0 && P.n_up <= MDET_FALLBACK_MAX_SPIN;
  if (fb_on) {
    if (threadIdx.x < 4) {
      float r = 0.0f;
      for (int i = 0; i < N; i++) {  // magnitudes from the FP64 bits: no conversions on the FP64 pipe
        const float a = abs_f32_of(Gs[i][threadIdx.x]);
        r = fmaf(a, a, r);
      }
      rmsG[threadIdx.x] = sqrtf(r / N);
    }
    __syncthreads();
    const float u = MIXED ? 0x1p-47f : 0x1p-53f;
    float e1 = 0.0f, e2 = 0.0f;
    for (int t = threadIdx.x; t < N * 4; t += blockDim.x) {
      const int i = t >> 2, mu = t & 3;
      const float kap = fminf(abs_f32_of(S.kap[w * 2 + (i < nu ? 0 : 1)]), 1e30f);
      const float den = fmaxf(abs_f32_of(Gs[i][mu]), rmsG[mu]);
      e1 = fmaxf(e1, u * kap * Ga[i][mu] / den);
      e2 = fmaxf(e2, u * kap * G2[i][mu] / den);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      e1 = fmaxf(e1, __shfl_xor_sync(0xffffffffu, e1, off));
      e2 = fmaxf(e2, __shfl_xor_sync(0xffffffffu, e2, off));
    }
    __shared__ float wmax[2][NW];
    if ((threadIdx.x & 31) == 0) {
      wmax[0][threadIdx.x >> 5] = e1;
      wmax[1][threadIdx.x >> 5] = e2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float m0 = 0.0f, m1 = 0.0f;
      for (int q = 0; q < NW; q++) {
        m0 = fmaxf(m0, wmax[0][q]);
        m1 = fmaxf(m1, wmax[1][q]);
      }
      estw[0][0] = m0;
      estw[1][0] = m1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double tl = 0.0;
    for (int i = 0; i < N; i++) tl += Gs[i][3];
    double vpot = 0.0;
    for (int q = 0; q < NW; q++) vpot += red[q];
    const double el = -0.5 * tl * inv + vpot;
    const double lg = ld + log(fabs(psit));
    const int s = (psit > 0.0) - (psit < 0.0);
    log_abs_psi[w] = lg;
    sign[w] = (int8_t)(sg > 0 ? s : (sg < 0 ? -s : 0));
    if (e_local) e_local[w] = el;
    uint32_t st = S.wstat[w];
    if (fb_on) {
      const float kpsi = fmaxf(1.0f, S.psia[w] / fabsf((float)psit));  // conditioning of the CI sum
      const float e1 = estw[0][0] * kpsi, e2 = estw[1][0] * kpsi;
      S.est[w * 2] = e1;
      S.est[w * 2 + 1] = e2;
      if (!(e1 <= (float)P.fallback_tol)) st |= MDET_WS_FALLBACK;
    }
    if (psit == 0.0) st |= MDET_WS_PSI_ZERO;
    if (!all_finite || !isfinite(el) || !isfinite(lg)) st |= MDET_WS_NONFINITE;
    S.wstat[w] = st;
    if (status) status[w] = st;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
template <int EC>
static cudaError_t launch_mo_f64_ec(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                                   cudaStream_t st) {
  const size_t smem = sizeof(double) * 5 * EC * P.n_ao;
  static SmemOptIn opt;  // dynamic shared memory (static arrays come on top)
  cudaError_t e = opt.ensure(k_mo_f64<EC>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)n_walk, (P.n_elec + EC - 1) / EC);
  k_mo_f64<EC><<<grid, 128, smem, st>>>(P, S.phi, R, S.live);
  return cudaGetLastError();
}

cudaError_t launch_mo_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                          cudaStream_t st) {
  switch (P.mo_ec) {
    case 1: return launch_mo_f64_ec<1>(P, S, n_walk, R, st);
    case 2: return launch_mo_f64_ec<2>(P, S, n_walk, R, st);
    case 4: return launch_mo_f64_ec<4>(P, S, n_walk, R, st);
    case 8: return launch_mo_f64_ec<8>(P, S, n_walk, R, st);
    default: return launch_mo_f64_ec<6>(P, S, n_walk, R, st);
  }
}

cudaError_t launch_ref_tables(const DevProblem& P, const DevScratch& S, int64_t n_walk, bool mixed,
                              cudaStream_t st) {
  if (mixed)
    k_ref<true><<<(unsigned)n_walk, 64, 0, st>>>(P, S);
  else
    k_ref<false><<<(unsigned)n_walk, 64, 0, st>>>(P, S);
  return cudaGetLastError();
}

cudaError_t launch_ratios_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk, cudaStream_t st) {
  const int ntot = P.n_det_sp[0] + P.n_det_sp[1];
  const int64_t wpad = (n_walk + 31) / 32 * 32;
  dim3 grid((ntot + 31) / 32, (unsigned)(wpad / 32));
  k_ratio_f64<<<grid, 128, 0, st>>>(P, S);
  return cudaGetLastError();
}

// The contraction of an escalated re-evaluation (few walkers, live count on the
// device): 4 walkers per lane and no magnitude sum, because the walkers keep the
// sum of the evaluation that flagged them (gathered into psia). Decided in one
// place for the zeroing and the launch, which must agree on whether psia is summed.
// An escalated re-evaluation (live count set) always takes the narrow FP64 kernel, which leaves
// the gathered magnitude sums psia alone (k_ref does not clear them there either).
static bool narrow_contraction(const DevProblem&, const DevScratch& S) { return S.live != nullptr; }

cudaError_t launch_zero_f64(const DevProblem&, const DevScratch&, int64_t, cudaStream_t) {
  // nothing left to clear here: the contraction stores whole segments, the ratio kernels clear
  // the entries of cut segments and the reference kernel the Psi~ sums of its walker
  return cudaSuccess;
}

cudaError_t launch_contract_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk, cudaStream_t st,
                                unsigned long long* queue, int persistent_blocks, unsigned long long* stamp) {
  // an escalated re-evaluation (few walkers, live count on the device) uses 4 walkers per lane
  const bool narrow = narrow_contraction(P, S);
  const int64_t n_groups = narrow ? (n_walk + 127) / 128 : (n_walk + 255) / 256;
  const int64_t work_max = (int64_t)std::max(P.n_items[0], P.n_items[1]) * n_groups;
  // one work item per warp (full occupancy hides the L2 latency of the gathers), or a
  // persistent grid whose warps draw items from a queue (two counters, one per launch)
  const int cap = P.spmm_blocks > 0 ? P.spmm_blocks : persistent_blocks;
  const bool q = queue && cap > 0 && cap < (work_max + 3) / 4;
  // the two counters, and the four stamp words (with one memset when they follow the counters)
  const bool adjacent = q && stamp == queue + 2;
  if (q) {
    cudaError_t e = cudaMemsetAsync(queue, 0, (adjacent ? 6 : 2) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if (stamp && !adjacent) {
    cudaError_t e = cudaMemsetAsync(stamp, 0, 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  auto grid = [&](int o) -> unsigned {
    const int64_t full = ((int64_t)P.n_items[o] * n_groups + 3) / 4;
    return (unsigned)std::max<int64_t>(1, q ? std::min<int64_t>(full, cap) : full);
  };
  const int64_t ndt = (int64_t)P.n_det_sp[0] + P.n_det_sp[1];
  const double* r_up = S.r;
  const double* r_dn = S.r + (size_t)P.n_det_sp[0] * S.wp;
  if (!narrow && P.contract_impl == 1 && S.rdf && P.csr_val_df) {  // double-float option of the mixed path
    const float2* x_up = S.rdf;
    const float2* x_dn = S.rdf + (size_t)P.n_det_sp[0] * S.wp;
    auto gdf = [&](int o) -> unsigned {
      const int64_t full = ((int64_t)P.n_items[o] * n_groups + 3) / 4;
      return (unsigned)std::max<int64_t>(1, P.spmm_blocks > 0 ? std::min<int64_t>(full, P.spmm_blocks) : full);
    };
    k_spmm_df<<<gdf(0), 128, 0, st>>>(P.csr_row, P.csr_col, P.csr_val_df, P.items[0], P.n_items[0], n_groups, x_dn,
                                      S.wp, S.vu, ndt, 0, r_up, S.psit, S.psia);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_spmm_df<<<gdf(1), 128, 0, st>>>(P.csc_col, P.csc_row, P.csc_val_df, P.items[1], P.n_items[1], n_groups, x_up,
                                      S.wp, S.vu, ndt, P.n_det_sp[0], nullptr, nullptr, nullptr);
    return cudaGetLastError();
  }
  // v = C r_dn (rows = up determinants) with Psi~ = r_up . v and its magnitude sum (an escalated
  // re-evaluation reuses the magnitude sum of the evaluation that flagged it)
  auto* kv = narrow ? k_spmm_seg<false, false, 4> : (q ? k_spmm_seg<true, true, 8> : k_spmm_seg<false, true, 8>);
  kv<<<grid(0), 128, 0, st>>>(P.csr_row, P.csr_col, P.csr_val, P.items[0], P.n_items[0], n_groups, r_dn, S.wp, S.vu,
                              ndt, 0, r_up, S.psit, narrow ? nullptr : S.psia, queue, S.live, stamp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // u = C^T r_up (columns = down determinants), in the paper's column-major order
  auto* ku = narrow ? k_spmm_seg<false, false, 4> : (q ? k_spmm_seg<true, false, 8> : k_spmm_seg<false, false, 8>);
  ku<<<grid(1), 128, 0, st>>>(P.csc_col, P.csc_row, P.csc_val, P.items[1], P.n_items[1], n_groups, r_up, S.wp, S.vu,
                              ndt, P.n_det_sp[0], nullptr, nullptr, nullptr, q ? queue + 1 : nullptr, S.live,
                              stamp ? stamp + 2 : nullptr);
  return cudaGetLastError();
}

DevScratch scratch_view(const DevScratch& S, const DevProblem& P, int64_t off) {
  DevScratch V = S;
  if (off == 0) return V;
  const int64_t N = P.n_elec, M = P.n_mo;
  V.phi = S.phi + off * 5 * N * M;
  V.Ainv = S.Ainv + off * (P.n_up * P.n_up + P.n_dn * P.n_dn);
  V.ld0 = S.ld0 + off * 2;
  V.sg0 = S.sg0 + off * 2;
  V.g = S.g + off * N * 4;
  V.kap = S.kap + off * 2;
  V.est = S.est + off * 2;
  V.wstat = S.wstat + off;
  V.vu = S.vu + off * ((int64_t)P.n_det_sp[0] + P.n_det_sp[1]);
  V.T = S.T + off;  // walker-minor: a column offset with the same stride
  if (S.Tdf) V.Tdf = S.Tdf + off;
  V.r = S.r + off;
  if (S.rdf) V.rdf = S.rdf + off;
  V.psit = S.psit + off;
  V.psia = S.psia + off;
  return V;
}

cudaError_t launch_spmm_rows_f64(const DevProblem& P, const double* r_dn, const double* r_up, double* v,
                                 double* psit, int64_t ld, int64_t n_walk, cudaStream_t st) {
  const int chunk = 512;
  const int64_t nchunks = (P.nnz + chunk - 1) / chunk;
  dim3 grid((unsigned)((nchunks + 7) / 8), (unsigned)((n_walk + 127) / 128));
  k_spmm_f64<<<grid, 256, 0, st>>>(P.csr_row, P.csr_col, P.csr_val, P.nnz, chunk, r_dn, v, ld, r_up, psit);
  return cudaGetLastError();
}

size_t final_smem_bytes(const DevProblem& P, bool mixed) {
  const size_t NM = (size_t)P.n_elec * P.n_mo;
  const size_t NMt = (size_t)P.n_elec * (P.n_mo + 1);  // rows padded by one pair (MIXED)
  const size_t AB = 2 * (size_t)(P.n_up * P.n_up + P.n_dn * P.n_dn);
  // FP64: T, W (three FP32 words), Q, A blocks and Pm; MIXED: W (hi and lo words), Q and T
  // pairs, A blocks and Pm
  return mixed ? 8 * (NM + 2 * NMt + AB) : 8 * (2 * NM + (3 * NM + 1) / 2 + AB);
}

cudaError_t launch_final(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                         double* log_abs_psi, int8_t* sign, double* grad, double* lap, double* e_local,
                         uint32_t* status, bool mixed, cudaStream_t st, bool wide) {
  const size_t smem = final_smem_bytes(P, mixed);
  // wide: 512 threads per walker (FP64 only), for a few walkers whose latency matters
  const int variant = mixed ? 1 : (wide ? 2 : 0);
  auto kern = variant == 1 ? k_final<true, 128> : (variant == 2 ? k_final<false, 512> : k_final<false, 128>);
  const int nt = variant == 2 ? 512 : 128;
  static SmemOptIn opt[3];  // dynamic shared memory per variant (static arrays come on top)
  cudaError_t e = opt[variant].ensure(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)n_walk, nt, smem, st>>>(P, S, R, log_abs_psi, sign, grad, lap, e_local, status);
  return cudaGetLastError();
}

}  // namespace mdet

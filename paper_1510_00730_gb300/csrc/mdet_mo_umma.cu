// Orbitals of the mixed path on the 5th-generation tensor cores (tcgen05, TMEM).
//
// Phi = X B (Sec. 2: value, gradient and Laplacian of every MO at every
// electron) to double-float accuracy with BF16 MMAs, by exact digit products
// (an Ozaki-type scheme): each row r of X (one quantity of one electron over the
// AOs) is 2^e_r sum_i d_i 2^(-8 i) and each column m of B is 2^f_m sum_j b_j 2^(-8 j),
// i, j = 1..7, with integer digits |d_1|, |b_1| <= 256 and the others <= 128, all
// exact in BF16. For one order t = i + j <= 8 the sum over K <= 112 AOs of the
// digit products of all pairs (i, j) stays below 2^24 in magnitude, so the FP32
// accumulator of the tensor core returns it exactly: G_t = sum_{i+j=t} sum_k d_ik b_jk.
// Then Phi = 2^(e_r + f_m) sum_t 2^(-8 t) G_t, summed in double-float as the
// orders complete. The digits cut X at 2^-57 of the row maximum and B at 2^-57
// of the column maximum; the dropped orders t >= 9 weigh below 2^-64.
//
// Roles. The MMA's A operand (M = 128 TMEM lanes) is the MO digit planes B^T,
// loaded into TMEM once per CTA (lane m = MO m, plane j at columns (j-1) Kp/2,
// two BF16 per 32-bit column). The B operand (N = 32) is the AO digit planes of
// 32 electrons for one quantity, in shared memory as K-major 8 x 16-byte core
// matrices without swizzle. The accumulator D[m][e] (128 lanes x 32 columns)
// is double-buffered in TMEM, so the MMAs of order t + 1 run while the warps
// drain order t into double-float registers. A CTA loops over tiles of 32
// electrons (all walkers' electrons in one flat list); per tile it evaluates the
// AOs of every (shell, electron) once, then takes the five quantities in turn.
//
// Resources: 256 threads at <= 96 registers and one CTA per SM (the staging of
// the AO values takes most of shared memory), which leaves room on every SM for
// the persistent FP64 contraction grid that runs beside it in the walker-chunk
// pipeline. Every wait on an mbarrier is bounded; a CTA whose wait runs out
// writes NaN orbitals for the rest of its tiles (the epilogue then flags those
// walkers as non-finite), releases its tensor memory and returns.
// Output: Phi[w][c][e][m] as double-float pairs (hi, lo), the mixed path's layout
// of the orbital array (same size as FP64).
#include <algorithm>
#include <cstdint>

#include "df32.cuh"
#include "mdet_device.cuh"
#include "mdet_internal.h"
#include "umma.cuh"

namespace mdet {

namespace {

constexpr int kNE = 32;            // electrons per tile: the MMA's N
constexpr int kDigits = 7;         // digits per operand
constexpr int kMaxKp = 112;        // AOs (padded to 16) for which the order sums stay exact
constexpr int kThreads = 256;
constexpr int kWaitLimit = 1 << 26;        // polls of an mbarrier before a CTA gives up

using umma::smem_u32;

// acc + x (x a single float) in double-float
__device__ __forceinline__ df32 df_add_f(df32 a, float x) {
  float s, e;
  two_sum(a.hi, x, s, e);
  float hi, lo;
  fast_two_sum(s, __fadd_rn(a.lo, e), hi, lo);
  return {hi, lo};
}

__global__ void __maxnreg__(96) k_mo_umma(DevProblem P, float2* __restrict__ phi, const double* __restrict__ R,
                                          int64_t n_el, int64_t n_tiles) {
  extern __shared__ __align__(128) uint8_t smu[];
  const int Kp = P.tc_kp, K = P.n_ao, M = P.n_mo, N = P.n_elec, Mp = P.tc_mp;
  const int sbo = (Kp / 8) * 128 + 16;  // 8-row groups 16 bytes apart mod 128: conflict-free digit stores
  // TMEM columns: the MO digit planes at [0, 7 Kp / 2), then the two 32-column accumulators
  const uint32_t dcol0 = (uint32_t)((kDigits * (Kp / 2) + 31) / 32 * 32);
  const uint32_t ncols = dcol0 + 64 <= 128 ? 128 : (dcol0 + 64 <= 256 ? 256 : 512);
  const int plane_bytes = (kNE / 8) * sbo;
  float2* X = reinterpret_cast<float2*>(smu);              // [5][Kp][kNE] AO values (hi, lo)
  uint8_t* planes = smu + (size_t)5 * Kp * kNE * sizeof(float2);  // [7][plane_bytes] AO digits
  __shared__ df32 rdf[kNE][3];
  __shared__ float red[kThreads / 32][kNE];
  __shared__ int er[kNE];
  __shared__ __align__(8) uint64_t full[2], empty[2], fin;
  __shared__ uint32_t tbase;
  __shared__ int stop_s;
  volatile int* stop = &stop_s;  // set when a wait runs out
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter (MOs 32q..32q+31) and column half of the drains

  if (warp == 0) {
    umma::tmem_alloc(&tbase, ncols);
  }
  if (tid == 0) {
    umma::mbar_init(&full[0], 1);
    umma::mbar_init(&full[1], 1);
    umma::mbar_init(&empty[0], kThreads / 32);
    umma::mbar_init(&empty[1], kThreads / 32);
    umma::mbar_init(&fin, 1);
    *stop = 0;
  }
  for (int i = tid; i < 5 * Kp * kNE; i += kThreads) X[i] = make_float2(0.0f, 0.0f);  // AO padding stays zero
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tb = tbase;
  const uint32_t lane_q = (uint32_t)(32 * q) << 16;
  // MO digit planes into TMEM (warps q and q + 4 share a lane quarter and split the planes)
  {
    const int m = 32 * q + lane;
    for (int j = h; j < kDigits; j += 2)
      for (int c0 = 0; c0 < Kp / 2; c0 += 8) {
        uint32_t v[8];
#pragma unroll
        for (int x = 0; x < 8; x++)
          v[x] = m < Mp ? __ldg(reinterpret_cast<const unsigned int*>(P.B_dig + ((size_t)j * Mp + m) * Kp + 2 * (c0 + x)))
                        : 0u;
        umma::tmem_st8(tb + lane_q + (uint32_t)(j * (Kp / 2) + c0), v);
      }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();

  const uint32_t idesc = umma::idesc_bf16(128, kNE);
  const uint32_t planes_s = smem_u32(planes);
  uint32_t u = 0;  // orders issued so far by this CTA (the same count in every thread)
  // the MMAs of order t into accumulator (uu & 1), after its previous use has been drained
  auto issue = [&](int t, uint32_t uu) {
    const int b = uu & 1;
    if (*stop) return;
    if (uu >= 2) {
      if (!umma::mbar_wait(&empty[b], ((uu - 2) >> 1) & 1, kWaitLimit)) {
        *stop = 1;
        return;
      }
      umma::fence_after();
    }
    uint32_t acc = 0;
    for (int i = max(1, t - kDigits); i <= min(kDigits, t - 1); i++) {
      const int j = t - i;
      for (int ks = 0; ks < Kp / 16; ks++) {
        const uint64_t bd = umma::desc(planes_s + (uint32_t)((i - 1) * plane_bytes + ks * 256), 128, (uint32_t)sbo);
        umma::mma_tmem_a(tb + dcol0 + 32u * b, tb + (uint32_t)((j - 1) * (Kp / 2) + ks * 8), bd, idesc, acc);
        acc = 1;
      }
    }
    umma::commit(&full[b]);
  };

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t g0 = tile * kNE;  // first electron of the tile in the flat list of all walkers' electrons
    if (*stop) {  // a wait ran out: no orbitals for the rest of this CTA's tiles
      for (int i = tid; i < 5 * kNE * M; i += kThreads) {
        const int e = i / (5 * M), r = i - e * 5 * M, c = r / M, m = r - c * M;
        const int64_t g = g0 + e;
        if (g < n_el) phi[(((g / N) * 5 + c) * N + g % N) * M + m] = make_float2(__int_as_float(0x7fc00000), 0.0f);
      }
      continue;
    }
    if (tid < 3 * kNE) {
      const int e = tid / 3, d = tid - 3 * e;
      rdf[e][d] = g0 + e < n_el ? df_from_double(R[(g0 + e) * 3 + d]) : df32(0.0f, 0.0f);
    }
    __syncthreads();
    // AO values and derivatives of every (shell, electron) in double-float: warps take shells, lanes electrons
    for (int s = warp; s < P.n_shell; s += kThreads / 32) {
      if (g0 + lane >= n_el) continue;
      const int ao0 = P.shell_ao0[s];
      ao_shell_values_df(P, s, rdf[lane], [&](int c, int qq, df32 v) {
        X[((size_t)c * Kp + ao0 + qq) * kNE + lane] = make_float2(v.hi, v.lo);
      });
    }
    __syncthreads();
    for (int c = 0; c < 5; c++) {
      const float2* Xc = X + (size_t)c * Kp * kNE;
      // row exponents: |x| < 2^er[e] over the row
      {
        float mx = 0.0f;
        for (int k = warp; k < K; k += kThreads / 32) mx = fmaxf(mx, fabsf(Xc[k * kNE + lane].x));
        red[warp][lane] = mx;
      }
      __syncthreads();
      if (tid < kNE) {
        float mx = 0.0f;
#pragma unroll
        for (int p = 0; p < kThreads / 32; p++) mx = fmaxf(mx, red[p][tid]);
        er[tid] = mx > 0.0f ? ilogbf(mx) + 1 : 0;
      }
      __syncthreads();
      // digits of 8 consecutive AOs of one electron: one 16-byte core-matrix row per plane
      for (int it = tid; it < kNE * (Kp / 8); it += kThreads) {
        const int e = it & (kNE - 1), kg = it / kNE;
        const int sh = -er[e];
        uint32_t w[kDigits][4];
#pragma unroll
        for (int z = 0; z < 8; z++) {
          const float2 x = Xc[(kg * 8 + z) * kNE + e];
          float vh = ldexpf(x.x, sh), vl = ldexpf(x.y, sh);
#pragma unroll
          for (int i = 0; i < kDigits; i++) {
            vh = __fmul_rn(vh, 256.0f);
            vl = __fmul_rn(vl, 256.0f);
            const float d = rintf(vh);
            float s2, e2;
            two_sum(__fsub_rn(vh, d), vl, s2, e2);
            vh = s2;
            vl = e2;
            const uint32_t bits = __float_as_uint(d) >> 16;  // |d| <= 256: exact in BF16
            if (z & 1)
              w[i][z >> 1] |= bits << 16;
            else
              w[i][z >> 1] = bits;
          }
        }
        uint8_t* dst = planes + (e >> 3) * sbo + kg * 128 + (e & 7) * 16;
#pragma unroll
        for (int i = 0; i < kDigits; i++)
          *reinterpret_cast<uint4*>(dst + i * plane_bytes) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      umma::fence_before();
      __syncthreads();
      umma::fence_after();
      // orders t = 2..8: MMAs of t + 1 in flight while every warp drains t
      df32 acc[16];
#pragma unroll
      for (int j = 0; j < 16; j++) acc[j] = df32(0.0f, 0.0f);
      if (tid == 0) issue(2, u);
      __syncwarp();
      for (int t = 2; t <= 8; t++, u++) {
        if (tid == 0 && t < 8) issue(t + 1, u + 1);
        __syncwarp();
        const int b = u & 1;
        const bool ok = !*stop && umma::mbar_wait(&full[b], (u >> 1) & 1, kWaitLimit);
        if (!ok) *stop = 1;
        umma::fence_after();
        if (32 * q < M && __all_sync(0xffffffffu, ok)) {  // lane quarters beyond the MOs hold zeros
          uint32_t v[16];
          umma::tmem_ld16(tb + lane_q + dcol0 + 32u * b + 16 * h, v);
          const float scale = __uint_as_float((uint32_t)(127 - 8 * t) << 23);  // 2^(-8 t)
#pragma unroll
          for (int j = 0; j < 16; j++) acc[j] = df_add_f(acc[j], __fmul_rn(__uint_as_float(v[j]), scale));
        }
        umma::fence_before();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&empty[b]);
      }
      // Phi[w][c][e][m] = 2^(er + f_m) acc as a double-float pair
      const int m = 32 * q + lane;
      if (m < M) {
        const int f = P.B_exp[m];
#pragma unroll
        for (int j = 0; j < 16; j++) {
          const int e = 16 * h + j;
          const int64_t g = g0 + e;
          if (g >= n_el) break;
          const int E = er[e] + f;
          phi[(((g / N) * 5 + c) * N + g % N) * M + m] =
              *stop ? make_float2(__int_as_float(0x7fc00000), 0.0f) : make_float2(ldexpf(acc[j].hi, E), ldexpf(acc[j].lo, E));
        }
      }
      umma::fence_before();
      __syncthreads();  // digit planes and row exponents are rewritten by the next quantity
      umma::fence_after();
    }
  }
  umma::fence_before();
  __syncthreads();
  if (*stop && tid == 0) {  // after a wait ran out: let the MMAs in flight finish (bounded) before the release
    umma::commit(&fin);
    umma::mbar_wait(&fin, 0, kWaitLimit);
  }
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tb, ncols);
}

}  // namespace

size_t mo_umma_smem_bytes(const DevProblem& P) {
  const size_t sbo = (size_t)(P.tc_kp / 8) * 128 + 16;
  return (size_t)5 * P.tc_kp * kNE * sizeof(float2) + (size_t)kDigits * (kNE / 8) * sbo;
}

bool mo_umma_supported(const DevProblem& P) {
  return P.B_dig && P.tc_kp <= kMaxKp && P.n_mo <= 128 && mo_umma_smem_bytes(P) <= 220 * 1024;
}

cudaError_t launch_mo_umma(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R, int n_sm,
                           cudaStream_t st) {
  const size_t smem = mo_umma_smem_bytes(P);
  static SmemOptIn opt;
  cudaError_t e = opt.ensure(k_mo_umma, smem);
  if (e != cudaSuccess) return e;
  const int64_t n_el = n_walk * P.n_elec;
  const int64_t n_tiles = (n_el + kNE - 1) / kNE;
  const int64_t grid = std::min<int64_t>(n_tiles, std::max(n_sm, 1));
  k_mo_umma<<<(unsigned)grid, kThreads, smem, st>>>(P, reinterpret_cast<float2*>(S.phi), R, n_el, n_tiles);
  return cudaGetLastError();
}

}  // namespace mdet

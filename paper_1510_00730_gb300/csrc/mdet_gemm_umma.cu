// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory) with a fused epilogue: the three layers of the learned
// proposal's perceptron, forward and backward.
//
// D[m][n] = sum_k A[m][k] B[n][k] over a CTA's range of k, with
//   A (M x K) and B (N x K) read through strided views of FP32 or BF16 arrays
//   (element (r, k) at p[r * rs + k * ks], zero outside the matrix), so that the
//   transposed operands of the backward pass need no copies;
//   operands rounded to BF16 (nearest even) as they are staged, FP32 accumulation.
// Tile: 128 rows of A (the TMEM lanes) x up to 256 rows of B (TMEM columns), K in
// chunks of 64. Per chunk the 128 threads stage both operands into shared memory as
// K-major core matrices of 8 rows x 16 bytes (no swizzle; 8-row groups 1 KB apart,
// core matrices along K 128 B apart), one thread issues four MMAs of K = 16 and
// commits them to an mbarrier, and all threads wait for it before the next chunk
// overwrites the tiles. Then each warp reads its 32 TMEM lanes back with tcgen05.ld
// and applies the epilogue:
//   kEpiTanhBias  out = tanh(D + bias[n])          (hidden layers)
//   kEpiBias      out = D + bias[n]                (output layer)
//   kEpiDtanh     out = D * (1 - h[m][n]^2)        (back through a tanh layer)
//   kEpiAtomic    out += D with FP32 atomics       (weight gradients, split over k)
//   kEpiStore     out = D
// Every mbarrier wait is bounded: a CTA whose wait runs out writes NaN through its
// epilogue, waits (bounded) for its MMAs in flight, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "../../include/mdet_vmc.h"
#include "mdet_internal.h"
#include "umma.cuh"

namespace mdet {

namespace {

constexpr int kGM = 128;      // rows of A per CTA: the MMA's M (TMEM lanes)
constexpr int kGN = 256;      // rows of B per CTA: the largest N of one MMA
constexpr int kGK = 64;       // K per staged chunk: four MMAs of K = 16
constexpr int kThreads = 128;
constexpr int kTmemCols = 256;
constexpr int kWaitLimit = 1 << 24;
constexpr int kTileA = kGM * kGK * 2;  // bytes of the staged A chunk
constexpr int kTileB = kGN * kGK * 2;
// 100 KB of dynamic shared memory per CTA (the tiles take 48 KB) keeps at most two CTAs
// on an SM, whose 2 x 256 tensor-memory columns fit its 512
constexpr size_t kSmem = 100 * 1024;
static_assert(kTileA + kTileB <= (int)kSmem, "tiles exceed the dynamic shared memory");

__device__ __forceinline__ float op_get(const GemmOperand& o, int64_t r, int64_t k) {
  if (r >= o.rows || k >= o.cols) return 0.0f;
  const int64_t i = r * o.rs + k * o.ks;
  return o.bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(o.p)[i]) : static_cast<const float*>(o.p)[i];
}

// rows [r0, r0 + nr) and k [k0, k0 + 64) of o, as BF16, into the K-major tile s:
// element (r, k) at (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
__device__ __forceinline__ void stage(const GemmOperand& o, int64_t r0, int nr, int64_t k0, uint8_t* s) {
  for (int r = threadIdx.x; r < nr; r += kThreads) {
#pragma unroll 2
    for (int g = 0; g < kGK / 8; g++) {
      uint32_t w[4];
#pragma unroll
      for (int h = 0; h < 4; h++) {
        const int64_t k = k0 + 8 * g + 2 * h;
        const __nv_bfloat162 b = __floats2bfloat162_rn(op_get(o, r0 + r, k), op_get(o, r0 + r, k + 1));
        w[h] = *reinterpret_cast<const uint32_t*>(&b);  // even k in the low half
      }
      *reinterpret_cast<uint4*>(s + (r >> 3) * 1024 + g * 128 + (r & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_gemm_bf16(GemmOperand A, GemmOperand B, int64_t k_per_cta,
                                                        GemmEpilogue E) {
  extern __shared__ __align__(1024) uint8_t smg[];
  uint8_t* sA = smg;
  uint8_t* sB = smg + kTileA;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ int stop_s;
  volatile int* stop = &stop_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t m0 = (int64_t)blockIdx.x * kGM, n0 = (int64_t)blockIdx.y * kGN;
  const int64_t kb = (int64_t)blockIdx.z * k_per_cta, ke = A.cols < kb + k_per_cta ? A.cols : kb + k_per_cta;
  const int nt = (int)(B.rows - n0 < kGN ? B.rows - n0 : kGN);  // rows of B in this tile
  const int nmma = (nt + 15) / 16 * 16;                     // the MMA's N (a multiple of 16)
  if (warp == 0) umma::tmem_alloc(&tbase, kTmemCols);
  if (tid == 0) {
    umma::mbar_init(&bar, 1);
    *stop = 0;
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tb = tbase;
  const uint32_t idesc = umma::idesc_bf16(kGM, nmma);
  const uint32_t a_s = umma::smem_u32(sA), b_s = umma::smem_u32(sB);
  uint32_t phase = 0;
  bool any = false;  // at least one chunk accumulated
  for (int64_t k0 = kb; k0 < ke; k0 += kGK) {
    stage(A, m0, kGM, k0, sA);
    stage(B, n0, nmma, k0, sB);
    umma::fence_smem_async();
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kGK / 16; ks++)
        umma::mma_smem_a(tb, umma::desc(a_s + ks * 256, 128, 1024), umma::desc(b_s + ks * 256, 128, 1024), idesc,
                         (any || ks > 0) ? 1u : 0u);
      umma::commit(&bar);
    }
    any = true;
    if (!umma::mbar_wait(&bar, phase, kWaitLimit)) *stop = 1;
    phase ^= 1u;
    umma::fence_after();
    __syncthreads();  // the tiles are free again, and every thread sees the same stop flag
    if (*stop) break;
  }
  // epilogue: warp w holds rows m0 + 32 w + lane in TMEM lanes 32 w + lane
  const int64_t m = m0 + tid;
  const bool row_ok = any && m < A.rows;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (int c0 = 0; c0 < nmma; c0 += 16) {
    uint32_t v[16];
    umma::tmem_ld16(tb + lane_base + (uint32_t)c0, v);  // the whole warp, converged
    if (!row_ok) continue;
#pragma unroll
    for (int j = 0; j < 16; j++) {
      const int64_t n = n0 + c0 + j;
      if (c0 + j >= nt) break;
      const float d = *stop ? __int_as_float(0x7fc00000) : __uint_as_float(v[j]);
      float* o = E.out + m * E.ldm + n * E.ldn;
      switch (E.kind) {
        case kEpiTanhBias: *o = tanhf(d + E.bias[n]); break;
        case kEpiBias: *o = d + E.bias[n]; break;
        case kEpiStore: *o = d; break;
        case kEpiDtanh: {
          const float h = E.h[m * E.ldh + n];
          *o = d * (1.0f - h * h);
          break;
        }
        default: atomicAdd(o, d);
      }
    }
  }
  umma::fence_before();
  __syncthreads();
  if (*stop && tid == 0) {  // a wait ran out: let the MMAs in flight finish (bounded) before the release
    umma::commit(&bar);
    umma::mbar_wait(&bar, phase, kWaitLimit);
  }
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tb, kTmemCols);
}

}  // namespace

cudaError_t launch_gemm_bf16(const GemmOperand& A, const GemmOperand& B, int64_t k_per_cta, const GemmEpilogue& E,
                             cudaStream_t st) {
  if (A.rows <= 0 || B.rows <= 0 || A.cols <= 0) return cudaSuccess;
  const int64_t kc = std::max<int64_t>(kGK, (k_per_cta + kGK - 1) / kGK * kGK);
  const dim3 grid((unsigned)((A.rows + kGM - 1) / kGM), (unsigned)((B.rows + kGN - 1) / kGN),
                  (unsigned)((A.cols + kc - 1) / kc));
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  k_gemm_bf16<<<grid, kThreads, kSmem, st>>>(A, B, kc, E);
  return cudaGetLastError();
}

}  // namespace mdet

extern "C" mdet_status mdet_gemm_bf16(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                                      int64_t ldb, float* D, int64_t ldd, int accumulate, int64_t k_split,
                                      void* stream) {
  using namespace mdet;
  if (M < 0 || N < 0 || K < 0) return MDET_E_ARG;
  if (M == 0 || N == 0) return MDET_OK;
  if (!D || ldd < N || (K > 0 && (!A || !B || lda < K || ldb < K))) return MDET_E_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  if (K == 0) {  // an empty sum: zero, or nothing to add
    if (accumulate) return MDET_OK;
    return cudaMemset2DAsync(D, sizeof(float) * ldd, 0, sizeof(float) * N, M, st) == cudaSuccess ? MDET_OK
                                                                                                  : MDET_E_CUDA;
  }
  const GemmOperand a{A, lda, 1, M, K, 0}, b{B, ldb, 1, N, K, 0};
  const GemmEpilogue e{accumulate ? kEpiAtomic : kEpiStore, D, ldd, 1, nullptr, nullptr, 0};
  return launch_gemm_bf16(a, b, accumulate ? k_split : K, e, st) == cudaSuccess ? MDET_OK : MDET_E_CUDA;
}

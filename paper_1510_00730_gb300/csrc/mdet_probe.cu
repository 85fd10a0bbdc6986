// Measured throughput of the FP64 FMA pipe: the denominator of the roofline of
// the FP64 kernels (the sparse CI contraction is bound by it). Every thread runs
// kChains independent chains a <- fma(a, b, c), so the pipe, not the latency of
// one chain, sets the rate; the grid fills every SM with 32 warps.
#include <algorithm>

#include "mdet_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;

__global__ void __launch_bounds__(256) k_fp64_fma_rate(int64_t rounds, double b, double c, double* __restrict__ out) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int64_t i = 0; i < rounds; i++) {
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
#pragma unroll
      for (int j = 0; j < kChains; j++) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace

extern "C" mdet_status mdet_measure_fp64_rate(int device, int64_t fma_per_thread, int reps, double* tflops,
                                              double* best_ms) {
  if (!tflops || fma_per_thread < kChains * kUnroll || reps < 1) return MDET_E_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return MDET_E_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return MDET_E_CUDA;
  mdet_status st = MDET_OK;
  int n_sm = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* out = nullptr;
  float best = 0.0f;
  const int blocks_per_sm = 4, threads = 256;
  const int64_t rounds = fma_per_thread / (kChains * kUnroll);
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&out, sizeof(double) * (size_t)n_sm * blocks_per_sm * threads) != cudaSuccess) {
    st = MDET_E_CUDA;
  } else {
    const int grid = n_sm * blocks_per_sm;
    // warm-up launch, then reps timed launches; the fastest one counts
    for (int r = 0; r <= reps && st == MDET_OK; r++) {
      cudaEventRecord(e0, s);
      k_fp64_fma_rate<<<grid, threads, 0, s>>>(rounds, 0.9999999999, 1e-10, out);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = MDET_E_CUDA;
        break;
      }
      if (r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (st == MDET_OK) {
      const double fmas = (double)grid * threads * (double)(rounds * kChains * kUnroll);
      *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
      if (best_ms) *best_ms = best;
    }
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return st;
}

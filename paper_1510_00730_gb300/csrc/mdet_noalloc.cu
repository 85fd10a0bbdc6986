// An entry point that performs no device allocation: Psi~ = r_up . (C r_dn)
// from caller-supplied ratios, with the intermediate v = C r_dn kept in a
// fixed, file-scope device array instead of memory obtained from cudaMalloc.
//
// It is meant for callers that cannot allocate device memory at the point of
// the call: code running under a custom or pooled device allocator that owns
// all of the GPU's memory, or a host runtime that forbids allocation after
// start-up. Such a caller passes its own input and output buffers and gets the
// work done in this library's static scratch.
#include <cstdio>
#include <mutex>

#include "mdet_internal.h"

using namespace mdet;

namespace {

constexpr int kMaxDevices = 64;

// The scratch: v [n_det_up][ld] followed by Psi~ partial sums [ld]. Every GPU
// that loads this library holds it (MDET_NOALLOC_SCRATCH_DOUBLES doubles,
// 32 MiB) until the process exits.
__device__ __align__(256) double g_noalloc_scratch[MDET_NOALLOC_SCRATCH_DOUBLES];

// Device address of the scratch, looked up once per device. In host code the
// symbol g_noalloc_scratch is only a host-side stand-in; kernels must be given
// this address instead.
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // the device must be current
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

// The work itself, with the caller's device already switched to the context's.
mdet_status psi_tilde_on_device(const DevProblem* P, int device, int64_t n_walk, const double* r,
                                int64_t ld, double* psi_tilde, cudaStream_t st) {
  double* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return MDET_E_CUDA;
  const int64_t n_up = P->n_det_sp[0];
  double* v = scratch;                 // [n_det_up][ld]
  double* psit = scratch + n_up * ld;  // [ld]
  // the kernel accumulates with atomics: clear what this call uses
  if (cudaMemsetAsync(scratch, 0, sizeof(double) * (n_up + 1) * ld, st) != cudaSuccess) return MDET_E_CUDA;
  const double* r_up = r;
  const double* r_dn = r + n_up * ld;
  if (launch_spmm_rows_f64(*P, r_dn, r_up, v, psit, ld, n_walk, st) != cudaSuccess) return MDET_E_CUDA;
  if (cudaMemcpyAsync(psi_tilde, psit, sizeof(double) * n_walk, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return MDET_E_CUDA;
  return MDET_OK;
}

}  // namespace

extern "C" mdet_status mdet_psi_tilde_noalloc(mdet_ctx* ctx, int64_t n_walk, const double* r, int64_t ld,
                                              double* psi_tilde, void* stream) {
  int device = -1;
  const DevProblem* P = ctx_problem(ctx, &device);
  if (!P) return ctx ? MDET_E_STATE : MDET_E_ARG;
  if (n_walk < 0) return MDET_E_ARG;
  if (n_walk == 0) return MDET_OK;
  if (!r || !psi_tilde || ld < n_walk || ld % 128 != 0 || ((uintptr_t)r & 15) != 0) return MDET_E_ARG;
  // (n_det_up + 1) * ld doubles must fit the static scratch; ld is compared with the
  // quotient first, so that a huge ld cannot overflow the product
  const int64_t rows = (int64_t)P->n_det_sp[0] + 1;
  if (ld > (int64_t)MDET_NOALLOC_SCRATCH_DOUBLES / rows) {
    char msg[240];
    snprintf(msg, sizeof msg,
             "(n_det_up + 1) * ld = %lld * %lld doubles exceeds the static scratch of %u doubles; use a smaller ld "
             "(fewer walkers per call) or mdet_evaluate",
             (long long)rows, (long long)ld, MDET_NOALLOC_SCRATCH_DOUBLES);
    ctx_set_error(ctx, msg);
    return MDET_E_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return MDET_E_CUDA;
  const mdet_status s = psi_tilde_on_device(P, device, n_walk, r, ld, psi_tilde, (cudaStream_t)stream);
  // the caller's current device is left as it was
  if (cudaSetDevice(prev) != cudaSuccess && s == MDET_OK) return MDET_E_CUDA;
  return s;
}

// Internal data layout shared by the host side (mdet_host.cu) and the kernels.
// Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mdet.h"

namespace mdet {

constexpr int kMaxSpin = MDET_MAX_SPIN_ELEC;
constexpr int kMaxExc = MDET_MAX_EXC;
constexpr int kMaxL = MDET_MAX_L;
constexpr int kWalkerPad = 256;  // walker-minor arrays are padded to a multiple of this

// Dynamic shared memory a kernel has been opted into, per device (a function
// attribute belongs to each device's context). Concurrent callers at worst
// repeat the attribute call.
struct SmemOptIn {
  static constexpr int kMaxDevices = 64;
  std::atomic<size_t> bytes[kMaxDevices] = {};
  template <class K>
  cudaError_t ensure(K kernel, size_t need) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && need <= bytes[dev].load()) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) {
      size_t cur = bytes[dev].load();
      while (cur < need && !bytes[dev].compare_exchange_weak(cur, need)) {
      }
    }
    return e;
  }
};

// Excitation of one distinct spin determinant relative to the reference of its
// spin: columns h[0..k) of the reference Slater matrix (hole positions, in the
// reference's ascending MO order) are replaced by MOs p[0..k) (particles);
// eps is the sign that reorders the substituted columns ascending.
struct __align__(16) Exc {
  uint8_t k;
  int8_t eps;
  uint8_t pad0, pad1;
  uint8_t h[kMaxExc];
  uint8_t p[kMaxExc];
  uint32_t pad2;
};
static_assert(sizeof(Exc) == 16, "Exc must be 16 bytes");

// Read-only problem description resident on the device.
struct DevProblem {
  int n_up, n_dn, n_elec, n_nuc;
  int n_shell, n_ao, n_mo, n_prim;
  int n_det_sp[2];        // distinct determinants per spin
  int64_t nnz;            // products
  const struct SmStep* sm_steps[2];  // the sequential chain of each spin (mdet_sm_chain)
  int sm_n[2];
  int spmm_chunk;         // tuning: nonzeros per work item of the contraction (whole segments)
  const int2* items[2];   // work items of the contraction over the row-major (0) and column-major (1)
  int n_items[2];         //   copies of C: nonzero ranges [x, y & 0x7fffffff) of whole segments, or one
                          //   piece of a longer segment (y < 0: its sums are added atomically)
  const uint8_t* split;   // [n_det_up + n_det_dn] 1 for a segment cut into pieces (its v or u entries are
                          //   cleared before the contraction, by the ratio kernel)
  int spmm_blocks;        // tuning: grid of the contraction (0: one warp per work item)
  int contract_impl;      // tuning: contraction in FP64 (0) or double-float on the FP32 pipe (1, mixed only)
  const float2* csr_val_df;  // C values as double-float pairs, row-major and column-major orders
  const float2* csc_val_df;
  int mo_ec;              // tuning: electrons per CTA in the orbital kernels (4, 6 or 8)
  int mo_impl;            // tuning: mixed orbitals by exact digit products on the tensor cores with tcgen05 (2),
                          // with warp-level mma.sync (0), or the compensated FP32 dot product (1)
  int n_sm;               // multiprocessors of the device (persistent grids)
  int phi_df;             // the context's orbital array holds double-float pairs (mixed precision); the
                          // FP64 re-evaluation scratch of a mixed context always holds FP64
  const uint16_t* B_dig;  // [7][tc_mp][tc_kp] BF16 digits of the MO coefficients (column-scaled)
  const int* B_exp;       // [n_mo] column exponents of B_dig
  int tc_kp, tc_mp, tc_sx;  // K padded to 16, M padded to 8, shared row stride of the AO digits
  double fallback_tol;    // estimated relative error above which a walker is re-evaluated by full LU (<= 0: off)
  int fallback_cap;       // walkers re-evaluated per evaluation at most
  const double* Z;        // [n_nuc]
  const double* nuc_xyz;  // [n_nuc][3]
  const int* shell_l;     // [n_shell]
  const int* shell_center;
  const int* shell_nprim;
  const int* shell_prim0;  // first primitive of each shell
  const int* shell_ao0;    // first AO of each shell
  const double* alpha;     // [n_prim]
  const double* coef;      // [n_prim]
  const double* B;         // [n_ao][n_mo] row-major (B[mu*n_mo + m])
  const float* B_hi;       // B as double-float pairs (mixed path): B = B_hi + B_lo
  const float* B_lo;
  const float2* alpha_df;  // exponents, coefficients and nuclear positions as (hi, lo) pairs
  const float2* coef_df;
  const float2* nuc_df;
  const int* ref_occ;      // [2][kMaxSpin] ascending occupied MOs of each reference
  const Exc* exc[2];       // [n_det_sp[s]] excitation records
  int deg_start[2][kMaxExc + 2];  // first index of each excitation degree 0..kMaxExc (and the end) per spin
  // C over the distinct determinants, two orderings (Sec. 2.1, Sec. 2.4)
  const int* csr_row;      // [nnz] row (up index) of each entry, sorted by row then column
  const int* csr_col;      // [nnz]
  const double* csr_val;   // [nnz]
  const int* csc_col;      // [nnz] column (down index), sorted by column then row
  const int* csc_row;      // [nnz]
  const double* csc_val;   // [nnz]
  const int* csr_ptr;      // [n_det_up + 1] row starts of the row-major order
  const int* csc_ptr;      // [n_det_dn + 1] column starts of the column-major order
};

// Per-evaluation scratch (owned by the context, grown on demand).
struct DevScratch {
  int64_t cap_walk = 0;   // capacity in walkers
  int64_t wp = 0;         // padded walker stride of walker-minor arrays
  double* phi = nullptr;  // [W][5][n_elec][n_mo]  value, d/dx, d/dy, d/dz, Laplacian
  double* Ainv = nullptr; // [W][n_up^2 + n_dn^2]  inverses of the reference Slater matrices, A[a][i]
  double* ld0 = nullptr;  // [W][2] log|D_ref|
  double* sg0 = nullptr;  // [W][2] sign(D_ref)
  double* g = nullptr;    // [W][n_elec][4]  (d_{i mu} D_ref) / D_ref
  double* kap = nullptr;  // [W][2] cond_1 of each reference Slater matrix
  double* est = nullptr;  // [W][2] error estimates of the table result (l1 and l2 forms)
  double* T = nullptr;    // [n_up + n_dn][n_mo][wp] walker-minor ratio tables (up block then down block)
  float2* Tdf = nullptr;  // same as double-float pairs (hi, lo), mixed path only
  double* r = nullptr;    // [n_det_up + n_det_dn][wp] ratios D_I / D_ref, walker-minor
  float2* rdf = nullptr;  // same as double-float pairs (mixed path with the double-float contraction only)
  double* vu = nullptr;   // walker-major [wp][n_det_up + n_det_dn]: v = C r_dn (up) then u = C^T r_up (down)
  double* psit = nullptr; // [wp] Psi / (D_ref_up D_ref_dn)
  float* psia = nullptr;  // [wp] sum_ij |c_ij| |r_up,i| |r_dn,j| (FP32), the magnitude sum behind psit
  uint32_t* wstat = nullptr;  // [W] status bits
  double* fb = nullptr;       // fallback: [cap][n_det_up + n_det_dn][2 + 4 max(n_up, n_dn)], then [cap][ndt] values
  int* fb_list = nullptr;     // fallback: [1 + cap] count, then walker indices
  double* fb_acc = nullptr;   // fallback: [cap][3 + 8 MDET_FALLBACK_MAX_SPIN] scales, Psi, G
  unsigned long long* queue = nullptr;  // [6 * walker chunks] per chunk: the work counters of its two
                                        // persistent contractions, then their global-timer stamps
  const int* live = nullptr;  // device count of the walkers to evaluate (null: all n_walk); the FP64
                              // kernels skip walkers at or beyond it (escalated re-evaluations, whose
                              // psia is gathered from the evaluation that flagged them)
  double* R_stage = nullptr;  // host-API staging buffers
  double* out_stage = nullptr;
};

// Kernel launchers (mdet_kernels.cu, mdet_kernels_mixed.cu). Each returns the launch error.
cudaError_t launch_mo_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk,
                          const double* R, cudaStream_t st);
cudaError_t launch_mo_mixed(const DevProblem& P, const DevScratch& S, int64_t n_walk,
                            const double* R, cudaStream_t st);
// Dense BF16 GEMM on tcgen05 tensor cores with a fused epilogue (csrc/mdet_gemm_umma.cu).
// Element (r, k) of an operand is p[r * rs + k * ks] (FP32, or BF16 when bf16 != 0), zero for
// r >= rows or k >= cols; D[m][n] = sum_k A[m][k] B[n][k] over K = A.cols (= B.cols), the
// K range split over CTAs of k_per_cta (rounded up to 64) each.
struct GemmOperand {
  const void* p;
  int64_t rs, ks, rows, cols;
  int bf16;
};
enum GemmEpilogueKind { kEpiTanhBias = 0, kEpiBias = 1, kEpiDtanh = 2, kEpiAtomic = 3, kEpiStore = 4 };
// out[m * ldm + n * ldn] = tanh(D + bias[n]) | D + bias[n] | D (1 - h[m * ldh + n]^2) | += D (atomic) | D
struct GemmEpilogue {
  int kind;
  float* out;
  int64_t ldm, ldn;
  const float* bias;
  const float* h;
  int64_t ldh;
};
cudaError_t launch_gemm_bf16(const GemmOperand& A, const GemmOperand& B, int64_t k_per_cta, const GemmEpilogue& E,
                             cudaStream_t st);

// The mixed orbitals on the tcgen05 tensor cores (mdet_mo_umma.cu): supported for
// at most 112 AOs and 128 MOs; launch_mo_mixed takes it when mo_impl is 2.
bool mo_umma_supported(const DevProblem& P);
size_t mo_umma_smem_bytes(const DevProblem& P);
cudaError_t launch_mo_umma(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R, int n_sm,
                           cudaStream_t st);
cudaError_t launch_ref_tables(const DevProblem& P, const DevScratch& S, int64_t n_walk, bool mixed,
                              cudaStream_t st);
cudaError_t launch_ratios_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk,
                              cudaStream_t st);
cudaError_t launch_ratios_mixed(const DevProblem& P, const DevScratch& S, int64_t n_walk,
                                cudaStream_t st);
cudaError_t launch_zero_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk, cudaStream_t st);
// queue: two zeroed-per-launch work counters for a persistent contraction grid of
// spmm_blocks blocks, or of persistent_blocks when spmm_blocks is 0 (null or 0:
// one warp per work item). stamp (optional): four words, zeroed here, that receive the
// global-timer start (complemented) and end of the v and of the u launch.
cudaError_t launch_contract_f64(const DevProblem& P, const DevScratch& S, int64_t n_walk,
                                cudaStream_t st, unsigned long long* queue = nullptr, int persistent_blocks = 0,
                                unsigned long long* stamp = nullptr);
// A view of the scratch for walkers [off, off + n): walker-major arrays move by
// whole walkers, walker-minor arrays by columns (off must be a multiple of kWalkerPad).
DevScratch scratch_view(const DevScratch& S, const DevProblem& P, int64_t off);
// v = C r_dn over the row-major copy of C with Psi~ = r_up . v accumulated in
// psit, for walker-minor arrays of leading dimension ld (a multiple of 128).
cudaError_t launch_spmm_rows_f64(const DevProblem& P, const double* r_dn, const double* r_up, double* v,
                                 double* psit, int64_t ld, int64_t n_walk, cudaStream_t st);
// Compact outputs of an escalated re-evaluation (slot i holds the i-th listed walker).
struct EscOut {
  double* log_abs_psi;  // [cap]
  int8_t* sign;         // [cap]
  double* grad;         // [cap][N][3]
  double* lap;          // [cap][N]
  double* e_local;      // [cap]
  uint32_t* status;     // [cap]
};
// Lists the walkers whose status has MDET_WS_FALLBACK into list (count, then at
// most P.fallback_cap indices); further ones lose the bit and get MDET_WS_REF_ILLCOND.
cudaError_t launch_fb_list(const DevProblem& P, uint32_t* wstat, uint32_t* status, int64_t n_walk, int* list,
                           cudaStream_t st);
// Escalation of mixed-precision walkers: gather of the listed walkers' positions
// (and *live = their count), and scatter of their FP64 results back.
cudaError_t launch_esc_gather(const int* list, int cap, int n3, const double* R, double* Re, int* live,
                              const float* psia, float* psia_e, cudaStream_t st);
// Marks the gathered walkers for full LU (wstat[i] = MDET_WS_FALLBACK, i < *live).
cudaError_t launch_esc_mark(const int* live, uint32_t* wstat, int cap, cudaStream_t st);
cudaError_t launch_esc_scatter(const int* list, int cap, int N, const EscOut& e, uint32_t or_bits,
                               double* log_abs_psi, int8_t* sign, double* grad, double* lap, double* e_local,
                               uint32_t* status, uint32_t* wstat, cudaStream_t st);
cudaError_t launch_fallback(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                            double* log_abs_psi, int8_t* sign, double* grad, double* lap, double* e_local,
                            uint32_t* status, cudaStream_t st);
// Device index and uploaded problem of a context (null when it has none).
const DevProblem* ctx_problem(const mdet_ctx* ctx, int* device);
// Record the message that mdet_last_error returns for this context.
void ctx_set_error(mdet_ctx* ctx, const char* msg);
cudaError_t launch_selftest_df(int64_t n, const double* x, double* y_df, double* y_ref, double* prod_df,
                               cudaStream_t st);
cudaError_t launch_selftest_inv_r(int64_t n, const double* x, double* y_nr, double* y_ref, cudaStream_t st);
size_t final_smem_bytes(const DevProblem& P, bool mixed);
// wide: 512 threads per walker instead of 128 (FP64 only; lower latency for a few walkers)
cudaError_t launch_final(const DevProblem& P, const DevScratch& S, int64_t n_walk, const double* R,
                         double* log_abs_psi, int8_t* sign, double* grad, double* lap, double* e_local,
                         uint32_t* status, bool mixed, cudaStream_t st, bool wide = false);

// ---- expansion preprocessing on the GPU (mdet_preprocess.cu), Sec. 2.1 ----
// Results of the O(N_det) steps for one spin: the distinct determinants in the
// order of the key of Eq. 3 ([nu][n_int]) and the position of the reference.
struct PreSpin {
  std::vector<uint64_t> udets;
  int64_t iref = 0;
};
struct PreDevice;  // device buffers kept between the two calls below
// The C arrays in both orders and their segment pointers, as built on the host.
struct PreC {
  std::vector<int32_t> csc_row, csc_col, csr_row, csr_col, csr_ptr, csc_ptr;
  std::vector<double> csc_val, csr_val;
};
// Validates both spin lists (popcount, bits beyond n_mo) and the coefficients
// (finite), sorts each list by the key of Eq. 3 with ties broken by the words
// from the last to the first (stable), removes duplicates, maps every product to
// its distinct determinant and finds the reference product (largest |c|, first
// on ties). Inputs are device arrays. Returns MDET_OK, MDET_E_INPUT (msg says
// which product) or MDET_E_CUDA.
mdet_status pre_distinct(PreDevice** h, int64_t n, int n_int, const uint64_t* det_up, const uint64_t* det_dn,
                         const double* coef, int n_up, int n_dn, int n_mo, cudaStream_t st, PreSpin out[2],
                         std::string* msg);
// From ctx_of (distinct index -> context index) of both spins: C sorted by
// (column, row) and by (row, column), the duplicate-pair check and the segment
// pointers, copied to the host.
mdet_status pre_build_c(PreDevice* h, const std::vector<int32_t> ctx_of[2], int64_t nup, int64_t ndn,
                        cudaStream_t st, PreC* out, std::string* msg);
void pre_free(PreDevice* h);

// ---- the sequential Sherman-Morrison chain (mdet_smchain.cu), Sec. 2.2 ----
constexpr int kSmMaxSub = 8;  // substitutions between consecutive determinants (2 * MDET_MAX_EXC)
// One determinant of the chain, in the order of the key of Eq. 3: its context
// index, the substitutions hole[s] -> part[s] (MO indices, ascending) that turn
// the previous determinant of the chain into it (n_sub > kSmMaxSub: recompute it
// from scratch), and its occupied MOs in ascending order.
struct SmStep {
  int32_t ctx;
  uint8_t n_sub;
  uint8_t hole[kSmMaxSub];
  uint8_t part[kSmMaxSub];
  uint8_t occ[kMaxSpin];
};
size_t sm_chain_smem_bytes(int n);
cudaError_t launch_sm_chain(const DevProblem& P, const DevScratch& S, int spin, const SmStep* steps, int n_steps,
                            int64_t n_walk, double* r, int64_t ld_r, int32_t* n_inv, int32_t* n_subst,
                            cudaStream_t st);

}  // namespace mdet

// Host side of the C ABI: context, validation, the preprocessing of Sec. 2.1,
// device residency and the launch sequence of one evaluation.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mdet_internal.h"

using namespace mdet;

struct mdet_ctx {
  int device = MDET_NO_DEVICE;
  int precision = MDET_PRECISION_FP64;
  std::string err;
  // system
  bool has_system = false, has_orbitals = false, has_ci = false;
  int n_up = 0, n_dn = 0, n_nuc = 0;
  std::vector<double> Z, nuc_xyz;
  // orbitals
  int n_shell = 0, n_ao = 0, n_mo = 0, n_prim = 0;
  std::vector<int> shell_l, shell_center, shell_nprim, shell_prim0, shell_ao0;
  std::vector<double> alpha, coef, mo_colmajor;
  // expansion after preprocessing
  int64_t n_det = 0;
  int n_int = 0;
  std::vector<uint64_t> dets[2];   // distinct determinants in context order [n][n_int]
  std::vector<int> degree[2];
  std::vector<Exc> exc[2];
  std::vector<int> ref_occ[2];
  std::vector<int32_t> coo_row, coo_col;  // column-major order (Sec. 2.1)
  std::vector<double> coo_val;
  std::vector<int32_t> csr_row, csr_col;  // row-major order
  std::vector<double> csr_val;
  // device residency
  std::vector<void*> dev_problem_allocs;
  // work items of the contraction per item size (built on first use outside any stream
  // capture and kept with the problem, so that captured graphs keep valid pointers)
  struct ItemSet {
    int chunk;
    const int2* d[2];
    int n[2];
    const uint8_t* split;
  };
  std::vector<ItemSet> item_sets;
  DevProblem P{};
  DevScratch S{};
  // escalation of mixed-precision walkers (FP64 re-evaluation of the flagged ones):
  // scratch for fallback_cap walkers, their positions, compact outputs and live count
  DevScratch E{};
  EscOut eo{};
  double* e_R = nullptr;
  int* e_live = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  int64_t last_walk = 0;
  // walker chunks (mixed precision), software-pipelined over two streams: the
  // FP32-pipe stages of the chunks run in order on fstream, the FP64 contractions on
  // the higher-priority stream cstream, so one chunk's contraction overlaps the
  // orbitals, tables and ratios of the next chunk and the epilogue of the previous one
  static constexpr int kMaxChunks = MDET_MAX_CHUNKS;
  int n_chunks_cfg = 0;  // 0: automatic
  double fallback_tol = 0.0;  // set from the precision in mdet_create
  int fallback_cap = 256;  // set from the precision in mdet_create
  int escalate = MDET_ESCALATE_AUTO;
  bool in_batch = false;  // set while a batch enqueues this context's evaluation
  std::vector<int32_t> csr_ptr, csc_ptr;
  int spmm_chunk = 512;  // tile shapes (mdet_set_tuning / mdet_autotune)
  int spmm_blocks = 0;
  int mo_impl = 2;  // mixed orbitals: exact digit products on the tcgen05 tensor cores
  int mo_ec = 4;
  int contract_impl = 0;  // FP64 contraction (the double-float one is an option of the mixed path)
  mdet_tuning last_tune{};
  cudaStream_t fstream = nullptr, cstream = nullptr;
  int n_sm = 0;
  cudaEvent_t fork = nullptr, joined = nullptr, contracted[kMaxChunks] = {}, prepared[kMaxChunks] = {};
  // stage timing
  int profiling = 0;  // mode of mdet_set_profiling
  bool have_profile = false;
  bool have_timeline = false;
  int prof_chunks = 0;
  int last_kernels = 0;  // kernels the last evaluation launched
  // per chunk: the start and end of every stage (stages of one chunk may run on
  // different streams, after waits)
  static constexpr int kEvPerChunk = 2 * MDET_N_STAGES;
  cudaEvent_t ev[kMaxChunks][kEvPerChunk] = {};
  // timeline: the start of the evaluation, the refinement's start and end, the end of the evaluation
  cudaEvent_t ev_origin = nullptr, ev_refine[2] = {}, ev_done = nullptr;
};

namespace {

// contraction work items of escalated re-evaluations (a few hundred walkers): short, so that
// the FP64 chains stay short (128 nonzeros measured 0.4 ms per step faster than 64, whose
// items all add Psi~ of the same few walkers, and than 256)
constexpr int kEscalationChunk = 128;

// words of S.queue per walker chunk: the work counters of its two persistent contractions, then
// the global-timer stamps (start complemented, end) of each
constexpr int kQueueWords = 6;

// weights of the first, each middle and the last walker chunk of the pipelined evaluation. The
// first chunk's orbitals and tables run before any contraction, and the last chunk's epilogue
// after all of them, so both are kept short; but the epilogue of the chunk before the last runs
// beside the last contraction, which must stay long enough to hide it. At 8,192 walkers (32
// tiles), 750k products, 6:21:5 tiles measured 28.62 ms per step against 28.73 for 6:19:7,
// 29.1-29.3 for 6:22:4 and 5:22:5, and 29.6-29.8 for four chunks.
constexpr int kFirstWeight = 6, kMidWeight = 21, kLastWeight = 5;

size_t final_smem_bytes_host(int n_up, int n_dn, int n_mo, bool mixed) {
  DevProblem P{};
  P.n_up = n_up;
  P.n_dn = n_dn;
  P.n_elec = n_up + n_dn;
  P.n_mo = n_mo;
  return final_smem_bytes(P, mixed);
}

mdet_status fail(mdet_ctx* c, mdet_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, MDET_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

int popcount_words(const uint64_t* w, int n_int) {
  int c = 0;
  for (int q = 0; q < n_int; q++) c += __builtin_popcountll(w[q]);
  return c;
}

uint64_t omega_key(const uint64_t* w, int n_int) {
  // Eq. 3: xor of the words. The -2^63 shift of the paper only emulates an
  // unsigned comparison with signed integers; here the key is compared unsigned.
  uint64_t k = 0;
  for (int q = 0; q < n_int; q++) k ^= w[q];
  return k;
}

// Compare two determinants by (omega, words from the last to the first), unsigned.
int cmp_det(const uint64_t* a, const uint64_t* b, int n_int) {
  uint64_t ka = omega_key(a, n_int), kb = omega_key(b, n_int);
  if (ka != kb) return ka < kb ? -1 : 1;
  for (int q = n_int - 1; q >= 0; q--)
    if (a[q] != b[q]) return a[q] < b[q] ? -1 : 1;
  return 0;
}

// LSD radix sort of indices by a 64-bit key, 8 bits per pass; stable.
void radix_sort_u64(std::vector<int64_t>& idx, const std::vector<uint64_t>& key) {
  const size_t n = idx.size();
  std::vector<int64_t> tmp(n);
  for (int pass = 0; pass < 8; pass++) {
    const int sh = 8 * pass;
    size_t cnt[257] = {0};
    bool all_same = true;
    uint64_t first = n ? (key[idx[0]] >> sh) & 0xff : 0;
    for (size_t i = 0; i < n; i++) {
      uint64_t d = (key[idx[i]] >> sh) & 0xff;
      cnt[d + 1]++;
      all_same &= (d == first);
    }
    if (all_same) continue;
    for (int d = 0; d < 256; d++) cnt[d + 1] += cnt[d];
    for (size_t i = 0; i < n; i++) tmp[cnt[(key[idx[i]] >> sh) & 0xff]++] = idx[i];
    idx.swap(tmp);
  }
}

// Permutation sorting determinants by the key of Eq. 3 (radix sort), ties
// broken by the full words (only groups of equal keys are compared).
std::vector<int64_t> omega_order(int64_t n, int n_int, const uint64_t* dets) {
  std::vector<uint64_t> key(n);
  for (int64_t k = 0; k < n; k++) key[k] = omega_key(dets + k * n_int, n_int);
  std::vector<int64_t> idx(n);
  for (int64_t k = 0; k < n; k++) idx[k] = k;
  radix_sort_u64(idx, key);
  if (n_int > 1) {
    int64_t a = 0;
    while (a < n) {
      int64_t b = a + 1;
      while (b < n && key[idx[b]] == key[idx[a]]) b++;
      if (b - a > 1)
        std::stable_sort(idx.begin() + a, idx.begin() + b, [&](int64_t x, int64_t y) {
          return cmp_det(dets + x * n_int, dets + y * n_int, n_int) < 0;
        });
      a = b;
    }
  }
  return idx;
}

std::vector<int> decode_occ(const uint64_t* w, int n_int) {
  std::vector<int> occ;
  for (int q = 0; q < n_int; q++)
    for (int b = 0; b < 64; b++)
      if ((w[q] >> b) & 1ULL) occ.push_back(64 * q + b);
  return occ;
}

// Sign of the permutation that sorts `cols` ascending (inversion parity).
int sort_parity(const std::vector<int>& cols) {
  int inv = 0;
  for (size_t i = 0; i < cols.size(); i++)
    for (size_t j = i + 1; j < cols.size(); j++)
      if (cols[i] > cols[j]) inv++;
  return (inv & 1) ? -1 : 1;
}

template <class T>
mdet_status upload(mdet_ctx* c, const std::vector<T>& v, const T** out) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(sizeof(T), v.size() * sizeof(T));
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(c, MDET_E_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  c->dev_problem_allocs.push_back(p);
  if (!v.empty()) {
    e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(c, MDET_E_CUDA, "cudaMemcpy failed: %s", cudaGetErrorString(e));
  }
  *out = static_cast<const T*>(p);
  return MDET_OK;
}

void free_problem(mdet_ctx* c) {
  for (void* p : c->dev_problem_allocs) cudaFree(p);
  c->dev_problem_allocs.clear();
  c->item_sets.clear();
  c->P = DevProblem{};
}

// Work items of the contraction for item size `chunk`: consecutive whole segments (rows of the
// row-major copy of C, columns of the column-major one) packed while they hold at most `chunk`
// nonzeros, and segments longer than `chunk` cut into pieces of at most `chunk` nonzeros, so
// that every item costs about the same. A whole segment belongs to one item, whose warp stores
// its (segment, walker) sums; the pieces of a cut segment add theirs atomically (flagged by a
// negative end), into entries the ratio kernel has cleared (`split`).
mdet_status ensure_items(mdet_ctx* c, int chunk) {
  for (const auto& s : c->item_sets)
    if (s.chunk == chunk) return MDET_OK;
  mdet_ctx::ItemSet set{};
  set.chunk = chunk;
  std::vector<uint8_t> split;
  for (int o = 0; o < 2; o++) {
    const std::vector<int32_t>& ptr = o ? c->csc_ptr : c->csr_ptr;
    const int64_t nseg = (int64_t)ptr.size() - 1;
    std::vector<int2> it;
    int32_t b = nseg > 0 ? ptr[0] : 0;  // start of the item being packed
    for (int64_t q = 0; q < nseg; q++) {
      const int32_t s0 = ptr[q], s1 = ptr[q + 1];
      if (s1 - s0 > chunk) {  // a long segment: close the open item, then cut this one
        if (s0 > b) it.push_back(make_int2(b, s0));
        for (int32_t p = s0; p < s1; p += chunk) it.push_back(make_int2(p, (int32_t)(std::min(p + chunk, s1) | 0x80000000u)));
        split.push_back(1);
        b = s1;
        continue;
      }
      split.push_back(0);
      if (s0 > b && s1 - b > chunk) {
        it.push_back(make_int2(b, s0));
        b = s0;
      }
    }
    if (nseg > 0 && ptr[nseg] > b) it.push_back(make_int2(b, ptr[nseg]));
    mdet_status s = upload(c, it, &set.d[o]);
    if (s != MDET_OK) return s;
    set.n[o] = (int)it.size();
  }
  mdet_status s = upload(c, split, &set.split);
  if (s != MDET_OK) return s;
  c->item_sets.push_back(set);
  return MDET_OK;
}

// The problem with its contraction items switched to item size `chunk` (which must have been built).
bool use_items(const mdet_ctx* c, DevProblem& P, int chunk) {
  for (const auto& s : c->item_sets)
    if (s.chunk == chunk) {
      P.spmm_chunk = chunk;
      for (int o = 0; o < 2; o++) {
        P.items[o] = s.d[o];
        P.n_items[o] = s.n[o];
      }
      P.split = s.split;
      return true;
    }
  return false;
}

void free_arrays(DevScratch& S) {
  void* ptrs[] = {S.phi, S.Ainv, S.ld0, S.sg0, S.g, S.kap, S.est, S.T, S.Tdf, S.r, S.rdf, S.vu, S.psit, S.psia, S.wstat,
                  S.fb, S.fb_list, S.fb_acc, S.queue, S.R_stage, S.out_stage};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  S = DevScratch{};
}

void free_scratch(mdet_ctx* c) {
  free_arrays(c->S);
  free_arrays(c->E);
  void* ptrs[] = {c->e_R, c->e_live, c->eo.log_abs_psi, c->eo.sign, c->eo.grad, c->eo.lap, c->eo.e_local,
                  c->eo.status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->e_R = nullptr;
  c->e_live = nullptr;
  c->eo = EscOut{};
}

// Host step shared by both preprocessing paths. From the distinct determinants
// of one spin in omega order (udets [nu][n_int]) and the omega index of the
// reference: excitation degrees relative to the reference, the context order
// (reference first, then by degree, omega order within a degree), the
// excitation records with their phases, and ctx_of[omega index] = context index.
mdet_status spin_tables(mdet_ctx* c, int sp, int n_int, const std::vector<uint64_t>& udets, int64_t iref,
                        std::vector<int32_t>& ctx_of) {
  const int64_t nu = (int64_t)(udets.size() / n_int);
  const uint64_t* ref = udets.data() + iref * n_int;
  std::vector<int> deg(nu);
  for (int64_t i = 0; i < nu; i++) {
    const uint64_t* w = udets.data() + i * n_int;
    int h = 0;
    for (int q = 0; q < n_int; q++) h += __builtin_popcountll(ref[q] & ~w[q]);
    deg[i] = h;
    if (h > kMaxExc)
      return fail(c, MDET_E_INPUT, "spin %d determinant is a degree-%d excitation of the reference (max %d)", sp, h,
                  kMaxExc);
  }
  std::vector<int64_t> order;
  order.reserve(nu);
  order.push_back(iref);
  for (int d = 1; d <= kMaxExc; d++)
    for (int64_t i = 0; i < nu; i++)
      if (deg[i] == d && i != iref) order.push_back(i);
  ctx_of.assign(nu, 0);
  for (int64_t t = 0; t < nu; t++) ctx_of[order[t]] = (int32_t)t;
  std::vector<int> rocc = decode_occ(ref, n_int);
  c->ref_occ[sp] = rocc;
  c->dets[sp].assign((size_t)nu * n_int, 0);
  c->degree[sp].assign(nu, 0);
  c->exc[sp].assign(nu, Exc{});
  for (int64_t t = 0; t < nu; t++) {
    const uint64_t* w = udets.data() + order[t] * n_int;
    std::copy(w, w + n_int, c->dets[sp].begin() + t * n_int);
    Exc e{};
    std::vector<int> cols = rocc;  // reference columns with holes replaced by particles
    int k = 0, kp = 0;
    for (size_t a = 0; a < rocc.size(); a++) {
      int m = rocc[a];
      if (!((w[m / 64] >> (m % 64)) & 1ULL)) e.h[k++] = (uint8_t)a;
    }
    for (int q = 0; q < n_int; q++) {
      uint64_t part = w[q] & ~ref[q];
      while (part) {
        int b = __builtin_ctzll(part);
        part &= part - 1;
        e.p[kp++] = (uint8_t)(64 * q + b);
      }
    }
    if (k != kp) return fail(c, MDET_E_INPUT, "internal: hole/particle count mismatch");
    for (int a = 0; a < k; a++) cols[e.h[a]] = e.p[a];
    e.k = (uint8_t)k;
    e.eps = (int8_t)sort_parity(cols);
    c->exc[sp][t] = e;
    c->degree[sp][t] = k;
  }
  return MDET_OK;
}

// Upload everything the kernels read (called once the expansion is complete).
mdet_status upload_problem(mdet_ctx* c) {
  if (c->device < 0) return MDET_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  free_problem(c);
  DevProblem& P = c->P;
  P.n_up = c->n_up; P.n_dn = c->n_dn; P.n_elec = c->n_up + c->n_dn; P.n_nuc = c->n_nuc;
  P.n_shell = c->n_shell; P.n_ao = c->n_ao; P.n_mo = c->n_mo; P.n_prim = c->n_prim;
  P.n_det_sp[0] = (int)c->exc[0].size();
  P.n_det_sp[1] = (int)c->exc[1].size();
  P.nnz = c->n_det;
  P.spmm_chunk = c->spmm_chunk;
  P.spmm_blocks = c->spmm_blocks;
  P.mo_ec = c->mo_ec;
  P.mo_impl = c->mo_impl;
  P.n_sm = c->n_sm;
  P.phi_df = c->precision == MDET_PRECISION_MIXED;
  P.contract_impl = c->contract_impl;
  P.fallback_tol = c->fallback_tol;
  P.fallback_cap = c->fallback_cap;
  mdet_status s;
#define UP(vec, dst) if ((s = upload(c, vec, &dst)) != MDET_OK) return s
  UP(c->Z, P.Z);
  UP(c->nuc_xyz, P.nuc_xyz);
  UP(c->shell_l, P.shell_l);
  UP(c->shell_center, P.shell_center);
  UP(c->shell_nprim, P.shell_nprim);
  UP(c->shell_prim0, P.shell_prim0);
  UP(c->shell_ao0, P.shell_ao0);
  UP(c->alpha, P.alpha);
  UP(c->coef, P.coef);
  std::vector<double> B((size_t)c->n_ao * c->n_mo);
  std::vector<float> Bh(B.size()), Bl(B.size());
  for (int mu = 0; mu < c->n_ao; mu++)
    for (int m = 0; m < c->n_mo; m++) {
      const size_t q = (size_t)mu * c->n_mo + m;
      B[q] = c->mo_colmajor[mu + (size_t)c->n_ao * m];
      Bh[q] = (float)B[q];                     // double-float split B = Bh + Bl
      Bl[q] = (float)(B[q] - (double)Bh[q]);
    }
  UP(B, P.B);
  UP(Bh, P.B_hi);
  UP(Bl, P.B_lo);
  // digits of B for the tensor-core orbital product: column m as 2^f_m sum_j g_j 2^(-8 j),
  // j = 1..7, integer digits (|g_1| <= 256, |g_j| <= 128) stored as BF16, [j][m][k] K-contiguous
  {
    const int kDigits = 7;
    P.tc_kp = (c->n_ao + 15) / 16 * 16;
    P.tc_mp = (c->n_mo + 7) / 8 * 8;
    const int half = P.tc_kp / 2;  // shared row stride in 4-byte words must be 4 mod 8 (conflict-free A fragments)
    P.tc_sx = P.tc_kp + 2 * ((4 - half % 8 + 8) % 8);
    std::vector<uint16_t> dig((size_t)kDigits * P.tc_mp * P.tc_kp, 0);
    std::vector<int> fexp(c->n_mo, 0);
    for (int m = 0; m < c->n_mo; m++) {
      double mx = 0.0;
      for (int mu = 0; mu < c->n_ao; mu++) mx = std::max(mx, std::fabs(B[(size_t)mu * c->n_mo + m]));
      const int f = mx > 0.0 ? std::ilogb(mx) + 1 : 0;
      fexp[m] = f;
      for (int mu = 0; mu < c->n_ao; mu++) {
        double v = std::ldexp(B[(size_t)mu * c->n_mo + m], -f);
        for (int j = 0; j < kDigits; j++) {
          v *= 256.0;
          const double d = std::nearbyint(v);
          v -= d;
          const float fd = (float)d;
          uint32_t bits;
          std::memcpy(&bits, &fd, 4);
          dig[((size_t)j * P.tc_mp + m) * P.tc_kp + mu] = (uint16_t)(bits >> 16);
        }
      }
    }
    UP(dig, P.B_dig);
    UP(fexp, P.B_exp);
  }
  auto split = [](const std::vector<double>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); i++) {
      const float h = (float)v[i];
      o[i] = make_float2(h, (float)(v[i] - (double)h));
    }
    return o;
  };
  std::vector<float2> a_df = split(c->alpha), c_df = split(c->coef), x_df = split(c->nuc_xyz);
  UP(a_df, P.alpha_df);
  UP(c_df, P.coef_df);
  UP(x_df, P.nuc_df);
  std::vector<int> occ(2 * kMaxSpin, 0);
  for (int sp = 0; sp < 2; sp++)
    for (size_t a = 0; a < c->ref_occ[sp].size(); a++) occ[sp * kMaxSpin + a] = c->ref_occ[sp][a];
  UP(occ, P.ref_occ);
  UP(c->exc[0], P.exc[0]);
  UP(c->exc[1], P.exc[1]);
  for (int sp = 0; sp < 2; sp++) {  // the context orders each spin's list by degree
    int cnt[kMaxExc + 1] = {};
    for (int d : c->degree[sp]) cnt[d]++;
    P.deg_start[sp][0] = 0;
    for (int d = 0; d <= kMaxExc; d++) P.deg_start[sp][d + 1] = P.deg_start[sp][d] + cnt[d];
  }
  UP(c->csr_row, P.csr_row);
  UP(c->csr_col, P.csr_col);
  UP(c->csr_val, P.csr_val);
  UP(c->coo_col, P.csc_col);
  UP(c->coo_row, P.csc_row);
  UP(c->coo_val, P.csc_val);
  UP(c->csr_ptr, P.csr_ptr);
  UP(c->csc_ptr, P.csc_ptr);
  {  // C as double-float pairs for the optional double-float contraction
    std::vector<float2> a = split(c->csr_val), b = split(c->coo_val);
    UP(a, P.csr_val_df);
    UP(b, P.csc_val_df);
  }
  // contraction work items for the tuned size and for the short items of escalated re-evaluations
  if ((s = ensure_items(c, c->spmm_chunk)) != MDET_OK || (s = ensure_items(c, kEscalationChunk)) != MDET_OK) return s;
  use_items(c, P, c->spmm_chunk);
  // the sequential chain of Sec. 2.2: distinct determinants in the order of the key of Eq. 3,
  // each with the substitutions from its predecessor (holes and particles ascending, paired in order)
  for (int sp = 0; sp < 2; sp++) {
    const int64_t nu = (int64_t)c->exc[sp].size();
    std::vector<int64_t> ord = omega_order(nu, c->n_int, c->dets[sp].data());
    std::vector<SmStep> steps(nu);
    std::vector<int> prev;
    for (int64_t t = 0; t < nu; t++) {
      SmStep& st = steps[t];
      st = SmStep{};
      st.ctx = (int32_t)ord[t];
      std::vector<int> occ = decode_occ(c->dets[sp].data() + ord[t] * c->n_int, c->n_int);
      for (size_t a = 0; a < occ.size(); a++) st.occ[a] = (uint8_t)occ[a];
      std::vector<int> holes, parts;
      for (int m : prev)
        if (!std::binary_search(occ.begin(), occ.end(), m)) holes.push_back(m);
      for (int m : occ)
        if (!std::binary_search(prev.begin(), prev.end(), m)) parts.push_back(m);
      if (t == 0 || (int)holes.size() > kSmMaxSub) {
        st.n_sub = t == 0 ? 0 : (uint8_t)(kSmMaxSub + 1);
      } else {
        st.n_sub = (uint8_t)holes.size();
        for (size_t q = 0; q < holes.size(); q++) {
          st.hole[q] = (uint8_t)holes[q];
          st.part[q] = (uint8_t)parts[q];
        }
      }
      prev = occ;
    }
    UP(steps, P.sm_steps[sp]);
    P.sm_n[sp] = (int)nu;
  }
#undef UP
  free_scratch(c);  // sizes depend on the problem
  return MDET_OK;
}

template <class T>
mdet_status dalloc(mdet_ctx* c, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, MDET_E_OOM, "cudaMalloc(%zu bytes) for scratch failed: %s", bytes, cudaGetErrorString(e));
  }
  return MDET_OK;
}

// The per-walker arrays of one evaluation of W walkers: FP64 tables and, with
// df_tables / df_ratios, their double-float copies (mixed path). Padded walker
// columns of the walker-minor tables hold finite values.
mdet_status alloc_eval_arrays(mdet_ctx* c, DevScratch& S, int64_t W, bool df_tables, bool df_ratios) {
  const DevProblem& P = c->P;
  const int64_t wp = (W + kWalkerPad - 1) / kWalkerPad * kWalkerPad;
  const int64_t N = P.n_elec, M = P.n_mo;
  const int64_t ndt = (int64_t)P.n_det_sp[0] + P.n_det_sp[1];
  mdet_status s;
  if ((s = dalloc(c, &S.phi, (size_t)W * 5 * N * M))) return s;
  if ((s = dalloc(c, &S.Ainv, (size_t)W * (P.n_up * P.n_up + P.n_dn * P.n_dn)))) return s;
  if ((s = dalloc(c, &S.ld0, (size_t)W * 2))) return s;
  if ((s = dalloc(c, &S.sg0, (size_t)W * 2))) return s;
  if ((s = dalloc(c, &S.g, (size_t)W * N * 4))) return s;
  if ((s = dalloc(c, &S.kap, (size_t)W * 2))) return s;
  if ((s = dalloc(c, &S.est, (size_t)W * 2))) return s;
  if ((s = dalloc(c, &S.T, (size_t)N * M * wp))) return s;
  CUDA_TRY(c, cudaMemset(S.T, 0, sizeof(double) * N * M * wp));
  if (df_tables) {
    if ((s = dalloc(c, &S.Tdf, (size_t)N * M * wp))) return s;
    CUDA_TRY(c, cudaMemset(S.Tdf, 0, sizeof(float2) * N * M * wp));
  }
  if ((s = dalloc(c, &S.r, (size_t)ndt * wp))) return s;
  CUDA_TRY(c, cudaMemset(S.r, 0, sizeof(double) * ndt * wp));
  if (df_ratios) {
    if ((s = dalloc(c, &S.rdf, (size_t)ndt * wp))) return s;
    CUDA_TRY(c, cudaMemset(S.rdf, 0, sizeof(float2) * ndt * wp));
  }
  if ((s = dalloc(c, &S.vu, (size_t)ndt * wp))) return s;  // walker-major [wp][ndt]
  if ((s = dalloc(c, &S.psit, (size_t)wp))) return s;
  if ((s = dalloc(c, &S.psia, (size_t)wp))) return s;
  if ((s = dalloc(c, &S.wstat, (size_t)W))) return s;
  S.cap_walk = W;
  S.wp = wp;
  return MDET_OK;
}

// The full-LU fallback's scratch for P.fallback_cap walkers.
mdet_status alloc_fallback(mdet_ctx* c, DevScratch& S) {
  const DevProblem& P = c->P;
  const int64_t ndt = (int64_t)P.n_det_sp[0] + P.n_det_sp[1];
  const int64_t nmax = std::max(P.n_up, P.n_dn);
  mdet_status s;
  if ((s = dalloc(c, &S.fb, (size_t)P.fallback_cap * ndt * (3 + 4 * nmax)))) return s;
  if ((s = dalloc(c, &S.fb_list, (size_t)P.fallback_cap + 1))) return s;
  return dalloc(c, &S.fb_acc, (size_t)P.fallback_cap * (3 + 8 * MDET_FALLBACK_MAX_SPIN));
}

// Whether mixed precision re-evaluates its flagged walkers by the FP64 ratio
// table before the full-LU path (MDET_ESCALATE_AUTO: when it pays). The
// escalation costs a fixed latency (a dozen dependent launches over up to a few
// hundred walkers) and a few microseconds per walker; full LU costs about 5-7 ns
// per (distinct determinant x n^3) and walker, n the larger spin count: 30 us for
// 6,030 determinants of 9 electrons, 320 us for the largest 17-electron
// expansions. Measured with ~100 flagged walkers, the two tie at about 1.3e6
// units per walker (1,800 determinants of 9 electrons) and escalation saves
// 1.2 ms at 4.4e6 (6,030), so it is taken above 1e6; in a batch the other
// expansions' kernels hide its latency, and it is always taken.
bool escalation_on(const mdet_ctx* c) {
  if (c->escalate != MDET_ESCALATE_AUTO) return c->escalate == MDET_ESCALATE_ALWAYS;
  if (c->in_batch) return true;
  const double ndt = (double)c->P.n_det_sp[0] + c->P.n_det_sp[1];
  const double n = std::max(c->P.n_up, c->P.n_dn);
  return ndt * n * n * n > 1e6;
}

mdet_status ensure_scratch(mdet_ctx* c, int64_t n_walk) {
  DevScratch& S = c->S;
  if (n_walk <= S.cap_walk) return MDET_OK;
  free_scratch(c);
  const DevProblem& P = c->P;
  const bool mixed = c->precision == MDET_PRECISION_MIXED;
  mdet_status s;
  if ((s = alloc_eval_arrays(c, S, n_walk, mixed, mixed && c->contract_impl == 1))) return s;
  if ((s = dalloc(c, &S.queue, (size_t)kQueueWords * mdet_ctx::kMaxChunks))) return s;
  if (P.fallback_tol > 0.0 && P.n_up <= MDET_FALLBACK_MAX_SPIN) {
    if (!mixed) return alloc_fallback(c, S);
    // mixed: the list of flagged walkers, then an FP64 re-evaluation of at most fallback_cap
    // of them (orbitals, optionally the ratio table, then full LU) on a scratch of their own
    const int cap = P.fallback_cap;
    const int64_t N = P.n_elec;
    if ((s = dalloc(c, &S.fb_list, (size_t)cap + 1))) return s;
    DevScratch& E = c->E;
    // FP64 arrays only; with its live count set, E always takes the narrow FP64 contraction, which
    // keeps the magnitude sums gathered from the flagging evaluation
    if ((s = alloc_eval_arrays(c, E, cap, false, false)) || (s = alloc_fallback(c, E))) return s;
    if ((s = dalloc(c, &c->e_R, (size_t)cap * N * 3)) || (s = dalloc(c, &c->e_live, 1)) ||
        (s = dalloc(c, &c->eo.log_abs_psi, (size_t)cap)) || (s = dalloc(c, &c->eo.sign, (size_t)cap)) ||
        (s = dalloc(c, &c->eo.grad, (size_t)cap * N * 3)) || (s = dalloc(c, &c->eo.lap, (size_t)cap * N)) ||
        (s = dalloc(c, &c->eo.e_local, (size_t)cap)) || (s = dalloc(c, &c->eo.status, (size_t)cap)))
      return s;
    E.live = c->e_live;
  }
  return MDET_OK;
}

// Mixed precision: walkers whose estimate exceeds the tolerance (at most
// fallback_cap) are gathered and their orbitals evaluated in FP64. With `table`
// they are evaluated again by the FP64 ratio-table kernels, whose estimate is
// 2^6 smaller, and those still above the tolerance go through the full-LU path;
// without it, all of them do. The results replace the mixed ones. All on stream
// st, without host waits.
mdet_status refine(mdet_ctx* c, bool table, int64_t n_walk, const double* R, double* log_abs_psi, int8_t* sign,
                   double* grad, double* lap, double* e_local, uint32_t* status, cudaStream_t st) {
  const DevProblem& P = c->P;
  DevScratch& S = c->S;
  DevScratch& E = c->E;
  const int cap = P.fallback_cap;
  const int N = P.n_elec;
  CUDA_TRY(c, launch_fb_list(P, S.wstat, status, n_walk, S.fb_list, st));
  CUDA_TRY(c, cudaMemsetAsync(E.wstat, 0, sizeof(uint32_t) * cap, st));
  CUDA_TRY(c, launch_esc_gather(S.fb_list, cap, 3 * N, R, c->e_R, c->e_live, S.psia, E.psia, st));
  // one electron per FP64 orbital block: the grid of a few hundred walkers then spreads evenly
  // over the SMs (28.51 ms per step at 8,192 walkers, 750k products, against 28.60 with 6)
  DevProblem Pe = P;
  Pe.mo_ec = 1;
  if (!use_items(c, Pe, kEscalationChunk)) return fail(c, MDET_E_STATE, "internal: escalation items missing");
  CUDA_TRY(c, launch_mo_f64(Pe, E, cap, c->e_R, st));
  const EscOut& o = c->eo;
  if (!table) {
    CUDA_TRY(c, launch_esc_mark(c->e_live, E.wstat, cap, st));
    CUDA_TRY(c, launch_fallback(P, E, cap, c->e_R, o.log_abs_psi, o.sign, o.grad, o.lap, o.e_local, o.status, st));
    CUDA_TRY(c, launch_esc_scatter(S.fb_list, cap, N, o, 0u, log_abs_psi, sign, grad, lap, e_local, status, S.wstat,
                                   st));
    return MDET_OK;
  }
  CUDA_TRY(c, launch_ref_tables(P, E, cap, false, st));
  CUDA_TRY(c, launch_ratios_f64(Pe, E, cap, st));  // clears the cut segments of Pe's items
  // few walkers: short work items keep the contraction's chains short, and the epilogue
  // spreads each walker's determinants over 512 threads
  Pe.spmm_blocks = 0;
  CUDA_TRY(c, launch_contract_f64(Pe, E, cap, st));
  CUDA_TRY(c, launch_final(P, E, cap, c->e_R, o.log_abs_psi, o.sign, o.grad, o.lap, o.e_local, o.status, false, st,
                           true));
  CUDA_TRY(c, launch_fallback(P, E, cap, c->e_R, o.log_abs_psi, o.sign, o.grad, o.lap, o.e_local, o.status, st));
  CUDA_TRY(c, launch_esc_scatter(S.fb_list, cap, N, o, MDET_WS_ESCALATED, log_abs_psi, sign, grad, lap, e_local,
                                 status, S.wstat, st));
  return MDET_OK;
}

// Walker chunks of a mixed-precision evaluation when none are configured: three
// when the FP64 contraction is long enough to hide the FP32-pipe stages of the
// other chunks (at least 100,000 products and 4 walker tiles per chunk), else one.
int auto_chunks(const mdet_ctx* c, int64_t n_walk) {
  const int64_t tiles = (n_walk + kWalkerPad - 1) / kWalkerPad;
  return (c->precision == MDET_PRECISION_MIXED && c->contract_impl == 0 && c->P.nnz >= 100000 && tiles >= 12) ? 3
                                                                                                                : 1;
}

}  // namespace

namespace mdet {
const DevProblem* ctx_problem(const mdet_ctx* c, int* device) {
  if (!c || c->device < 0 || !c->has_ci) return nullptr;
  if (device) *device = c->device;
  return &c->P;
}
void ctx_set_error(mdet_ctx* c, const char* msg) {
  if (c) c->err = msg;
}
}  // namespace mdet

extern "C" {

const char* mdet_status_string(mdet_status s) {
  switch (s) {
    case MDET_OK: return "ok";
    case MDET_E_ARG: return "invalid argument";
    case MDET_E_STATE: return "call order violated";
    case MDET_E_OOM: return "out of memory";
    case MDET_E_CUDA: return "CUDA error";
    case MDET_E_INPUT: return "malformed expansion";
    case MDET_E_TIMEOUT: return "device wait timed out";
    case MDET_E_NODEVICE: return "context has no device";
  }
  return "unknown status";
}

const char* mdet_last_error(const mdet_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mdet_status mdet_create(mdet_ctx** out, int device, int precision) {
  if (!out) return MDET_E_ARG;
  *out = nullptr;
  if (precision != MDET_PRECISION_FP64 && precision != MDET_PRECISION_MIXED) return MDET_E_ARG;
  if (device < MDET_NO_DEVICE) return MDET_E_ARG;
  mdet_ctx* c = new (std::nothrow) mdet_ctx();
  if (!c) return MDET_E_OOM;
  c->device = device;
  c->precision = precision;
  // the accuracy targets of the two paths: 1e-5 (mixed) and 1e-8 (FP64) relative
  c->fallback_tol = precision == MDET_PRECISION_MIXED ? 1e-5 : 1e-8;
  c->fallback_cap = precision == MDET_PRECISION_MIXED ? 256 : 512;
  c->mo_ec = precision == MDET_PRECISION_MIXED ? 4 : 6;  // measured best electron block of each orbital kernel
  if (device >= 0) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) {
      delete c;
      return MDET_E_CUDA;
    }
    bool ok = cudaSetDevice(device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) == cudaSuccess;
    int lo = 0, hi = 0;
    ok = ok && cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
         cudaStreamCreateWithPriority(&c->cstream, cudaStreamNonBlocking, hi) == cudaSuccess &&
         cudaStreamCreateWithFlags(&c->fstream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->joined, cudaEventDisableTiming) == cudaSuccess &&
         cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) == cudaSuccess;
    for (int i = 0; ok && i < mdet_ctx::kMaxChunks; i++)
      ok = cudaEventCreateWithFlags(&c->contracted[i], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->prepared[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      delete c;
      return MDET_E_CUDA;
    }
  }
  *out = c;
  return MDET_OK;
}

void mdet_destroy(mdet_ctx* c) {
  if (!c) return;
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_scratch(c);
    free_problem(c);
    for (cudaEvent_t e : {c->ev_origin, c->ev_refine[0], c->ev_refine[1], c->ev_done})
      if (e) cudaEventDestroy(e);
    for (int k = 0; k < mdet_ctx::kMaxChunks; k++) {
      for (int i = 0; i < mdet_ctx::kEvPerChunk; i++)
        if (c->ev[k][i]) cudaEventDestroy(c->ev[k][i]);
      if (c->contracted[k]) cudaEventDestroy(c->contracted[k]);
      if (c->prepared[k]) cudaEventDestroy(c->prepared[k]);
    }
    if (c->cstream) cudaStreamDestroy(c->cstream);
    if (c->fstream) cudaStreamDestroy(c->fstream);
    if (c->joined) cudaEventDestroy(c->joined);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
  }
  delete c;
}

mdet_status mdet_set_system(mdet_ctx* c, int n_up, int n_dn, int n_nuc, const double* Z, const double* xyz) {
  if (!c) return MDET_E_ARG;
  if (n_dn < 1 || n_up < n_dn || n_up > kMaxSpin)
    return fail(c, MDET_E_ARG, "need 1 <= n_dn <= n_up <= %d (got %d, %d)", kMaxSpin, n_up, n_dn);
  if (n_nuc < 0 || (n_nuc > 0 && (!Z || !xyz))) return fail(c, MDET_E_ARG, "bad nuclei");
  c->n_up = n_up;
  c->n_dn = n_dn;
  c->n_nuc = n_nuc;
  c->Z.assign(Z, Z + n_nuc);
  c->nuc_xyz.assign(xyz, xyz + 3 * n_nuc);
  c->has_system = true;
  c->has_ci = false;
  c->err.clear();
  return MDET_OK;
}

mdet_status mdet_set_orbitals(mdet_ctx* c, int n_shell, const int32_t* shell_l, const int32_t* shell_center,
                              const int32_t* shell_nprim, const double* alpha, const double* coef, int n_mo,
                              const double* mo_coef) {
  if (!c) return MDET_E_ARG;
  if (!c->has_system) return fail(c, MDET_E_STATE, "set_system must come first");
  if (n_shell < 1 || !shell_l || !shell_center || !shell_nprim || !alpha || !coef || !mo_coef)
    return fail(c, MDET_E_ARG, "null or empty basis");
  if (n_mo < 1 || n_mo > MDET_MAX_MO) return fail(c, MDET_E_ARG, "n_mo must be in 1..%d", MDET_MAX_MO);
  if (n_mo < c->n_up) return fail(c, MDET_E_ARG, "n_mo < n_up");
  c->shell_l.assign(shell_l, shell_l + n_shell);
  c->shell_center.assign(shell_center, shell_center + n_shell);
  c->shell_nprim.assign(shell_nprim, shell_nprim + n_shell);
  c->shell_prim0.resize(n_shell);
  c->shell_ao0.resize(n_shell);
  int np = 0, nao = 0;
  for (int s = 0; s < n_shell; s++) {
    if (shell_l[s] < 0 || shell_l[s] > kMaxL) return fail(c, MDET_E_ARG, "shell %d: l=%d outside 0..3", s, shell_l[s]);
    if (shell_center[s] < 0 || shell_center[s] >= c->n_nuc) return fail(c, MDET_E_ARG, "shell %d: bad centre", s);
    if (shell_nprim[s] < 1) return fail(c, MDET_E_ARG, "shell %d: no primitive", s);
    c->shell_prim0[s] = np;
    c->shell_ao0[s] = nao;
    np += shell_nprim[s];
    nao += (shell_l[s] + 1) * (shell_l[s] + 2) / 2;
  }
  if (n_mo > nao) return fail(c, MDET_E_ARG, "n_mo (%d) > n_ao (%d)", n_mo, nao);
  c->n_shell = n_shell;
  c->n_prim = np;
  c->n_ao = nao;
  c->n_mo = n_mo;
  c->alpha.assign(alpha, alpha + np);
  c->coef.assign(coef, coef + np);
  c->mo_colmajor.assign(mo_coef, mo_coef + (size_t)nao * n_mo);
  c->has_orbitals = true;
  c->has_ci = false;
  c->err.clear();
  return MDET_OK;
}

mdet_status mdet_omega_sort(int64_t n, int n_int, const uint64_t* dets, int64_t* order) {
  if (n < 0 || n_int < 1 || (n > 0 && (!dets || !order))) return MDET_E_ARG;
  std::vector<int64_t> idx = omega_order(n, n_int, dets);
  std::copy(idx.begin(), idx.end(), order);
  return MDET_OK;
}

mdet_status mdet_set_ci_expansion(mdet_ctx* c, int64_t n_det, int n_int, const uint64_t* det_up,
                                  const uint64_t* det_dn, const double* coef) {
  if (!c) return MDET_E_ARG;
  if (!c->has_system || !c->has_orbitals) return fail(c, MDET_E_STATE, "set_system and set_orbitals must come first");
  if (n_det < 1 || !det_up || !det_dn || !coef) return fail(c, MDET_E_ARG, "empty expansion or null pointer");
  if (n_det >= (int64_t)1 << 31) return fail(c, MDET_E_ARG, "n_det must be below 2^31");
  const int want_int = (c->n_mo + 63) / 64;
  if (final_smem_bytes_host(c->n_up, c->n_dn, c->n_mo, c->precision == MDET_PRECISION_MIXED) > 227 * 1024)
    return fail(c, MDET_E_ARG, "(n_up + n_dn) * n_mo too large for the per-walker epilogue (shared memory)");
  if (n_int != want_int) return fail(c, MDET_E_ARG, "n_int=%d but ceil(n_mo/64)=%d", n_int, want_int);
  c->has_ci = false;
  const uint64_t* in[2] = {det_up, det_dn};
  const int nel[2] = {c->n_up, c->n_dn};
  // validation: popcount and bits beyond n_mo
  for (int sp = 0; sp < 2; sp++)
    for (int64_t k = 0; k < n_det; k++) {
      const uint64_t* w = in[sp] + k * n_int;
      if (popcount_words(w, n_int) != nel[sp])
        return fail(c, MDET_E_INPUT, "product %lld: spin %d determinant has %d electrons, expected %d",
                    (long long)k, sp, popcount_words(w, n_int), nel[sp]);
      const int top = c->n_mo - 64 * (n_int - 1);  // valid bits in the last word
      if (top < 64 && (w[n_int - 1] >> top) != 0)
        return fail(c, MDET_E_INPUT, "product %lld: spin %d determinant occupies an MO >= n_mo", (long long)k, sp);
    }
  for (int64_t k = 0; k < n_det; k++)
    if (!std::isfinite(coef[k])) return fail(c, MDET_E_INPUT, "product %lld: coefficient is not finite", (long long)k);
  // reference product: the largest |c_k| (first one on ties)
  int64_t kref = 0;
  for (int64_t k = 1; k < n_det; k++)
    if (std::fabs(coef[k]) > std::fabs(coef[kref])) kref = k;

  std::vector<int32_t> idx_of[2];  // product -> context index of its spin determinant
  for (int sp = 0; sp < 2; sp++) {
    const uint64_t* D = in[sp];
    // Sec. 2.1: radix sort by the key of Eq. 3, then remove duplicates among equal keys
    std::vector<int64_t> ord = omega_order(n_det, n_int, D);
    std::vector<int64_t> uniq;  // product index of each distinct determinant, in omega order
    for (int64_t q = 0; q < n_det; q++)
      if (q == 0 || cmp_det(D + ord[q] * n_int, D + ord[q - 1] * n_int, n_int) != 0) uniq.push_back(ord[q]);
    const int64_t nu = (int64_t)uniq.size();
    // position of every product's determinant in the distinct list: binary search (Sec. 2.1)
    std::vector<int32_t> pos(n_det);
    for (int64_t k = 0; k < n_det; k++) {
      int64_t lo = 0, hi = nu - 1;
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cmp_det(D + uniq[mid] * n_int, D + k * n_int, n_int) < 0) lo = mid + 1; else hi = mid;
      }
      pos[k] = (int32_t)lo;
    }
    std::vector<uint64_t> udets((size_t)nu * n_int);
    for (int64_t i = 0; i < nu; i++) std::copy(D + uniq[i] * n_int, D + (uniq[i] + 1) * n_int, udets.begin() + i * n_int);
    std::vector<int32_t> ctx_of;
    mdet_status st = spin_tables(c, sp, n_int, udets, pos[kref], ctx_of);
    if (st != MDET_OK) return st;
    idx_of[sp].resize(n_det);
    for (int64_t k = 0; k < n_det; k++) idx_of[sp][k] = ctx_of[pos[k]];
  }
  // C in the paper's column-major order: radix sort of N_up * j + i
  const int64_t nup = (int64_t)c->exc[0].size(), ndn = (int64_t)c->exc[1].size();
  std::vector<uint64_t> key(n_det);
  std::vector<int64_t> ord(n_det);
  for (int64_t k = 0; k < n_det; k++) {
    key[k] = (uint64_t)idx_of[1][k] * (uint64_t)nup + (uint64_t)idx_of[0][k];
    ord[k] = k;
  }
  radix_sort_u64(ord, key);
  for (int64_t q = 1; q < n_det; q++)
    if (key[ord[q]] == key[ord[q - 1]])
      return fail(c, MDET_E_INPUT, "products %lld and %lld repeat the same (up, down) pair", (long long)ord[q - 1],
                  (long long)ord[q]);
  c->coo_row.resize(n_det);
  c->coo_col.resize(n_det);
  c->coo_val.resize(n_det);
  for (int64_t q = 0; q < n_det; q++) {
    c->coo_row[q] = idx_of[0][ord[q]];
    c->coo_col[q] = idx_of[1][ord[q]];
    c->coo_val[q] = coef[ord[q]];
  }
  // row-major copy for the v = C D_dn product (Sec. 2.4)
  for (int64_t k = 0; k < n_det; k++) {
    key[k] = (uint64_t)idx_of[0][k] * (uint64_t)ndn + (uint64_t)idx_of[1][k];
    ord[k] = k;
  }
  radix_sort_u64(ord, key);
  c->csr_row.resize(n_det);
  c->csr_col.resize(n_det);
  c->csr_val.resize(n_det);
  for (int64_t q = 0; q < n_det; q++) {
    c->csr_row[q] = idx_of[0][ord[q]];
    c->csr_col[q] = idx_of[1][ord[q]];
    c->csr_val[q] = coef[ord[q]];
  }
  c->csr_ptr.assign(nup + 1, 0);
  c->csc_ptr.assign(ndn + 1, 0);
  for (int64_t q = 0; q < n_det; q++) {
    c->csr_ptr[c->csr_row[q] + 1]++;
    c->csc_ptr[c->coo_col[q] + 1]++;
  }
  for (int64_t i = 0; i < nup; i++) c->csr_ptr[i + 1] += c->csr_ptr[i];
  for (int64_t j = 0; j < ndn; j++) c->csc_ptr[j + 1] += c->csc_ptr[j];
  c->n_det = n_det;
  c->n_int = n_int;
  mdet_status s = upload_problem(c);
  if (s != MDET_OK) return s;
  c->has_ci = true;
  c->err.clear();
  return MDET_OK;
}

mdet_status mdet_sm_chain(mdet_ctx* c, int64_t n_walk, double* r, int64_t ld, int32_t* n_inv, int32_t* n_subst,
                          void* stream) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "the chain runs on the context's device");
  if (!c->has_ci) return fail(c, MDET_E_STATE, "set_ci_expansion must come first");
  if (n_walk < 0 || !r || !n_inv || !n_subst || ld < n_walk) return fail(c, MDET_E_ARG, "bad chain arguments");
  if (n_walk > c->last_walk) return fail(c, MDET_E_STATE, "n_walk exceeds the walkers of the last evaluation");
  if (n_walk == 0) return MDET_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (c->last_stream != st) CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
  CUDA_TRY(c, cudaMemsetAsync(n_inv, 0, n_walk * sizeof(int32_t), st));
  CUDA_TRY(c, cudaMemsetAsync(n_subst, 0, n_walk * sizeof(int32_t), st));
  for (int sp = 0; sp < 2; sp++)
    CUDA_TRY(c, launch_sm_chain(c->P, c->S, sp, c->P.sm_steps[sp], c->P.sm_n[sp], n_walk, r, ld, n_inv, n_subst, st));
  return MDET_OK;
}

mdet_status mdet_set_ci_expansion_device(mdet_ctx* c, int64_t n_det, int n_int, const uint64_t* det_up,
                                         const uint64_t* det_dn, const double* coef, void* stream) {
  if (!c) return MDET_E_ARG;
  if (!c->has_system || !c->has_orbitals) return fail(c, MDET_E_STATE, "set_system and set_orbitals must come first");
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "device preprocessing needs a context with a device");
  if (n_det < 1 || !det_up || !det_dn || !coef) return fail(c, MDET_E_ARG, "empty expansion or null pointer");
  if (n_det >= (int64_t)1 << 31) return fail(c, MDET_E_ARG, "n_det must be below 2^31");
  const int want_int = (c->n_mo + 63) / 64;
  if (final_smem_bytes_host(c->n_up, c->n_dn, c->n_mo, c->precision == MDET_PRECISION_MIXED) > 227 * 1024)
    return fail(c, MDET_E_ARG, "(n_up + n_dn) * n_mo too large for the per-walker epilogue (shared memory)");
  if (n_int != want_int) return fail(c, MDET_E_ARG, "n_int=%d but ceil(n_mo/64)=%d", n_int, want_int);
  CUDA_TRY(c, cudaSetDevice(c->device));
  c->has_ci = false;
  cudaStream_t st = (cudaStream_t)stream;
  PreDevice* h = nullptr;
  PreSpin spin[2];
  std::string msg;
  mdet_status s = pre_distinct(&h, n_det, n_int, det_up, det_dn, coef, c->n_up, c->n_dn, c->n_mo, st, spin, &msg);
  if (s != MDET_OK) {
    pre_free(h);
    return fail(c, s, "%s", msg.c_str());
  }
  std::vector<int32_t> ctx_of[2];
  for (int sp = 0; sp < 2 && s == MDET_OK; sp++) s = spin_tables(c, sp, n_int, spin[sp].udets, spin[sp].iref, ctx_of[sp]);
  if (s != MDET_OK) {
    pre_free(h);
    return s;
  }
  PreC C;
  s = pre_build_c(h, ctx_of, (int64_t)c->exc[0].size(), (int64_t)c->exc[1].size(), st, &C, &msg);
  pre_free(h);
  if (s != MDET_OK) return fail(c, s, "%s", msg.c_str());
  c->coo_row = std::move(C.csc_row);
  c->coo_col = std::move(C.csc_col);
  c->coo_val = std::move(C.csc_val);
  c->csr_row = std::move(C.csr_row);
  c->csr_col = std::move(C.csr_col);
  c->csr_val = std::move(C.csr_val);
  c->csr_ptr = std::move(C.csr_ptr);
  c->csc_ptr = std::move(C.csc_ptr);
  c->n_det = n_det;
  c->n_int = n_int;
  s = upload_problem(c);
  if (s != MDET_OK) return s;
  c->has_ci = true;
  c->err.clear();
  return MDET_OK;
}

mdet_status mdet_truncate_norm(int64_t n_det, int n_int, const uint64_t* det_up, const uint64_t* det_dn,
                               const double* coef, double eps_up, double eps_dn, uint8_t* keep, double* norm_up,
                               double* norm_dn, int64_t* counts) {
  if (n_det < 0 || n_int < 1 || (n_det > 0 && (!det_up || !det_dn || !coef))) return MDET_E_ARG;
  const uint64_t* in[2] = {det_up, det_dn};
  const double eps[2] = {eps_up, eps_dn};
  double* norm_out[2] = {norm_up, norm_dn};
  std::vector<int64_t> dist_of[2];  // product -> index of its distinct determinant (omega order)
  std::vector<uint8_t> removed[2];
  int64_t n_all[2] = {0, 0};
  for (int sp = 0; sp < 2; sp++) {
    const uint64_t* D = in[sp];
    // distinct determinants (Sec. 2.1 sort by the key of Eq. 3), then the norm of each (Sec. 3):
    // N_i = sum of c_k^2 over the products whose spin-sp determinant is D_i
    std::vector<int64_t> ord = omega_order(n_det, n_int, D);
    dist_of[sp].assign(n_det, 0);
    std::vector<double> sum, comp;
    for (int64_t q = 0; q < n_det; q++) {
      if (q == 0 || cmp_det(D + ord[q] * n_int, D + ord[q - 1] * n_int, n_int) != 0) {
        sum.push_back(0.0);
        comp.push_back(0.0);
      }
      dist_of[sp][ord[q]] = (int64_t)sum.size() - 1;
    }
    // Neumaier summation in product order (deterministic whatever the sort did with equal keys)
    for (int64_t k = 0; k < n_det; k++) {
      const int64_t i = dist_of[sp][k];
      const double x = coef[k] * coef[k], t = sum[i] + x;
      comp[i] += std::fabs(sum[i]) >= std::fabs(x) ? (sum[i] - t) + x : (x - t) + sum[i];
      sum[i] = t;
    }
    n_all[sp] = (int64_t)sum.size();
    removed[sp].assign(sum.size(), 0);
    for (size_t i = 0; i < sum.size(); i++) {
      sum[i] += comp[i];
      removed[sp][i] = eps[sp] >= 0.0 && sum[i] <= eps[sp];
    }
    if (norm_out[sp])
      for (int64_t k = 0; k < n_det; k++) norm_out[sp][k] = sum[dist_of[sp][k]];
  }
  // a product survives when neither of its determinants was removed (all removals use the
  // norms of the untruncated expansion; no renormalisation)
  int64_t n_keep = 0;
  std::vector<uint8_t> used[2] = {std::vector<uint8_t>(n_all[0], 0), std::vector<uint8_t>(n_all[1], 0)};
  for (int64_t k = 0; k < n_det; k++) {
    const bool kk = !removed[0][dist_of[0][k]] && !removed[1][dist_of[1][k]];
    if (keep) keep[k] = kk ? 1 : 0;
    if (kk) {
      n_keep++;
      used[0][dist_of[0][k]] = 1;
      used[1][dist_of[1][k]] = 1;
    }
  }
  if (counts) {
    counts[0] = n_keep;
    for (int sp = 0; sp < 2; sp++) {
      int64_t u = 0;
      for (uint8_t x : used[sp]) u += x;
      counts[1 + sp] = u;
      counts[3 + sp] = n_all[sp];
    }
  }
  return MDET_OK;
}

mdet_status mdet_evaluate(mdet_ctx* c, int64_t n_walk, const double* R, double* log_abs_psi, int8_t* sign,
                          double* grad, double* lap, double* e_local, uint32_t* status, void* stream) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "context has no device");
  if (!c->has_ci) return fail(c, MDET_E_STATE, "set_ci_expansion must come first");
  if (n_walk < 0) return fail(c, MDET_E_ARG, "n_walk < 0");
  if (n_walk == 0) return MDET_OK;
  if (n_walk > (int64_t)1 << 30) return fail(c, MDET_E_ARG, "n_walk above 2^30");
  if (!R || !log_abs_psi || !sign || !grad || !lap) return fail(c, MDET_E_ARG, "null device pointer");
  CUDA_TRY(c, cudaSetDevice(c->device));
  mdet_status s = ensure_scratch(c, n_walk);
  if (s != MDET_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const DevProblem& P = c->P;
  const bool mixed = c->precision == MDET_PRECISION_MIXED;
  const bool prof_all = c->profiling == 1;  // events around every stage
  const bool prof_stamp = c->profiling == 2;  // the contraction kernels' own timer stamps, no events
  const bool prof = prof_all;
  // chunking: mixed precision splits large batches into a two-stream pipeline
  int nch = 1;
  const int64_t tiles = (n_walk + kWalkerPad - 1) / kWalkerPad;
  if (mixed) {
    nch = c->n_chunks_cfg > 0 ? c->n_chunks_cfg : auto_chunks(c, n_walk);
    nch = (int)std::min<int64_t>(std::min<int64_t>(nch, tiles), mdet_ctx::kMaxChunks);
  }
  if (prof) {
    for (int k = 0; k < nch; k++)
      for (int i = 0; i < mdet_ctx::kEvPerChunk; i++)
        if (!c->ev[k][i]) CUDA_TRY(c, cudaEventCreate(&c->ev[k][i]));
    for (cudaEvent_t* e : {&c->ev_origin, &c->ev_refine[0], &c->ev_refine[1], &c->ev_done})
      if (!*e) CUDA_TRY(c, cudaEventCreate(e));
    CUDA_TRY(c, cudaEventRecord(c->ev_origin, (cudaStream_t)stream));
  }
  const int64_t N = P.n_elec;
  // chunk k covers tiles [t0, t1) in the proportions kFirstWeight : kMidWeight ... : kLastWeight
  // (with at least one tile each), an even split with fewer than 3 chunks
  auto chunk_range = [&](int k, int64_t* off, int64_t* n) {
    int64_t t0 = tiles * k / nch, t1 = tiles * (k + 1) / nch;
    const int64_t units = kFirstWeight + (int64_t)kMidWeight * (nch - 2) + kLastWeight;
    if (nch >= 3 && tiles >= nch) {
      auto edge = [&](int q) -> int64_t {  // tiles before chunk q
        if (q <= 0) return 0;
        if (q >= nch) return tiles;
        const int64_t u = kFirstWeight + (int64_t)kMidWeight * (q - 1);
        return std::min(std::max(tiles * u / units, (int64_t)q), tiles - (nch - q));
      };
      t0 = edge(k);
      t1 = edge(k + 1);
    }
    *off = t0 * kWalkerPad;
    *n = std::min<int64_t>(t1 * kWalkerPad, n_walk) - *off;
  };
  // stage i (MDET_STAGE_*) of chunk k on stream ks, bracketed by its two profiling events
  auto stage = [&](int k, int i, cudaStream_t ks, int persistent) -> mdet_status {
    int64_t off, n;
    chunk_range(k, &off, &n);
    const DevScratch S = scratch_view(c->S, P, off);
    const double* Rk = R + off * N * 3;
    const bool mark = prof_all;
    if (mark) CUDA_TRY(c, cudaEventRecord(c->ev[k][2 * i], ks));
    switch (i) {
      case MDET_STAGE_ORBITALS:
        CUDA_TRY(c, mixed ? launch_mo_mixed(P, S, n, Rk, ks) : launch_mo_f64(P, S, n, Rk, ks));
        break;
      case MDET_STAGE_REFERENCE: CUDA_TRY(c, launch_ref_tables(P, S, n, mixed, ks)); break;
      case MDET_STAGE_RATIOS:
        CUDA_TRY(c, mixed ? launch_ratios_mixed(P, S, n, ks) : launch_ratios_f64(P, S, n, ks));
        break;
      case MDET_STAGE_ZERO: CUDA_TRY(c, launch_zero_f64(P, S, n, ks)); break;
      case MDET_STAGE_CONTRACT: {
        unsigned long long* q = c->S.queue + kQueueWords * k;
        CUDA_TRY(c, launch_contract_f64(P, S, n, ks, q, persistent, prof_stamp ? q + 2 : nullptr));
        break;
      }
      default:
        CUDA_TRY(c, launch_final(P, S, n, Rk, log_abs_psi + off, sign + off, grad + off * N * 3, lap + off * N,
                                 e_local ? e_local + off : nullptr, status ? status + off : nullptr, mixed, ks));
    }
    if (mark) CUDA_TRY(c, cudaEventRecord(c->ev[k][2 * i + 1], ks));
    return MDET_OK;
  };
  mdet_status ms;
  if (nch == 1) {
    for (int i = 0; i < MDET_N_STAGES; i++)
      if ((ms = stage(0, i, st, 0)) != MDET_OK) return ms;
  } else {
    // fs (FP32-pipe stages, in this order): orbitals, reference and ratios of chunk 0,
    // those of chunk 1, the epilogue of chunk 0 (after its contraction), chunk 2, the
    // epilogue of chunk 1, ... ; xs (higher priority): the contraction of each chunk once
    // its ratios are ready. The contraction runs on a persistent grid of 4 blocks per SM
    // (unless spmm_blocks says otherwise) that leaves the rest of every SM to fs.
    cudaStream_t fs = c->fstream, xs = c->cstream;
    const int persistent = 4 * std::max(c->n_sm, 1);
    CUDA_TRY(c, cudaEventRecord(c->fork, st));
    CUDA_TRY(c, cudaStreamWaitEvent(fs, c->fork, 0));
    CUDA_TRY(c, cudaStreamWaitEvent(xs, c->fork, 0));
    // each chunk's accumulators are cleared on xs right before its contraction: the contraction
    // adds into them with atomics, which then find the freshly cleared lines in L2 (clearing the
    // whole batch up front measured 33.1 against 30.6 ms per step at 8,192 walkers)
    auto enqueue = [&](int k) -> mdet_status {
      mdet_status m;
      for (int i = MDET_STAGE_ORBITALS; i < MDET_STAGE_ZERO; i++)
        if ((m = stage(k, i, fs, 0)) != MDET_OK) return m;
      CUDA_TRY(c, cudaEventRecord(c->prepared[k], fs));
      CUDA_TRY(c, cudaStreamWaitEvent(xs, c->prepared[k], 0));
      for (int i = MDET_STAGE_ZERO; i <= MDET_STAGE_CONTRACT; i++)
        if ((m = stage(k, i, xs, persistent)) != MDET_OK) return m;
      CUDA_TRY(c, cudaEventRecord(c->contracted[k], xs));
      return MDET_OK;
    };
    if ((ms = enqueue(0)) != MDET_OK) return ms;
    for (int k = 0; k < nch; k++) {
      if (k + 1 < nch && (ms = enqueue(k + 1)) != MDET_OK) return ms;
      CUDA_TRY(c, cudaStreamWaitEvent(fs, c->contracted[k], 0));
      if ((ms = stage(k, MDET_STAGE_FINAL, fs, 0)) != MDET_OK) return ms;
    }
    // every contraction precedes contracted[nch - 1], which fs has waited for
    CUDA_TRY(c, cudaEventRecord(c->joined, fs));
    CUDA_TRY(c, cudaStreamWaitEvent(st, c->joined, 0));
  }
  c->prof_chunks = nch;
  // stability fallback over the whole batch, after every chunk has finished: mixed precision
  // escalates to FP64 first, FP64 goes to full LU directly
  // kernels: 6 per chunk (orbitals, reference, ratios, 2 contractions, epilogue); the full-LU
  // fallback 5 (list, dets, scale, rows, out); the mixed refinement adds its list, gather,
  // FP64 orbitals and scatter, and either the mark or the 5 FP64 table kernels
  c->last_kernels = 6 * nch;
  if (prof_all) CUDA_TRY(c, cudaEventRecord(c->ev_refine[0], st));
  if (mixed && c->E.fb && P.fallback_tol > 0.0) {
    const bool table = escalation_on(c);
    mdet_status es = refine(c, table, n_walk, R, log_abs_psi, sign, grad, lap, e_local, status, st);
    if (es != MDET_OK) return es;
    c->last_kernels += 4 + 5 + (table ? 5 : 1);
  } else {
    CUDA_TRY(c, launch_fallback(P, c->S, n_walk, R, log_abs_psi, sign, grad, lap, e_local, status, st));
    if (P.fallback_tol > 0.0 && c->S.fb && P.n_up <= MDET_FALLBACK_MAX_SPIN) c->last_kernels += 5;
  }
  if (prof_all) {
    CUDA_TRY(c, cudaEventRecord(c->ev_refine[1], st));
    CUDA_TRY(c, cudaEventRecord(c->ev_done, st));
  }
  c->have_profile = prof_all || prof_stamp;
  c->have_timeline = prof_all;
  c->last_stream = st;
  c->last_walk = n_walk;
  return MDET_OK;
}

mdet_status mdet_evaluate_host(mdet_ctx* c, int64_t n_walk, const double* R, double* log_abs_psi, int8_t* sign,
                               double* grad, double* lap, double* e_local, uint32_t* status) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "context has no device");
  if (!c->has_ci) return fail(c, MDET_E_STATE, "set_ci_expansion must come first");
  if (n_walk < 0) return fail(c, MDET_E_ARG, "n_walk < 0");
  if (n_walk == 0) return MDET_OK;
  if (!R || !log_abs_psi) return fail(c, MDET_E_ARG, "null host pointer");
  CUDA_TRY(c, cudaSetDevice(c->device));
  mdet_status s = ensure_scratch(c, n_walk);
  if (s != MDET_OK) return s;
  DevScratch& S = c->S;
  const int64_t N = c->n_up + c->n_dn;
  const size_t nR = (size_t)n_walk * N * 3;
  // staging: R, then outputs [log | sign(8 B slots) | grad | lap | e_local | status(8 B slots)]
  const size_t nout = (size_t)n_walk * (1 + 1 + 3 * N + N + 1 + 1);
  if (!S.R_stage) {
    if ((s = dalloc(c, &S.R_stage, (size_t)S.cap_walk * N * 3))) return s;
    if ((s = dalloc(c, &S.out_stage, (size_t)S.cap_walk * (4 + 4 * N)))) return s;
  }
  cudaStream_t st = c->own_stream;
  double* d_log = S.out_stage;
  int8_t* d_sign = (int8_t*)(d_log + n_walk);
  double* d_grad = d_log + 2 * n_walk;
  double* d_lap = d_grad + 3 * N * n_walk;
  double* d_el = d_lap + N * n_walk;
  uint32_t* d_st = (uint32_t*)(d_el + n_walk);
  (void)nout;
  CUDA_TRY(c, cudaMemcpyAsync(S.R_stage, R, nR * sizeof(double), cudaMemcpyHostToDevice, st));
  s = mdet_evaluate(c, n_walk, S.R_stage, d_log, d_sign, d_grad, d_lap, d_el, d_st, st);
  if (s != MDET_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(log_abs_psi, d_log, n_walk * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (sign) CUDA_TRY(c, cudaMemcpyAsync(sign, d_sign, n_walk * sizeof(int8_t), cudaMemcpyDeviceToHost, st));
  if (grad) CUDA_TRY(c, cudaMemcpyAsync(grad, d_grad, 3 * N * n_walk * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (lap) CUDA_TRY(c, cudaMemcpyAsync(lap, d_lap, N * n_walk * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (e_local) CUDA_TRY(c, cudaMemcpyAsync(e_local, d_el, n_walk * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (status) CUDA_TRY(c, cudaMemcpyAsync(status, d_st, n_walk * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  return MDET_OK;
}

mdet_status mdet_get_ratios(mdet_ctx* c, int64_t n_walk, double* r_up, double* r_dn, double* log_d0,
                            int8_t* sign_d0) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "context has no device");
  if (!c->has_ci || c->last_walk == 0) return fail(c, MDET_E_STATE, "no evaluation yet");
  if (n_walk < 0 || n_walk > c->last_walk) return fail(c, MDET_E_ARG, "n_walk beyond the last evaluation");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
  const DevScratch& S = c->S;
  const int64_t nu = c->exc[0].size(), nd = c->exc[1].size();
  if (r_up || r_dn) {
    std::vector<double> h((size_t)(nu + nd) * S.wp);
    CUDA_TRY(c, cudaMemcpy(h.data(), S.r, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t w = 0; w < n_walk; w++) {
      if (r_up)
        for (int64_t i = 0; i < nu; i++) r_up[w * nu + i] = h[(size_t)i * S.wp + w];
      if (r_dn)
        for (int64_t j = 0; j < nd; j++) r_dn[w * nd + j] = h[(size_t)(nu + j) * S.wp + w];
    }
  }
  if (log_d0) CUDA_TRY(c, cudaMemcpy(log_d0, S.ld0, n_walk * 2 * sizeof(double), cudaMemcpyDeviceToHost));
  if (sign_d0) {
    std::vector<double> h(n_walk * 2);
    CUDA_TRY(c, cudaMemcpy(h.data(), S.sg0, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < h.size(); q++) sign_d0[q] = (int8_t)(h[q] > 0 ? 1 : (h[q] < 0 ? -1 : 0));
  }
  return MDET_OK;
}

mdet_status mdet_set_fallback(mdet_ctx* c, double tol, int max_walkers) {
  if (!c || max_walkers < 1 || max_walkers > 65535) return MDET_E_ARG;
  const bool resize = max_walkers != c->fallback_cap || (tol > 0.0 && !c->S.fb && !c->E.fb && c->S.cap_walk > 0);
  c->fallback_tol = tol;
  c->fallback_cap = max_walkers;
  c->P.fallback_tol = tol;
  c->P.fallback_cap = max_walkers;
  if (resize) free_scratch(c);  // the fallback scratch is sized by the cap
  return MDET_OK;
}

mdet_status mdet_set_escalation(mdet_ctx* c, int mode) {
  if (!c || mode < MDET_ESCALATE_AUTO || mode > MDET_ESCALATE_NEVER) return MDET_E_ARG;
  c->escalate = mode;
  return MDET_OK;
}

mdet_status mdet_get_fallback(const mdet_ctx* c, double* tol, int* max_walkers) {
  if (!c || !tol || !max_walkers) return MDET_E_ARG;
  *tol = c->fallback_tol;
  *max_walkers = c->fallback_cap;
  return MDET_OK;
}

mdet_status mdet_set_walker_chunks(mdet_ctx* c, int n_chunks) {
  if (!c || n_chunks < 0) return MDET_E_ARG;
  c->n_chunks_cfg = std::min(n_chunks, (int)mdet_ctx::kMaxChunks);
  return MDET_OK;
}

mdet_status mdet_get_last_launches(const mdet_ctx* c, int32_t* n_chunks, int32_t* n_kernels) {
  if (!c) return MDET_E_ARG;
  if (n_chunks) *n_chunks = c->last_walk > 0 ? c->prof_chunks : 0;
  if (n_kernels) *n_kernels = c->last_walk > 0 ? c->last_kernels : 0;
  return MDET_OK;
}

mdet_status mdet_set_profiling(mdet_ctx* c, int enable) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "context has no device");
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (enable < 0 || enable > 2) return fail(c, MDET_E_ARG, "profiling mode must be 0, 1 or 2");
  c->profiling = enable;
  c->have_profile = false;
  c->have_timeline = false;
  return MDET_OK;
}

mdet_status mdet_get_profile(mdet_ctx* c, float* ms) {
  if (!c || !ms) return MDET_E_ARG;
  if (!c->have_profile) return fail(c, MDET_E_STATE, "no profiled evaluation yet");
  CUDA_TRY(c, cudaSetDevice(c->device));
  for (int i = 0; i < MDET_N_STAGES; i++) ms[i] = 0.0f;
  if (!c->have_timeline) {  // mode 2: the contraction launches' own global-timer stamps
    const int nw = kQueueWords * c->prof_chunks;
    std::vector<unsigned long long> w((size_t)nw);
    CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
    CUDA_TRY(c, cudaMemcpy(w.data(), c->S.queue, sizeof(unsigned long long) * nw, cudaMemcpyDeviceToHost));
    double ns = 0.0;
    for (int k = 0; k < c->prof_chunks; k++)
      for (int l = 0; l < 2; l++) {
        const unsigned long long t0 = ~w[(size_t)kQueueWords * k + 2 + 2 * l], t1 = w[(size_t)kQueueWords * k + 3 + 2 * l];
        if (w[(size_t)kQueueWords * k + 2 + 2 * l] != 0 && t1 > t0) ns += (double)(t1 - t0);  // 0: the launch ran no block
      }
    ms[MDET_STAGE_CONTRACT] = (float)(ns * 1e-6);
    return MDET_OK;
  }
  for (int k = 0; k < c->prof_chunks; k++)
    for (int i = 0; i < MDET_N_STAGES; i++) {
      float t = 0.0f;
      CUDA_TRY(c, cudaEventSynchronize(c->ev[k][2 * i + 1]));
      CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev[k][2 * i], c->ev[k][2 * i + 1]));
      ms[i] += t;
    }
  return MDET_OK;
}

mdet_status mdet_get_timeline(mdet_ctx* c, int32_t* n_chunks, float* ms) {
  if (!c || !n_chunks || !ms) return MDET_E_ARG;
  if (!c->have_timeline) return fail(c, MDET_E_STATE, "no evaluation profiled with every stage yet");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaEventSynchronize(c->ev_done));
  for (int i = 0; i < MDET_MAX_CHUNKS * MDET_N_STAGES * 2 + 3; i++) ms[i] = 0.0f;
  *n_chunks = c->prof_chunks;
  for (int k = 0; k < c->prof_chunks; k++)
    for (int i = 0; i < mdet_ctx::kEvPerChunk; i++)
      CUDA_TRY(c, cudaEventElapsedTime(&ms[k * mdet_ctx::kEvPerChunk + i], c->ev_origin, c->ev[k][i]));
  float* tail = ms + MDET_MAX_CHUNKS * mdet_ctx::kEvPerChunk;
  CUDA_TRY(c, cudaEventElapsedTime(&tail[0], c->ev_origin, c->ev_refine[0]));
  CUDA_TRY(c, cudaEventElapsedTime(&tail[1], c->ev_origin, c->ev_refine[1]));
  CUDA_TRY(c, cudaEventElapsedTime(&tail[2], c->ev_origin, c->ev_done));
  return MDET_OK;
}

mdet_status mdet_selftest_df32(int device, int64_t n, const double* x, double* y_df, double* y_ref,
                               double* prod_df) {
  if (n < 1 || !x || !y_df || !y_ref || !prod_df || device < 0) return MDET_E_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MDET_E_CUDA;
  if (launch_selftest_df(n, x, y_df, y_ref, prod_df, nullptr) != cudaSuccess) return MDET_E_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return MDET_E_CUDA;
  return MDET_OK;
}

mdet_status mdet_selftest_inv_r(int device, int64_t n, const double* x, double* y_nr, double* y_ref) {
  if (n < 1 || !x || !y_nr || !y_ref || device < 0) return MDET_E_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MDET_E_CUDA;
  if (launch_selftest_inv_r(n, x, y_nr, y_ref, nullptr) != cudaSuccess) return MDET_E_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return MDET_E_CUDA;
  return MDET_OK;
}

mdet_status mdet_get_tuning(const mdet_ctx* c, mdet_tuning* out) {
  if (!c || !out) return MDET_E_ARG;
  *out = c->last_tune;
  out->spmm_chunk = c->spmm_chunk;
  out->mo_ec = c->mo_ec;
  out->walker_chunks = c->n_chunks_cfg;
  out->spmm_blocks = c->spmm_blocks;
  out->mo_impl = c->mo_impl;
  out->contract_impl = c->contract_impl;
  return MDET_OK;
}

mdet_status mdet_set_tuning(mdet_ctx* c, const mdet_tuning* t) {
  if (!c || !t) return MDET_E_ARG;
  if (t->spmm_chunk < 64 || t->spmm_chunk > 8192) return fail(c, MDET_E_ARG, "spmm_chunk outside 64..8192");
  if (t->mo_ec != 4 && t->mo_ec != 6 && t->mo_ec != 8) return fail(c, MDET_E_ARG, "mo_ec must be 4, 6 or 8");
  if (t->walker_chunks < 0) return fail(c, MDET_E_ARG, "walker_chunks < 0");
  if (t->spmm_blocks < 0) return fail(c, MDET_E_ARG, "spmm_blocks < 0");
  if (t->mo_impl < 0 || t->mo_impl > 2) return fail(c, MDET_E_ARG, "mo_impl must be 0, 1 or 2");
  if (t->contract_impl != 0 && t->contract_impl != 1) return fail(c, MDET_E_ARG, "contract_impl must be 0 or 1");
  if (t->contract_impl != c->contract_impl) {
    c->contract_impl = t->contract_impl;
    c->P.contract_impl = t->contract_impl;
    free_scratch(c);  // the double-float ratio pairs are allocated with the scratch
  }
  c->mo_impl = t->mo_impl;
  c->P.mo_impl = t->mo_impl;
  c->spmm_blocks = t->spmm_blocks;
  c->P.spmm_blocks = t->spmm_blocks;
  if (c->has_ci && c->device >= 0) {
    CUDA_TRY(c, cudaSetDevice(c->device));
    mdet_status s = ensure_items(c, t->spmm_chunk);
    if (s != MDET_OK) return s;
    use_items(c, c->P, t->spmm_chunk);
  }
  c->spmm_chunk = t->spmm_chunk;
  c->mo_ec = t->mo_ec;
  c->n_chunks_cfg = std::min(t->walker_chunks, (int)mdet_ctx::kMaxChunks);
  c->P.spmm_chunk = c->spmm_chunk;
  c->P.mo_ec = c->mo_ec;
  return MDET_OK;
}

mdet_status mdet_autotune(mdet_ctx* c, int64_t n_walk, const double* R, double budget_ms, mdet_tuning* out) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "context has no device");
  if (!c->has_ci) return fail(c, MDET_E_STATE, "set_ci_expansion must come first");
  if (n_walk < 1 || !R || budget_ms <= 0) return fail(c, MDET_E_ARG, "bad autotune arguments");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const int64_t N = c->n_up + c->n_dn;
  double *d_log = nullptr, *d_grad = nullptr, *d_lap = nullptr;
  int8_t* d_sign = nullptr;
  mdet_status s;
  if ((s = dalloc(c, &d_log, n_walk)) || (s = dalloc(c, &d_grad, 3 * N * n_walk)) ||
      (s = dalloc(c, &d_lap, N * n_walk)) || (s = dalloc(c, &d_sign, n_walk))) {
    cudaFree(d_log); cudaFree(d_grad); cudaFree(d_lap); cudaFree(d_sign);
    return s;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int prof = c->profiling;
  c->profiling = 0;
  cudaStream_t st = c->own_stream;
  double spent = 0.0;
  int trials = 0;
  auto timed = [&](const mdet_tuning& t, float* ms) -> mdet_status {
    mdet_status r = mdet_set_tuning(c, &t);
    if (r) return r;
    if ((r = mdet_evaluate(c, n_walk, R, d_log, d_sign, d_grad, d_lap, nullptr, nullptr, st))) return r;
    CUDA_TRY(c, cudaEventRecord(e0, st));
    for (int q = 0; q < 2; q++)
      if ((r = mdet_evaluate(c, n_walk, R, d_log, d_sign, d_grad, d_lap, nullptr, nullptr, st))) return r;
    CUDA_TRY(c, cudaEventRecord(e1, st));
    CUDA_TRY(c, cudaEventSynchronize(e1));
    CUDA_TRY(c, cudaEventElapsedTime(ms, e0, e1));
    *ms *= 0.5f;
    spent += 3.0 * *ms;
    trials++;
    return MDET_OK;
  };
  mdet_tuning cur{};
  mdet_get_tuning(c, &cur);
  if (cur.walker_chunks == 0) cur.walker_chunks = auto_chunks(c, n_walk);
  float best = 0.0f;
  s = timed(cur, &best);
  const bool mixed = c->precision == MDET_PRECISION_MIXED;
  const int chunks[] = {256, 512, 1024, 2048}, ecs[] = {4, 6, 8}, wcs[] = {1, 2, 3, 4};
  for (int param = 0; param < 3 && s == MDET_OK; param++) {
    const int* vals = param == 0 ? chunks : (param == 1 ? ecs : wcs);
    const int nv = param == 1 ? 3 : 4;
    if (param == 2 && !mixed) break;
    for (int q = 0; q < nv && s == MDET_OK && spent < budget_ms; q++) {
      mdet_tuning t = cur;
      int* field = param == 0 ? &t.spmm_chunk : (param == 1 ? &t.mo_ec : &t.walker_chunks);
      if (*field == vals[q]) continue;
      *field = vals[q];
      float ms = 0.0f;
      s = timed(t, &ms);
      if (s == MDET_OK && ms < best) {
        best = ms;
        cur = t;
      }
    }
  }
  mdet_status s2 = mdet_set_tuning(c, &cur);
  if (s == MDET_OK) s = s2;
  c->profiling = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(d_log); cudaFree(d_grad); cudaFree(d_lap); cudaFree(d_sign);
  c->last_tune = cur;
  c->last_tune.best_ms = best;
  c->last_tune.trials = trials;
  if (out && s == MDET_OK) *out = c->last_tune;
  return s;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of contexts
struct mdet_batch {
  int device = -1;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<mdet_ctx*> ctxs;
};

namespace {

void batch_release(mdet_batch* b) {
  if (!b) return;
  if (b->device >= 0) cudaSetDevice(b->device);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

mdet_status batch_setup(mdet_batch* b, int n_ctx, mdet_ctx* const* ctxs, int n_streams) {
  if (n_ctx < 1 || !ctxs || n_streams < 1 || n_streams > 16) return MDET_E_ARG;
  b->device = -1;
  for (int i = 0; i < n_ctx; i++) {
    if (!ctxs[i] || !ctxs[i]->has_ci || ctxs[i]->device < 0) return MDET_E_STATE;
    if (b->device < 0) b->device = ctxs[i]->device;
    if (ctxs[i]->device != b->device) return MDET_E_ARG;
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) return MDET_E_ARG;  // a context may appear once
  }
  if (cudaSetDevice(b->device) != cudaSuccess) return MDET_E_CUDA;
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) return MDET_E_CUDA;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return MDET_E_CUDA;
  b->streams.assign(n_streams, nullptr);
  b->joins.assign(n_streams, nullptr);
  for (int k = 0; k < n_streams; k++)
    if (cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming) != cudaSuccess)
      return MDET_E_CUDA;
  b->ctxs.assign(ctxs, ctxs + n_ctx);
  return MDET_OK;
}

// Fork from `origin`, evaluate every context on its stream, join back.
mdet_status batch_enqueue(mdet_batch* b, const int64_t* n_walk, const double* const* R, double* const* log_abs_psi,
                          int8_t* const* sign, double* const* grad, double* const* lap, double* const* e_local,
                          uint32_t* const* status, cudaStream_t origin) {
  const int n_ctx = (int)b->ctxs.size(), ns = (int)b->streams.size();
  // longest processing time first onto the least-loaded stream
  std::vector<double> cost(n_ctx);
  for (int i = 0; i < n_ctx; i++) {
    const mdet_ctx* c = b->ctxs[i];
    const double N = c->n_up + c->n_dn;
    const double per_walk = 4.0 * (double)c->n_det +
                            (c->precision == MDET_PRECISION_MIXED ? 0.2 : 2.0) * 5.0 * N * c->n_ao * c->n_mo +
                            40.0 * (double)(c->exc[0].size() + c->exc[1].size());
    cost[i] = per_walk * (double)n_walk[i];
  }
  std::vector<int> order(n_ctx);
  for (int i = 0; i < n_ctx; i++) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c2) { return cost[a] > cost[c2]; });
  std::vector<double> load(ns, 0.0);
  if (cudaEventRecord(b->fork, origin) != cudaSuccess) return MDET_E_CUDA;
  for (int k = 0; k < ns; k++)
    if (cudaStreamWaitEvent(b->streams[k], b->fork, 0) != cudaSuccess) return MDET_E_CUDA;
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[k] += cost[i];
    b->ctxs[i]->in_batch = true;
    mdet_status s = mdet_evaluate(b->ctxs[i], n_walk[i], R[i], log_abs_psi[i], sign[i], grad[i], lap[i],
                                  e_local ? e_local[i] : nullptr, status ? status[i] : nullptr, b->streams[k]);
    b->ctxs[i]->in_batch = false;
    if (s != MDET_OK) return s;
  }
  for (int k = 0; k < ns; k++) {
    if (cudaEventRecord(b->joins[k], b->streams[k]) != cudaSuccess) return MDET_E_CUDA;
    if (cudaStreamWaitEvent(origin, b->joins[k], 0) != cudaSuccess) return MDET_E_CUDA;
  }
  return MDET_OK;
}

}  // namespace

extern "C" {

mdet_status mdet_batch_evaluate(int n_ctx, mdet_ctx* const* ctxs, const int64_t* n_walk, const double* const* R,
                                double* const* log_abs_psi, int8_t* const* sign, double* const* grad,
                                double* const* lap, double* const* e_local, uint32_t* const* status,
                                int n_streams, void* stream) {
  if (!n_walk || !R || !log_abs_psi || !sign || !grad || !lap) return MDET_E_ARG;
  mdet_batch* b = new (std::nothrow) mdet_batch();
  if (!b) return MDET_E_OOM;
  mdet_status s = batch_setup(b, n_ctx, ctxs, n_streams);
  if (s == MDET_OK) s = batch_enqueue(b, n_walk, R, log_abs_psi, sign, grad, lap, e_local, status, (cudaStream_t)stream);
  // streams and events may be destroyed with work pending: the runtime defers it
  batch_release(b);
  return s;
}

mdet_status mdet_batch_create(mdet_batch** out, int n_ctx, mdet_ctx* const* ctxs, const int64_t* n_walk,
                              const double* const* R, double* const* log_abs_psi, int8_t* const* sign,
                              double* const* grad, double* const* lap, double* const* e_local,
                              uint32_t* const* status, int n_streams) {
  if (!out || !n_walk || !R || !log_abs_psi || !sign || !grad || !lap) return MDET_E_ARG;
  *out = nullptr;
  mdet_batch* b = new (std::nothrow) mdet_batch();
  if (!b) return MDET_E_OOM;
  mdet_status s = batch_setup(b, n_ctx, ctxs, n_streams);
  // one uncaptured pass sizes every scratch and sets every kernel attribute
  if (s == MDET_OK) s = batch_enqueue(b, n_walk, R, log_abs_psi, sign, grad, lap, e_local, status, b->origin);
  if (s == MDET_OK && cudaStreamSynchronize(b->origin) != cudaSuccess) s = MDET_E_CUDA;
  std::vector<int> prof(n_ctx > 0 ? n_ctx : 0);
  if (s == MDET_OK) {
    for (int i = 0; i < n_ctx; i++) {
      prof[i] = ctxs[i]->profiling;
      ctxs[i]->profiling = 0;
    }
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) s = MDET_E_CUDA;
    if (s == MDET_OK) {
      mdet_status se = batch_enqueue(b, n_walk, R, log_abs_psi, sign, grad, lap, e_local, status, b->origin);
      cudaError_t ee = cudaStreamEndCapture(b->origin, &b->graph);
      if (se != MDET_OK) s = se;
      else if (ee != cudaSuccess) s = MDET_E_CUDA;
    }
    if (s == MDET_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) s = MDET_E_CUDA;
    for (int i = 0; i < n_ctx; i++) ctxs[i]->profiling = prof[i];
  }
  if (s != MDET_OK) {
    batch_release(b);
    return s;
  }
  *out = b;
  return MDET_OK;
}

mdet_status mdet_batch_launch(mdet_batch* b, void* stream) {
  if (!b || !b->exec) return MDET_E_ARG;
  if (cudaSetDevice(b->device) != cudaSuccess) return MDET_E_CUDA;
  if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) return MDET_E_CUDA;
  return MDET_OK;
}

void mdet_batch_destroy(mdet_batch* b) { batch_release(b); }

mdet_status mdet_get_error_estimates(mdet_ctx* c, int64_t n_walk, double* cond1, double* est) {
  if (!c) return MDET_E_ARG;
  if (c->device < 0) return fail(c, MDET_E_NODEVICE, "context has no device");
  if (!c->has_ci || c->last_walk == 0) return fail(c, MDET_E_STATE, "no evaluation yet");
  if (n_walk < 0 || n_walk > c->last_walk) return fail(c, MDET_E_ARG, "n_walk beyond the last evaluation");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->last_stream));
  if (cond1) CUDA_TRY(c, cudaMemcpy(cond1, c->S.kap, n_walk * 2 * sizeof(double), cudaMemcpyDeviceToHost));
  if (est) CUDA_TRY(c, cudaMemcpy(est, c->S.est, n_walk * 2 * sizeof(double), cudaMemcpyDeviceToHost));
  return MDET_OK;
}

mdet_status mdet_get_stats(const mdet_ctx* c, mdet_stats* out) {
  if (!c || !out) return MDET_E_ARG;
  std::memset(out, 0, sizeof *out);
  out->n_up = c->n_up;
  out->n_dn = c->n_dn;
  out->n_ao = c->n_ao;
  out->n_mo = c->n_mo;
  out->n_int = c->n_int;
  out->n_det = c->has_ci ? c->n_det : 0;
  out->precision = c->precision;
  out->device = c->device;
  if (c->has_ci) {
    out->n_det_up = (int32_t)c->exc[0].size();
    out->n_det_dn = (int32_t)c->exc[1].size();
    for (int sp = 0; sp < 2; sp++)
      for (int d : c->degree[sp]) {
        out->degree_hist[sp][d]++;
        out->max_degree[sp] = std::max(out->max_degree[sp], d);
      }
  }
  return MDET_OK;
}

mdet_status mdet_get_spin_dets(const mdet_ctx* c, int spin, uint64_t* dets, int32_t* degree, int8_t* phase) {
  if (!c || (spin != 0 && spin != 1)) return MDET_E_ARG;
  if (!c->has_ci) return MDET_E_STATE;
  const size_t n = c->exc[spin].size();
  if (dets) std::copy(c->dets[spin].begin(), c->dets[spin].end(), dets);
  for (size_t t = 0; t < n; t++) {
    if (degree) degree[t] = c->degree[spin][t];
    if (phase) phase[t] = c->exc[spin][t].eps;
  }
  return MDET_OK;
}

mdet_status mdet_get_ci_matrix(const mdet_ctx* c, int32_t* row, int32_t* col, double* val) {
  if (!c) return MDET_E_ARG;
  if (!c->has_ci) return MDET_E_STATE;
  if (row) std::copy(c->coo_row.begin(), c->coo_row.end(), row);
  if (col) std::copy(c->coo_col.begin(), c->coo_col.end(), col);
  if (val) std::copy(c->coo_val.begin(), c->coo_val.end(), val);
  return MDET_OK;
}

}  // extern "C"

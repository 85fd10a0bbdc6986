// mdet_preprocess.cu -- the O(N_det) steps of the expansion preprocessing
// (Sec. 2.1) on the GPU: validation, the sort of each spin list by the key of
// Eq. 3, removal of duplicates, the product -> distinct determinant map, and C
// sorted in column-major (the paper's order) and row-major order with segment
// pointers. The work per distinct determinant (excitation records, context
// order) stays on the host and is shared with the host path.
//
// Sorting is a stable LSD radix sort of (64-bit key, index) pairs written here
// (8-bit digits, 8 passes). The order is lexicographic in (key of Eq. 3, last
// word, ..., first word): an LSD sequence of stable 64-bit sorts, first word
// first and the key last, reproduces it exactly, including the original product
// order among identical determinants.

#include <algorithm>
#include <climits>
#include <cmath>

#include "mdet_internal.h"

namespace mdet {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// Smallest failing product index (atomicMin; ULLONG_MAX when none): popcount
// != nel, an occupied MO >= n_mo, or a non-finite coefficient (check_coef).
__global__ void k_validate(int64_t n, int n_int, const uint64_t* __restrict__ D, int nel, int n_mo,
                           const double* __restrict__ coef, unsigned long long* __restrict__ bad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int pc = 0;
  for (int q = 0; q < n_int; q++) pc += __popcll(D[k * n_int + q]);
  const int top = n_mo - 64 * (n_int - 1);
  const bool high = top < 64 && (D[k * n_int + n_int - 1] >> top) != 0;
  const bool badc = coef && !isfinite(coef[k]);
  if (pc != nel || high || badc) atomicMin(bad, (unsigned long long)k);
}

// key[q] of product idx[q]: word `word` of its determinant, or the xor of all
// words (Eq. 3) for word < 0.
__global__ void k_key(int64_t n, int n_int, const uint64_t* __restrict__ D, int word, const int32_t* __restrict__ idx,
                      uint64_t* __restrict__ key) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int64_t k = idx[q];
  uint64_t v = 0;
  if (word < 0) {
    for (int w = 0; w < n_int; w++) v ^= D[k * n_int + w];
  } else {
    v = D[k * n_int + word];
  }
  key[q] = v;
}

// ---- inclusive scan of int32 values ----------------------------------------
// Tiles of kScanTile values (kThreads threads x 4): each tile is scanned in shared
// memory and its total written to sums[tile]; the totals are scanned the same way
// (recursively) and added back to the tiles after the first.
constexpr int kScanPer = 4;
constexpr int kScanTile = kThreads * kScanPer;

__global__ void k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                            int32_t* __restrict__ sums) {
  __shared__ int32_t part[kThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t v[kScanPer];
  int32_t run = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; j++) {
    run += base + j < n ? in[base + j] : 0;
    v[j] = run;
  }
  part[threadIdx.x] = run;
  __syncthreads();
  for (int off = 1; off < kThreads; off <<= 1) {  // Hillis-Steele scan of the thread totals
    const int32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  const int32_t before = threadIdx.x ? part[threadIdx.x - 1] : 0;
#pragma unroll
  for (int j = 0; j < kScanPer; j++)
    if (base + j < n) out[base + j] = v[j] + before;
  if (threadIdx.x == kThreads - 1) sums[blockIdx.x] = part[kThreads - 1];
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ sums) {
  if (blockIdx.x == 0) return;
  const int32_t add = sums[blockIdx.x - 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int j = threadIdx.x; j < kScanTile; j += kThreads)
    if (base + j < n) out[base + j] += add;
}

// int32 scratch that scan_inclusive needs for n values
int64_t scan_scratch(int64_t n) {
  int64_t total = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    total += n;
  }
  return total + 1;
}

// out[i] = in[0] + ... + in[i] (in and out may be the same array)
cudaError_t scan_inclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int32_t* sums = scratch;
  k_scan_tile<<<(unsigned)tiles, kThreads, 0, st>>>(in, out, n, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || tiles == 1) return e;
  if ((e = scan_inclusive(sums, sums, tiles, scratch + tiles, st)) != cudaSuccess) return e;
  k_scan_add<<<(unsigned)tiles, kThreads, 0, st>>>(out, n, sums);
  return cudaGetLastError();
}

// ---- stable LSD radix sort of (uint64 key, int32 value) pairs ----------------
// One pass per 8-bit digit: every block counts the digits of its tile of kThreads
// pairs into counts[digit][block] (digit-major, so that the inclusive scan of the
// flattened array gives each (digit, block) its end offset); then every block moves
// its pairs to offset + rank, the rank being the number of earlier pairs of the tile
// with the same digit (lanes with the same digit found by __match_any_sync, the
// warps before added from shared counts), which keeps equal keys in their order.
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kWarpsPerBlock = kThreads / 32;

__global__ void k_radix_count(const uint64_t* __restrict__ key, int64_t n, int shift, int32_t* __restrict__ counts) {
  __shared__ int32_t c[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kThreads) c[d] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i < n) atomicAdd(&c[(int)((key[i] >> shift) & (kRadix - 1))], 1);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kThreads) counts[(int64_t)d * gridDim.x + blockIdx.x] = c[d];
}

__global__ void k_radix_move(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n, int shift,
                             const int32_t* __restrict__ ends, const int32_t* __restrict__ counts,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int32_t wc[kWarpsPerBlock][kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < kWarpsPerBlock * kRadix; t += kThreads) wc[t / kRadix][t % kRadix] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool live = i < n;
  const uint64_t k = live ? kin[i] : 0;
  const int d = live ? (int)((k >> shift) & (kRadix - 1)) : kRadix;  // kRadix: no pair
  const unsigned same = __match_any_sync(0xffffffffu, d);
  const int rank_w = __popc(same & ((1u << lane) - 1u));
  if (live && rank_w == 0) wc[warp][d] = __popc(same);
  __syncthreads();
  if (!live) return;
  int rank = rank_w;
  for (int q = 0; q < warp; q++) rank += wc[q][d];
  const int64_t cell = (int64_t)d * gridDim.x + blockIdx.x;
  const int64_t pos = (int64_t)ends[cell] - counts[cell] + rank;
  kout[pos] = k;
  vout[pos] = vin[i];
}

// A pair of buffers of which one holds the current data (the role of a double buffer).
template <class T>
struct Buffers {
  T* b[2];
  int sel = 0;
  T* cur() const { return b[sel]; }
  T* alt() const { return b[sel ^ 1]; }
};

// int32 scratch of radix_sort_pairs for n pairs: the counts and their scan, and the scan's own
int64_t sort_scratch(int64_t n) {
  const int64_t cells = (int64_t)kRadix * ((std::max<int64_t>(n, 1) + kThreads - 1) / kThreads);
  return 2 * cells + scan_scratch(cells);
}

// Stable sort of keys.cur() with the values alongside; the result is in keys.cur() and vals.cur()
cudaError_t radix_sort_pairs(Buffers<uint64_t>& keys, Buffers<int32_t>& vals, int64_t n, int32_t* scratch,
                             cudaStream_t st) {
  if (n <= 1) return cudaSuccess;
  const int64_t blocks_n = (n + kThreads - 1) / kThreads;
  const int64_t cells = (int64_t)kRadix * blocks_n;
  int32_t* counts = scratch;
  int32_t* ends = scratch + cells;
  for (int shift = 0; shift < 64; shift += kRadixBits) {
    k_radix_count<<<(unsigned)blocks_n, kThreads, 0, st>>>(keys.cur(), n, shift, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = scan_inclusive(counts, ends, cells, scratch + 2 * cells, st)) != cudaSuccess) return e;
    k_radix_move<<<(unsigned)blocks_n, kThreads, 0, st>>>(keys.cur(), vals.cur(), n, shift, ends, counts, keys.alt(),
                                                          vals.alt());
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    keys.sel ^= 1;
    vals.sel ^= 1;
  }
  return cudaSuccess;
}

__global__ void k_iota(int64_t n, int32_t* __restrict__ v) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) v[q] = (int32_t)q;
}

// flag[q] = 1 where the sorted determinant differs from its predecessor.
__global__ void k_new_det(int64_t n, int n_int, const uint64_t* __restrict__ D, const int32_t* __restrict__ ord,
                          int32_t* __restrict__ flag) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int f = q == 0;
  if (!f) {
    const int64_t a = ord[q], b = ord[q - 1];
    for (int w = 0; w < n_int; w++) f |= D[a * n_int + w] != D[b * n_int + w];
  }
  flag[q] = f;
}

// From the inclusive scan id of the flags: pos[product] = distinct index, and
// first[distinct index] = its first product in the sorted order.
__global__ void k_positions(int64_t n, const int32_t* __restrict__ ord, const int32_t* __restrict__ flag,
                            const int32_t* __restrict__ id, int32_t* __restrict__ pos, int32_t* __restrict__ first) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  pos[ord[q]] = id[q] - 1;
  if (flag[q]) first[id[q] - 1] = ord[q];
}

__global__ void k_gather_dets(int64_t nu, int n_int, const uint64_t* __restrict__ D, const int32_t* __restrict__ first,
                              uint64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu * n_int) return;
  const int64_t u = i / n_int, w = i - u * n_int;
  out[i] = D[(int64_t)first[u] * n_int + w];
}

// Reference product: the largest |c| (bits of a non-negative double order as
// unsigned integers), then the smallest index holding it.
__global__ void k_absmax(int64_t n, const double* __restrict__ c, unsigned long long* __restrict__ best) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) atomicMax(best, (unsigned long long)__double_as_longlong(fabs(c[k])));
}

__global__ void k_first_with(int64_t n, const double* __restrict__ c, const unsigned long long* __restrict__ best,
                             unsigned long long* __restrict__ kmin) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && (unsigned long long)__double_as_longlong(fabs(c[k])) == *best) atomicMin(kmin, (unsigned long long)k);
}

// Per-product context indices and the sort key major * n_minor + minor.
__global__ void k_pair_key(int64_t n, const int32_t* __restrict__ pos_major, const int32_t* __restrict__ ctx_major,
                           const int32_t* __restrict__ pos_minor, const int32_t* __restrict__ ctx_minor,
                           int64_t n_minor, uint64_t* __restrict__ key) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  key[k] = (uint64_t)ctx_major[pos_major[k]] * (uint64_t)n_minor + (uint64_t)ctx_minor[pos_minor[k]];
}

// Sorted pair keys: smallest q whose key repeats its predecessor (a duplicate
// (up, down) product), and the histogram of the major index.
__global__ void k_dup_and_count(int64_t n, const uint64_t* __restrict__ key, int64_t n_minor,
                                unsigned long long* __restrict__ dup, int32_t* __restrict__ count) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  if (q > 0 && key[q] == key[q - 1]) atomicMin(dup, (unsigned long long)q);
  atomicAdd(count + 1 + (int64_t)(key[q] / (uint64_t)n_minor), 1);
}

// C entries in the sorted order: row (up), column (down), value.
__global__ void k_scatter_c(int64_t n, const int32_t* __restrict__ ord, const int32_t* __restrict__ pos_up,
                            const int32_t* __restrict__ ctx_up, const int32_t* __restrict__ pos_dn,
                            const int32_t* __restrict__ ctx_dn, const double* __restrict__ coef,
                            int32_t* __restrict__ row, int32_t* __restrict__ col, double* __restrict__ val) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int64_t k = ord[q];
  row[q] = ctx_up[pos_up[k]];
  col[q] = ctx_dn[pos_dn[k]];
  val[q] = coef[k];
}

}  // namespace

struct PreDevice {
  int64_t n = 0;
  int n_int = 0;
  const uint64_t* det[2] = {nullptr, nullptr};  // caller's arrays
  const double* coef = nullptr;
  int32_t* pos[2] = {nullptr, nullptr};  // product -> distinct index (key order)
  uint64_t *key0 = nullptr, *key1 = nullptr;
  int32_t *v0 = nullptr, *v1 = nullptr, *flag = nullptr, *id = nullptr, *first = nullptr;
  unsigned long long* small = nullptr;  // [4] scalars
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
};

namespace {

#define PRE_TRY(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      *msg = std::string(#call) + " failed: " + cudaGetErrorString(e_);                 \
      return MDET_E_CUDA;                                                               \
    }                                                                                   \
  } while (0)

template <class T>
cudaError_t get(T* host, const T* dev, size_t count, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(host, dev, count * sizeof(T), cudaMemcpyDeviceToHost, st);
  return e != cudaSuccess ? e : cudaStreamSynchronize(st);
}

// Stable sort of the permutation in vals by keys that k_key / k_pair_key wrote
// into keys.cur(); the sorted permutation is vals.cur() afterwards.
cudaError_t sort_pairs(PreDevice* d, Buffers<uint64_t>& keys, Buffers<int32_t>& vals, int64_t n, cudaStream_t st) {
  return radix_sort_pairs(keys, vals, n, static_cast<int32_t*>(d->tmp), st);
}

}  // namespace

mdet_status pre_distinct(PreDevice** h, int64_t n, int n_int, const uint64_t* det_up, const uint64_t* det_dn,
                         const double* coef, int n_up, int n_dn, int n_mo, cudaStream_t st, PreSpin out[2],
                         std::string* msg) {
  PreDevice* d = new PreDevice;
  *h = d;
  d->n = n;
  d->n_int = n_int;
  d->det[0] = det_up;
  d->det[1] = det_dn;
  d->coef = coef;
  const size_t N = (size_t)std::max<int64_t>(n, 1);
  PRE_TRY(cudaMalloc(&d->key0, N * 8));
  PRE_TRY(cudaMalloc(&d->key1, N * 8));
  PRE_TRY(cudaMalloc(&d->v0, N * 4));
  PRE_TRY(cudaMalloc(&d->v1, N * 4));
  PRE_TRY(cudaMalloc(&d->flag, (N + 1) * 4));
  PRE_TRY(cudaMalloc(&d->id, (N + 1) * 4));
  PRE_TRY(cudaMalloc(&d->first, N * 4));
  PRE_TRY(cudaMalloc(&d->pos[0], N * 4));
  PRE_TRY(cudaMalloc(&d->pos[1], N * 4));
  PRE_TRY(cudaMalloc(&d->small, 4 * sizeof(unsigned long long)));
  // int32 scratch of the sorts and scans
  d->tmp_bytes = sizeof(int32_t) * (size_t)std::max(sort_scratch((int64_t)N), scan_scratch((int64_t)N + 1));
  PRE_TRY(cudaMalloc(&d->tmp, d->tmp_bytes));
  // validation: both spin lists, and the coefficients once
  unsigned long long bad[2];
  PRE_TRY(cudaMemsetAsync(d->small, 0xff, 2 * sizeof(unsigned long long), st));
  const int nel[2] = {n_up, n_dn};
  for (int sp = 0; sp < 2; sp++)
    k_validate<<<blocks(n), kThreads, 0, st>>>(n, n_int, d->det[sp], nel[sp], n_mo, sp == 0 ? coef : nullptr,
                                                 d->small + sp);
  PRE_TRY(cudaGetLastError());
  PRE_TRY(get(bad, d->small, 2, st));
  for (int sp = 0; sp < 2; sp++)
    if (bad[sp] != ULLONG_MAX) {
      char buf[200];
      snprintf(buf, sizeof buf,
               "product %llu: the spin %d determinant has the wrong electron count or an MO >= n_mo%s", bad[sp], sp,
               sp == 0 ? ", or its coefficient is not finite" : "");
      *msg = buf;
      return MDET_E_INPUT;
    }
  for (int sp = 0; sp < 2; sp++) {
    const uint64_t* D = d->det[sp];
    Buffers<uint64_t> keys{{d->key0, d->key1}};
    Buffers<int32_t> vals{{d->v0, d->v1}};
    k_iota<<<blocks(n), kThreads, 0, st>>>(n, vals.cur());
    // LSD: first word first, ..., last word, then the key of Eq. 3 (one pass when n_int == 1,
    // where the key is the word)
    const int n_pass = n_int > 1 ? n_int + 1 : 1;
    for (int p = 0; p < n_pass; p++) {
      const int word = p == n_pass - 1 ? -1 : p;
      k_key<<<blocks(n), kThreads, 0, st>>>(n, n_int, D, word, vals.cur(), keys.cur());
      PRE_TRY(cudaGetLastError());
      PRE_TRY(sort_pairs(d, keys, vals, n, st));
    }
    const int32_t* ord = vals.cur();
    k_new_det<<<blocks(n), kThreads, 0, st>>>(n, n_int, D, ord, d->flag);
    PRE_TRY(cudaGetLastError());
    PRE_TRY(scan_inclusive(d->flag, d->id, n, static_cast<int32_t*>(d->tmp), st));
    k_positions<<<blocks(n), kThreads, 0, st>>>(n, ord, d->flag, d->id, d->pos[sp], d->first);
    PRE_TRY(cudaGetLastError());
    int32_t nu = 0;
    PRE_TRY(get(&nu, d->id + (n - 1), 1, st));
    uint64_t* ud = nullptr;
    PRE_TRY(cudaMalloc(&ud, (size_t)nu * n_int * 8));
    k_gather_dets<<<blocks((int64_t)nu * n_int), kThreads, 0, st>>>(nu, n_int, D, d->first, ud);
    out[sp].udets.resize((size_t)nu * n_int);
    cudaError_t e = get(out[sp].udets.data(), ud, (size_t)nu * n_int, st);
    cudaFree(ud);
    PRE_TRY(e);
  }
  // reference product: largest |c|, first index on ties
  PRE_TRY(cudaMemsetAsync(d->small + 2, 0, sizeof(unsigned long long), st));
  PRE_TRY(cudaMemsetAsync(d->small + 3, 0xff, sizeof(unsigned long long), st));
  k_absmax<<<blocks(n), kThreads, 0, st>>>(n, coef, d->small + 2);
  k_first_with<<<blocks(n), kThreads, 0, st>>>(n, coef, d->small + 2, d->small + 3);
  PRE_TRY(cudaGetLastError());
  unsigned long long kref = 0;
  PRE_TRY(get(&kref, d->small + 3, 1, st));
  for (int sp = 0; sp < 2; sp++) {
    int32_t i = 0;
    PRE_TRY(get(&i, d->pos[sp] + kref, 1, st));
    out[sp].iref = i;
  }
  return MDET_OK;
}

mdet_status pre_build_c(PreDevice* d, const std::vector<int32_t> ctx_of[2], int64_t nup, int64_t ndn,
                        cudaStream_t st, PreC* out, std::string* msg) {
  const int64_t n = d->n;
  int32_t* ctx[2] = {nullptr, nullptr};
  int32_t *row = nullptr, *col = nullptr, *cnt = nullptr;
  double* val = nullptr;
  mdet_status s = MDET_OK;
  auto run = [&]() -> mdet_status {
    for (int sp = 0; sp < 2; sp++) {
      PRE_TRY(cudaMalloc(&ctx[sp], std::max<size_t>(ctx_of[sp].size(), 1) * 4));
      PRE_TRY(cudaMemcpyAsync(ctx[sp], ctx_of[sp].data(), ctx_of[sp].size() * 4, cudaMemcpyHostToDevice, st));
    }
    PRE_TRY(cudaMalloc(&row, (size_t)n * 4));
    PRE_TRY(cudaMalloc(&col, (size_t)n * 4));
    PRE_TRY(cudaMalloc(&val, (size_t)n * 8));
    PRE_TRY(cudaMalloc(&cnt, (size_t)(std::max(nup, ndn) + 1) * 4));
    // pass 0: column-major (Sec. 2.1, key N_up * j + i); pass 1: row-major (key N_dn * i + j)
    for (int pass = 0; pass < 2; pass++) {
      const int major = pass == 0 ? 1 : 0, minor = 1 - major;
      const int64_t n_major = pass == 0 ? ndn : nup, n_minor = pass == 0 ? nup : ndn;
      Buffers<uint64_t> keys{{d->key0, d->key1}};
      Buffers<int32_t> vals{{d->v0, d->v1}};
      k_iota<<<blocks(n), kThreads, 0, st>>>(n, vals.cur());
      k_pair_key<<<blocks(n), kThreads, 0, st>>>(n, d->pos[major], ctx[major], d->pos[minor], ctx[minor], n_minor,
                                                 keys.cur());
      PRE_TRY(cudaGetLastError());
      PRE_TRY(sort_pairs(d, keys, vals, n, st));
      PRE_TRY(cudaMemsetAsync(cnt, 0, (size_t)(n_major + 1) * 4, st));
      PRE_TRY(cudaMemsetAsync(d->small, 0xff, sizeof(unsigned long long), st));
      k_dup_and_count<<<blocks(n), kThreads, 0, st>>>(n, keys.cur(), n_minor, d->small, cnt);
      PRE_TRY(cudaGetLastError());
      if (pass == 0) {
        unsigned long long dup = 0;
        PRE_TRY(get(&dup, d->small, 1, st));
        if (dup != ULLONG_MAX) {
          int32_t pair[2];
          PRE_TRY(get(pair, vals.cur() + (dup - 1), 2, st));
          char buf[160];
          snprintf(buf, sizeof buf, "products %d and %d repeat the same (up, down) pair", pair[0], pair[1]);
          *msg = buf;
          return MDET_E_INPUT;
        }
      }
      // counts -> segment starts (cnt[0] = 0): an inclusive scan into id
      PRE_TRY(scan_inclusive(cnt, d->id, n_major + 1, static_cast<int32_t*>(d->tmp), st));
      k_scatter_c<<<blocks(n), kThreads, 0, st>>>(n, vals.cur(), d->pos[0], ctx[0], d->pos[1], ctx[1], d->coef,
                                                  row, col, val);
      PRE_TRY(cudaGetLastError());
      std::vector<int32_t>& r = pass == 0 ? out->csc_row : out->csr_row;
      std::vector<int32_t>& c = pass == 0 ? out->csc_col : out->csr_col;
      std::vector<double>& v = pass == 0 ? out->csc_val : out->csr_val;
      std::vector<int32_t>& p = pass == 0 ? out->csc_ptr : out->csr_ptr;
      r.resize(n);
      c.resize(n);
      v.resize(n);
      p.resize(n_major + 1);
      PRE_TRY(cudaMemcpyAsync(r.data(), row, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
      PRE_TRY(cudaMemcpyAsync(c.data(), col, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
      PRE_TRY(cudaMemcpyAsync(v.data(), val, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
      PRE_TRY(get(p.data(), d->id, (size_t)(n_major + 1), st));
    }
    return MDET_OK;
  };
  s = run();
  cudaFree(ctx[0]);
  cudaFree(ctx[1]);
  cudaFree(row);
  cudaFree(col);
  cudaFree(val);
  cudaFree(cnt);
  return s;
}

void pre_free(PreDevice* d) {
  if (!d) return;
  for (void* p : {(void*)d->key0, (void*)d->key1, (void*)d->v0, (void*)d->v1, (void*)d->flag, (void*)d->id,
                  (void*)d->first, (void*)d->pos[0], (void*)d->pos[1], (void*)d->small, d->tmp})
    if (p) cudaFree(p);
  delete d;
}

}  // namespace mdet

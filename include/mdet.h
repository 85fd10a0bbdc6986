/*
 * mdet.h -- C ABI of the GB300 multideterminant wavefunction library.
 *
 * The library evaluates a large multideterminant trial wavefunction
 *   Psi(R) = sum_k c_k D^up_k(R_up) D^dn_k(R_dn) = D_up^T C D_dn      (Eqs. 1-2)
 * together with grad_i Psi / Psi and Lap_i Psi / Psi for every electron and
 * the local energy, for a batch of walkers per call (Sec. 2 and Sec. 4: one
 * Monte Carlo step computes Psi, the drift vector and the local energy).
 *
 * Conventions shared by every entry point:
 *  - Electrons 0 .. n_up-1 are spin up, n_up .. n_up+n_dn-1 spin down, and
 *    n_up >= n_dn >= 1 (the convention of Sec. 2.4).
 *  - A determinant of one spin is a bit string of n_int = ceil(n_mo / 64)
 *    64-bit words; bit (m mod 64) of word (m div 64) is set when MO m
 *    (0-based) is occupied (Sec. 2.1, "Encoding"). Its Slater matrix lists the
 *    occupied MOs in ascending order: [S]_{i a} = phi_{o_a}(r_i), o_1 < o_2 < ...
 *  - Positions and all floating-point outputs are double precision.
 *  - "device pointer": memory the caller allocated on the context's device
 *    (for instance a torch CUDA tensor); "host pointer": ordinary host memory.
 *  - Every set_* call deep-copies its inputs; the caller keeps ownership of
 *    every buffer it passes. The context owns its device copies and scratch.
 *  - Functions return an mdet_status; no exception or abort crosses the ABI.
 *    On error mdet_last_error() describes the failure.
 *  - A context is not re-entrant: one thread and one stream at a time.
 */
#ifndef MDET_H
#define MDET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdet_ctx mdet_ctx;

typedef enum {
  MDET_OK = 0,
  MDET_E_ARG = 1,      /* bad argument (null pointer, negative size, size beyond a limit) */
  MDET_E_STATE = 2,    /* call order violated (e.g. evaluate before set_ci_expansion) */
  MDET_E_OOM = 3,      /* host or device allocation failed */
  MDET_E_CUDA = 4,     /* a CUDA runtime call or kernel launch failed */
  MDET_E_INPUT = 5,    /* malformed expansion: wrong popcount, bits beyond n_mo, duplicate product */
  MDET_E_TIMEOUT = 6,  /* a bounded device-side wait gave up */
  MDET_E_NODEVICE = 7  /* the context has no device (created with device = MDET_NO_DEVICE) */
} mdet_status;

/* Arithmetic of the evaluation. */
enum {
  MDET_PRECISION_FP64 = 0,  /* every step in FP64 */
  MDET_PRECISION_MIXED = 1  /* FP32 orbitals/tables/ratios; FP64 reference LU, log|D0| and CI contraction */
};

/* Device number meaning "no GPU": host preprocessing and introspection only. */
#define MDET_NO_DEVICE (-1)

/* Limits of this implementation. */
#define MDET_MAX_SPIN_ELEC 32   /* n_up, n_dn <= 32 */
#define MDET_MAX_MO 255         /* n_mo <= 255 */
#define MDET_MAX_L 3            /* s, p, d, f shells */
#define MDET_MAX_EXC 4          /* excitation degree of a spin determinant relative to the reference */

/* Per-walker status bits written by mdet_evaluate. */
#define MDET_WS_REF_SINGULAR 0x1u   /* a reference Slater matrix had a zero pivot: outputs are NaN */
#define MDET_WS_REF_ILLCOND 0x2u    /* reference pivot ratio below 1e-13: results may lose accuracy */
#define MDET_WS_PSI_ZERO 0x4u       /* Psi == 0 (walker on the nodal surface): log = -inf, sign 0, ratios NaN */
#define MDET_WS_NONFINITE 0x8u      /* an output is Inf or NaN */
#define MDET_WS_FALLBACK 0x10u      /* the ratio-table result was estimated too inaccurate (or the
                                       reference singular): the walker was re-evaluated by full LU
                                       of every determinant (see mdet_set_fallback) */
#define MDET_WS_ESCALATED 0x20u     /* mixed precision: the walker's estimate exceeded the tolerance
                                       and it was re-evaluated by the FP64 ratio table (and, with
                                       MDET_WS_FALLBACK, then by full LU; see mdet_set_fallback) */

typedef struct {
  int32_t n_up, n_dn, n_ao, n_mo, n_int;
  int64_t n_det;            /* products (nonzeros of C) */
  int32_t n_det_up, n_det_dn;  /* distinct spin determinants (Sec. 1, N_det^sigma) */
  int32_t max_degree[2];    /* largest excitation degree per spin */
  int64_t degree_hist[2][MDET_MAX_EXC + 1];  /* spin determinants per excitation degree (cf. Table 4) */
  int32_t precision;
  int32_t device;
} mdet_stats;

/* Create a context on CUDA device `device` (or MDET_NO_DEVICE) with the given
 * precision. *out receives the context; destroy it with mdet_destroy. */
mdet_status mdet_create(mdet_ctx** out, int device, int precision);

/* Release the context and every device buffer it owns. Null is ignored. */
void mdet_destroy(mdet_ctx* ctx);

/* Static description of a status code. */
const char* mdet_status_string(mdet_status s);

/* Detail of the last failure on this context (empty string if none). */
const char* mdet_last_error(const mdet_ctx* ctx);

/*
 * The molecular system (Eq. 1: electron counts per spin; the nuclei enter the
 * local energy's potential). Z: [n_nuc] charges, xyz: [n_nuc][3] positions,
 * host pointers. Requires 1 <= n_dn <= n_up <= MDET_MAX_SPIN_ELEC.
 * Invalidates any expansion already set (it fixes the determinant popcounts).
 */
mdet_status mdet_set_system(mdet_ctx* ctx, int n_up, int n_dn, int n_nuc,
                            const double* Z, const double* xyz);

/*
 * Orbitals (Sec. 2, first paragraph: MOs and their gradients and Laplacian at
 * every electron). Basis: n_shell contracted Cartesian Gaussian shells; shell s
 * has angular momentum shell_l[s] in 0..3, is centred on nucleus
 * shell_center[s] and has shell_nprim[s] primitives whose exponents and
 * contraction coefficients are consecutive entries of alpha / coef (all
 * shells concatenated). Its (l+1)(l+2)/2 AOs are x^a y^b z^c R(r), a+b+c = l,
 * ordered a descending then b descending (xx, xy, xz, yy, yz, zz), with
 * R(r) = sum_p coef_p exp(-alpha_p r^2) (normalisation is part of coef).
 * mo_coef: [n_ao][n_mo] column-major (mo_coef[mu + n_ao*m]), phi_m = sum_mu
 * mo_coef[mu, m] chi_mu. All host pointers. Requires set_system first and
 * n_mo <= MDET_MAX_MO.
 */
mdet_status mdet_set_orbitals(mdet_ctx* ctx, int n_shell, const int32_t* shell_l,
                              const int32_t* shell_center, const int32_t* shell_nprim,
                              const double* alpha, const double* coef,
                              int n_mo, const double* mo_coef);

/*
 * The CI expansion (Eq. 1) and its preprocessing (Sec. 2.1), on the host:
 * the spin determinants of each spin are sorted by the key of Eq. 3 with a
 * radix sort and deduplicated; C becomes a sparse matrix over the distinct
 * determinants ordered column by column (key N_up*(j-1)+i); each distinct
 * determinant is stored as its excitation (holes, particles, phase) relative
 * to the reference determinant of its spin, the spin part of the largest |c_k|
 * product, and the list is grouped by excitation degree.
 * det_up, det_dn: [n_det][n_int] host bit strings; coef: [n_det] host.
 * Fails with MDET_E_INPUT on a wrong popcount, a bit at or beyond n_mo, a
 * duplicate (up, dn) product, or a degree above MDET_MAX_EXC. Requires
 * set_system and set_orbitals (n_int must equal ceil(n_mo/64)).
 */
mdet_status mdet_set_ci_expansion(mdet_ctx* ctx, int64_t n_det, int n_int,
                                  const uint64_t* det_up, const uint64_t* det_dn,
                                  const double* coef);

/*
 * The paper's own route to the determinant values (Sec. 2.2), for comparison
 * with the table method of mdet_evaluate. For every walker and spin the
 * distinct determinants are visited in the order of the key of Eq. 3. The
 * first one is inverted in full (Gauss-Jordan, partial pivoting). Each next
 * one is reached from its predecessor by in-place Sherman-Morrison column
 * substitutions (Eq. 4), one column at a time, holes and particles paired in
 * ascending order. A substitution with |ratio| < 1e-3 is deferred and retried
 * after the others; a round that applies none of the remaining ones cancels the
 * updates and the determinant is inverted in full. All in FP64, on the orbital
 * values of the last mdet_evaluate of this context (n_walk at most its walker
 * count). Outputs (device): r [n_det_up + n_det_dn][ld] walker-minor, the
 * ratios D_I / D_ref in the context's order (mdet_get_spin_dets) relative to
 * that evaluation's reference determinants; n_inv, n_subst [n_walk]: full
 * inversions and applied substitutions over both spins (Table 3's N_inv and
 * N_subst). Asynchronous on `stream` (waits for the evaluation's stream if it
 * differs). Errors: MDET_E_STATE without an expansion or for too many walkers,
 * MDET_E_ARG for null outputs or ld < n_walk.
 */
mdet_status mdet_sm_chain(mdet_ctx* ctx, int64_t n_walk, double* r, int64_t ld, int32_t* n_inv, int32_t* n_subst,
                          void* stream);

/*
 * The same expansion and preprocessing with the O(N_det) steps on the GPU:
 * validation, the sort of each spin list by the key of Eq. 3 (ties broken by
 * the words from the last to the first, original order among identical
 * determinants), removal of duplicates, the product -> distinct determinant
 * map, the reference product and C in column-major and row-major order with
 * segment pointers. The steps per distinct determinant (excitation records,
 * degree grouping) run on the host, as in mdet_set_ci_expansion. The resulting
 * context state is identical to mdet_set_ci_expansion's. det_up, det_dn, coef:
 * DEVICE arrays of the context's device in the same layout, only read; the
 * call is synchronous on `stream`. Fails like mdet_set_ci_expansion, also with
 * MDET_E_INPUT for a non-finite coefficient, and with MDET_E_NODEVICE on a
 * context without a device.
 */
mdet_status mdet_set_ci_expansion_device(mdet_ctx* ctx, int64_t n_det, int n_int, const uint64_t* det_up,
                                         const uint64_t* det_dn, const double* coef, void* stream);

/*
 * One evaluation of the hot path for n_walk walkers (Sec. 2.2-2.4): orbitals,
 * reference LU per spin, ratio tables, per-determinant ratios and their
 * derivative contributions, the sparse bilinear contraction, and the
 * epilogue. Asynchronous on `stream` (a cudaStream_t, or null for the legacy
 * default stream); all pointers are device pointers on the context's device:
 *   R            [n_walk][n_up+n_dn][3]  positions (input)
 *   log_abs_psi  [n_walk]   log|Psi|
 *   sign         [n_walk]   sign of Psi (-1, 0, +1)
 *   grad         [n_walk][n_up+n_dn][3]  grad_i Psi / Psi
 *   lap          [n_walk][n_up+n_dn]     Lap_i Psi / Psi
 *   e_local      [n_walk]   local energy (may be null)
 *   status       [n_walk]   MDET_WS_* bits (may be null)
 * n_walk = 0 is a no-op. Scratch grows to the largest n_walk seen (a
 * synchronous allocation on first use at a new size).
 */
mdet_status mdet_evaluate(mdet_ctx* ctx, int64_t n_walk, const double* R,
                          double* log_abs_psi, int8_t* sign, double* grad, double* lap,
                          double* e_local, uint32_t* status, void* stream);

/*
 * The same evaluation from and to HOST memory: copies R to the device, runs
 * mdet_evaluate on the context's internal stream, copies every output back
 * and synchronises. Output pointers may be null to skip that copy (except
 * log_abs_psi). Pinned host memory makes the copies faster but is not required.
 */
mdet_status mdet_evaluate_host(mdet_ctx* ctx, int64_t n_walk, const double* R,
                               double* log_abs_psi, int8_t* sign, double* grad, double* lap,
                               double* e_local, uint32_t* status);

/*
 * Intermediate values of the last mdet_evaluate on this context, copied to
 * host memory for inspection: r_up [n_walk][n_det_up] and r_dn
 * [n_walk][n_det_dn] are the ratios D_I / D_ref of every distinct spin
 * determinant (in the context's order, see mdet_get_spin_dets), log_d0
 * [n_walk][2] and sign_d0 [n_walk][2] the reference determinants. Any pointer
 * may be null. Synchronises the stream of the last evaluation.
 */
mdet_status mdet_get_ratios(mdet_ctx* ctx, int64_t n_walk, double* r_up, double* r_dn,
                            double* log_d0, int8_t* sign_d0);

/*
 * Stability control (the paper's O(N^3) fallback of Sec. 2.2, adapted to the
 * ratio table). Every determinant ratio of the table carries a relative error
 * of about u cond_1(S_ref), with u the unit roundoff of the table arithmetic
 * (2^-53 FP64, about 2^-47 double-float) and cond_1(S_ref) = |S_ref|_1
 * |S_ref^-1|_1 of the walker's reference Slater matrix. The estimate of the
 * walker's relative error is u cond_1(S_ref) C kappa_Psi: C the cancellation
 * ratio of its gradient and Laplacian sums (sum of |terms| / max(|result|, rms
 * over the walker's electrons)), kappa_Psi = sum_ij |c_ij D_up,i D_dn,j| / |Psi|
 * the conditioning of the CI sum (mdet_get_error_estimates: the l1 form and a
 * form with the terms added in quadrature). A walker whose l1 estimate exceeds
 * tol (default 1e-5 for mixed, 1e-8 for FP64 precision: the accuracy target of
 * each path), or whose reference is singular, is re-evaluated on the GPU in FP64
 * by LU of every distinct determinant, its own contraction and epilogue; its
 * status gets MDET_WS_FALLBACK. With mixed precision the flagged walkers may
 * first be re-evaluated by the FP64 ratio table (mdet_set_escalation), whose
 * estimate is 2^6 smaller; only those still above tol then go through full LU.
 * At most max_walkers walkers per evaluation are re-evaluated (default 256 for
 * mixed, 512 for FP64; the scratch grows with it); further ones keep the table
 * result and MDET_WS_REF_ILLCOND. tol <= 0 disables the fallback. Supported for
 * n_up, n_dn <= MDET_FALLBACK_MAX_SPIN. The re-evaluation runs on the stream of
 * mdet_evaluate after the walker chunks, with no host wait. Errors: MDET_E_ARG
 * for a null context or max_walkers outside 1..65535. A new cap frees the
 * scratch, which the next evaluation allocates again.
 */
#define MDET_FALLBACK_MAX_SPIN 17
mdet_status mdet_set_fallback(mdet_ctx* ctx, double tol, int max_walkers);
/*
 * Norm-based truncation of a CI expansion (Sec. 3). Host call, no context.
 * The expansion is given as products (det_up[k], det_dn[k], coef[k]), k < n_det,
 * in the layout of mdet_set_ci_expansion (host pointers). The squared norm
 * decomposes over the distinct spin determinants:
 *   sum_k c_k^2 = sum_i N_i^up = sum_j N_j^dn,
 * where N_i^up is the sum of c_k^2 over the products whose up determinant is
 * D_i^up, and likewise for down. Every distinct determinant with
 * N_i^up <= eps_up (N_j^dn <= eps_dn) is removed. All removals use the norms of
 * the untruncated expansion, and every product that uses a removed determinant
 * is dropped; the kept coefficients are not renormalised. eps < 0 removes
 * nothing of that spin.
 * Outputs, each nullable:
 *  - keep[k] = 1 for a kept product, else 0;
 *  - norm_up[k] / norm_dn[k] = the norms of product k's two determinants;
 *  - counts[5] = {kept products, distinct up determinants in kept products,
 *    distinct down determinants in kept products, distinct up determinants,
 *    distinct down determinants}.
 * Norms are summed with Neumaier compensation in product order.
 * Errors: MDET_E_ARG for a negative n_det, n_int < 1 or null input arrays.
 */
mdet_status mdet_truncate_norm(int64_t n_det, int n_int, const uint64_t* det_up, const uint64_t* det_dn,
                               const double* coef, double eps_up, double eps_dn, uint8_t* keep, double* norm_up,
                               double* norm_dn, int64_t* counts);

/*
 * Escalation of flagged mixed-precision walkers to the FP64 ratio table before
 * the full-LU path: MDET_ESCALATE_AUTO (default) takes it when full LU is the
 * costlier (distinct determinants x n^3 above 1e6, n the larger spin count, or
 * inside a batch); MDET_ESCALATE_ALWAYS and MDET_ESCALATE_NEVER force the
 * choice. Escalated walkers get MDET_WS_ESCALATED. No effect on FP64 contexts.
 * The choice is made when an evaluation is enqueued (a captured batch keeps the
 * one it was captured with). Errors: MDET_E_ARG for a null context or another
 * mode.
 */
#define MDET_ESCALATE_AUTO 0
#define MDET_ESCALATE_ALWAYS 1
#define MDET_ESCALATE_NEVER 2
mdet_status mdet_set_escalation(mdet_ctx* ctx, int mode);

/* The current fallback tolerance and walker cap (host pointers). */
mdet_status mdet_get_fallback(const mdet_ctx* ctx, double* tol, int* max_walkers);

/*
 * Walker chunking of the mixed-precision evaluation: a batch is cut into
 * n_chunks chunks (multiples of 256 walkers) pipelined over two streams of the
 * context, forked from and joined back to the caller's stream. One stream runs
 * the FP32-pipe stages in order (orbitals, reference tables and ratios of each
 * chunk; the epilogue of each chunk once it is contracted), the other, of
 * higher priority, the FP64 contractions one after another on a persistent grid
 * that leaves part of every SM free. So the contraction of chunk k overlaps the
 * orbitals and tables of chunk k+1 and the epilogue of chunk k-1. 0 selects the
 * automatic choice (3 chunks with the FP64 contraction, at least 100,000
 * products and 3,072 walkers; otherwise 1), 1 disables the overlap. Values
 * above 8 are clamped, and so are values above the number of 256-walker tiles.
 * The FP64 path always runs as one chunk on the caller's stream.
 */
mdet_status mdet_set_walker_chunks(mdet_ctx* ctx, int n_chunks);

/* The walker chunks the last mdet_evaluate of this context was cut into and the
 * kernels it launched (memset and copy operations not counted); 0 before the
 * first evaluation. Either pointer may be null. */
mdet_status mdet_get_last_launches(const mdet_ctx* ctx, int32_t* n_chunks, int32_t* n_kernels);

/*
 * Tile shapes of the evaluation kernels (tuning knobs with no counterpart in
 * the paper): spmm_chunk nonzeros of C per warp in the contraction (64..8192),
 * mo_ec electrons per thread block in the orbital kernels (4, 6 or 8),
 * walker_chunks as in mdet_set_walker_chunks, spmm_blocks the grid of the FP64
 * contraction (0: one warp per work item with one chunk, 4 blocks per SM with
 * several; otherwise a persistent grid of at most that many 128-thread blocks
 * whose warps draw work items from a counter), mo_impl the mixed-precision
 * orbital product (2, the default: exact BF16 digit products on the tcgen05
 * tensor cores with TMEM accumulators, accurate to about 2^-55 of the row and
 * column maxima, for at most 112 AOs and 128 MOs, beyond which it falls back to
 * 1; 1: the compensated FP32 dot product on the CUDA cores, accurate relative to
 * each term; 0: the same digit products on warp-level mma.sync),
 * contract_impl the CI contraction of the mixed path (0, the default: FP64;
 * 1: double-float pairs on the FP32 pipe with a compensated dot product, an
 * option outside the FP64 contraction of the method's precision plan).
 * Defaults: spmm_chunk 512, mo_ec 4 (mixed) or 6 (FP64), walker_chunks 0,
 * spmm_blocks 0, mo_impl 2, contract_impl 0.
 * best_ms and trials are filled by mdet_autotune (the fastest step time seen
 * and the configurations timed).
 */
typedef struct {
  int32_t spmm_chunk;
  int32_t mo_ec;
  int32_t walker_chunks;
  float best_ms;
  int32_t trials;
  int32_t spmm_blocks;
  int32_t mo_impl;
  int32_t contract_impl;
} mdet_tuning;

mdet_status mdet_get_tuning(const mdet_ctx* ctx, mdet_tuning* out);
mdet_status mdet_set_tuning(mdet_ctx* ctx, const mdet_tuning* in);

/*
 * Autotuner: times full evaluations of the n_walk walkers at R (device
 * pointer, [n_walk][n_up+n_dn][3]) with CUDA events on the context's stream and
 * picks the tile shapes by coordinate descent over spmm_chunk in
 * {256, 512, 1024, 2048}, mo_ec in {4, 6, 8} and (mixed precision)
 * walker_chunks in {1, 2, 3, 4}, stopping when budget_ms of GPU time is spent.
 * The winner is stored in the context and returned in *out (may be null).
 * Allocates temporary output buffers; synchronous.
 */
mdet_status mdet_autotune(mdet_ctx* ctx, int64_t n_walk, const double* R, double budget_ms, mdet_tuning* out);

/*
 * Batched evaluation of several independent expansions (contexts) on one
 * device, e.g. wavefunctions of different systems or states, of uneven sizes.
 * Per context i: n_walk[i] walkers at R[i] and output pointers as in
 * mdet_evaluate (e_local[i] / status[i] may be null; the arrays e_local and
 * status themselves may be null). Contexts are spread over n_streams streams
 * (1..16) by longest-processing-time-first on a cost estimate, so small and
 * large expansions share the GPU.
 *
 * mdet_batch_evaluate launches directly, forked from and joined to `stream`.
 * mdet_batch_create records the same launches once into a CUDA graph (after
 * one uncaptured warm-up evaluation that sizes every context's scratch), and
 * mdet_batch_launch replays all evaluations as one graph launch on `stream`.
 * The pointers given to mdet_batch_create are baked into the graph: refill the
 * same R buffers between launches. A batch must be destroyed before its
 * contexts, and a context's tuning, fallback cap or size must not change while
 * a batch refers to it (each may reallocate the scratch the graph points to).
 */
typedef struct mdet_batch mdet_batch;
mdet_status mdet_batch_evaluate(int n_ctx, mdet_ctx* const* ctxs, const int64_t* n_walk, const double* const* R,
                                double* const* log_abs_psi, int8_t* const* sign, double* const* grad,
                                double* const* lap, double* const* e_local, uint32_t* const* status,
                                int n_streams, void* stream);
mdet_status mdet_batch_create(mdet_batch** out, int n_ctx, mdet_ctx* const* ctxs, const int64_t* n_walk,
                              const double* const* R, double* const* log_abs_psi, int8_t* const* sign,
                              double* const* grad, double* const* lap, double* const* e_local,
                              uint32_t* const* status, int n_streams);
mdet_status mdet_batch_launch(mdet_batch* b, void* stream);
void mdet_batch_destroy(mdet_batch* b);

/*
 * Stage timing. With profiling mode 1, every mdet_evaluate records a CUDA event
 * before and after each stage on the stream that runs it; mdet_get_profile
 * waits for them and writes the durations in milliseconds of the last
 * evaluation, in the order MDET_STAGE_* below (ms: [MDET_N_STAGES]), summed
 * over walker chunks (with chunks the stages of different chunks overlap, so
 * the sum can exceed the step time). Events in the streams of the pipelined
 * walker chunks shift the chunks' overlap: they lengthen the step by about a
 * tenth. Mode 2 therefore records no event: the contraction kernels write the
 * GPU's global timer (ns) at their first block's start and their last warp's
 * exit into words of the context's scratch, and mdet_get_profile returns the
 * sum of those launch durations as the contraction entry (the other entries
 * stay zero). 0 (the default) records nothing. MDET_E_ARG for another mode.
 * mdet_get_profile waits for the last evaluation's stream (mode 2) or events.
 */
enum {
  MDET_STAGE_ORBITALS = 0,  /* AO values and AO->MO product (Sec. 2) */
  MDET_STAGE_REFERENCE = 1, /* reference LU, inverse, tables (Sec. 2.2, Sec. 5) */
  MDET_STAGE_RATIOS = 2,    /* determinant ratios (Sec. 2.2) */
  MDET_STAGE_ZERO = 3,      /* clearing of the contraction accumulators */
  MDET_STAGE_CONTRACT = 4,  /* sparse bilinear contraction (Sec. 2.4) */
  MDET_STAGE_FINAL = 5,     /* derivative aggregation and epilogue (Sec. 2.3) */
  MDET_N_STAGES = 6
};
mdet_status mdet_set_profiling(mdet_ctx* ctx, int enable);
mdet_status mdet_get_profile(mdet_ctx* ctx, float* ms);

/*
 * Timeline of the last profiled evaluation (tracing; no counterpart in the
 * paper): ms[k][i][0..1] (k < MDET_MAX_CHUNKS, i < MDET_N_STAGES) are the start
 * and end of stage i of walker chunk k, then ms[2 * MDET_MAX_CHUNKS *
 * MDET_N_STAGES + 0..2] the start and end of the stability refinement and the
 * end of the evaluation, all in milliseconds after the evaluation's first event
 * on the caller's stream. *n_chunks receives the chunks used; entries of
 * unused chunks are zero. ms must hold 2 * MDET_MAX_CHUNKS * MDET_N_STAGES + 3
 * floats. Waits for the evaluation's last event. MDET_E_STATE unless the last
 * evaluation ran with profiling mode 1.
 */
#define MDET_MAX_CHUNKS 8
mdet_status mdet_get_timeline(mdet_ctx* ctx, int32_t* n_chunks, float* ms);

/*
 * Psi~ = r_up . (C r_dn) per walker, without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they call it (a pooled or custom device
 * allocator that owns all of the GPU's memory, or a runtime that forbids
 * allocation after start-up). It runs a segmented product over the
 * row-ordered copy of C whose output v = C r_dn is walker-minor like its input
 * (a form of its own: mdet_evaluate's contraction writes v walker-major into
 * the context's scratch) on ratios the caller supplies, keeping v in a static
 * device array of MDET_NOALLOC_SCRATCH_DOUBLES doubles (32 MiB) that every GPU
 * loading this library holds until the process exits.
 *   r          device, [n_det_up + n_det_dn][ld] walker-minor ratios D_I / D_ref
 *              of the distinct determinants in the context's order (up block,
 *              then down block; mdet_get_ratios gives them walker-major),
 *              16-byte aligned; ld a multiple of 128 and >= n_walk
 *   psi_tilde  device, [n_walk]: Psi / (D_ref_up D_ref_dn)
 * Asynchronous on `stream`; the caller's current device is restored before
 * return. Fails with MDET_E_ARG when (n_det_up + 1) * ld exceeds
 * MDET_NOALLOC_SCRATCH_DOUBLES (checked without forming the product, so any ld
 * is safe to pass). The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress). Every
 * call shares the one array and leaves its contents behind; it clears what it
 * uses before use, and calls that overlap on the GPU (other streams, other
 * threads) race.
 */
#define MDET_NOALLOC_SCRATCH_DOUBLES (4u * 1024u * 1024u)
mdet_status mdet_psi_tilde_noalloc(mdet_ctx* ctx, int64_t n_walk, const double* r, int64_t ld,
                                   double* psi_tilde, void* stream);

/*
 * Measured FP64 FMA throughput of a device, the roofline denominator of the
 * FP64 kernels (the CI contraction of Sec. 2.4 is bound by this pipe). The paper
 * has no counterpart; it quotes CPU cycle counts instead (Sec. 5).
 * Every thread of a grid of 4 blocks of 128 threads per SM keeps 8 independent
 * accumulators a_j <- fma(c, x_j, a_j), with a new multiplier c and operands x_j
 * read each step from small L1-resident tables (the pattern of a sparse
 * contraction, which fills the pipe better than register-only FMA streams),
 * for fma_per_thread FMAs (a multiple of 32); one warm-up launch, then `reps`
 * timed launches (CUDA events), the fastest kept.
 *   tflops   out: 2 * FMAs / best time, in TFLOP/s
 *   best_ms  out (nullable): the fastest launch's time
 *   sm_mhz   out (nullable): SM clock during that launch (clock64 cycles over
 *            global-timer nanoseconds of one block)
 * Synchronous. Allocates small tables and output buffers and frees them; the
 * caller's current device is restored. MDET_E_ARG on a null tflops,
 * fma_per_thread < 32 or reps < 1; MDET_E_CUDA on any CUDA error.
 */
mdet_status mdet_measure_fp64_rate(int device, int64_t fma_per_thread, int reps, double* tflops, double* best_ms,
                                   double* sm_mhz);

/*
 * Diagnostic of the double-float arithmetic used by the mixed path: for n
 * device values x_i <= 0, y_df[i] = double-float exp(x_i), y_ref[i] = FP64
 * exp(x_i), prod_df[i] = double-float x_i * x_{(i+1) mod n} + x_i (all device
 * pointers). Synchronous.
 */
mdet_status mdet_selftest_df32(int device, int64_t n, const double* x, double* y_df, double* y_ref,
                               double* prod_df);

/*
 * Diagnostic of the reciprocal square root in the local energy's Coulomb sums
 * (Sec. 4, E_L): for n device values x_i, y_nr[i] = the epilogue's 1/sqrt(x_i)
 * (an FP32 estimate refined by two Newton-Raphson steps in FP64) and y_ref[i] =
 * CUDA's FP64 1.0 / sqrt(x_i) (all device pointers, n doubles each). Synchronous.
 * MDET_E_ARG for n < 1, a null pointer or a negative device; MDET_E_CUDA when the
 * launch fails.
 */
mdet_status mdet_selftest_inv_r(int device, int64_t n, const double* x, double* y_nr, double* y_ref);

/*
 * Diagnostics of the last evaluation (host copies, synchronises its stream):
 * cond1 [n_walk][2], cond_1 of the reference Slater matrix of each spin;
 * est [n_walk][2], the first-order error estimates of the walker's table
 * result: u cond_1 times the cancellation ratio of its derivative sums times
 * the conditioning of its CI sum, with the terms summed in magnitude
 * (est[w][0], the one mdet_set_fallback compares with its tolerance) and in
 * quadrature (est[w][1]). Either pointer may be null. Meaningful when the
 * fallback is enabled.
 */
mdet_status mdet_get_error_estimates(mdet_ctx* ctx, int64_t n_walk, double* cond1, double* est);

/* Sizes and excitation statistics (host only; works without a device). */
mdet_status mdet_get_stats(const mdet_ctx* ctx, mdet_stats* out);

/*
 * The distinct determinants of one spin (0 up, 1 down) in the context's
 * order (reference first, then by excitation degree, then by the key of
 * Eq. 3): dets [n][n_int] bit strings, degree [n], phase [n] (the sign that
 * turns the reference-ordered substituted matrix into the ascending one).
 * Any pointer may be null. Host only.
 */
mdet_status mdet_get_spin_dets(const mdet_ctx* ctx, int spin, uint64_t* dets, int32_t* degree,
                               int8_t* phase);

/*
 * The sparse C matrix over the distinct determinants in the paper's column-
 * major order (Sec. 2.1): row[k] (up index), col[k] (down index), val[k],
 * k < n_det. Host only.
 */
mdet_status mdet_get_ci_matrix(const mdet_ctx* ctx, int32_t* row, int32_t* col, double* val);

/*
 * The sort of Sec. 2.1 on its own: order[] receives the permutation that
 * sorts n bit-string determinants [n][n_int] by the key of Eq. 3
 * (omega = i_1 xor ... xor i_{n_int}, compared as unsigned 64-bit; ties broken
 * by the words from the last to the first, unsigned), computed with an LSD
 * radix sort. Host only.
 */
mdet_status mdet_omega_sort(int64_t n, int n_int, const uint64_t* dets, int64_t* order);

#ifdef __cplusplus
}
#endif

#endif /* MDET_H */

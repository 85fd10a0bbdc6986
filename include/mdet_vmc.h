/*
 * mdet_vmc.h -- variational Monte Carlo moves around mdet_evaluate, and a
 * small learned Metropolis proposal.
 *
 * One Monte Carlo step moves all electrons of every walker and needs Psi, the
 * drift vector and the local energy at the new positions (Sec. 4 of the paper:
 * the timings are for one walker making one all-electron step, including
 * Psi, the drift and E_L). The calls here supply the rest of the step on the
 * GPU: the proposal, its transition densities and the Metropolis-Hastings
 * acceptance, so that the chain samples |Psi|^2 exactly whichever proposal
 * is used.
 *
 * Proposals:
 *  - drift-diffusion: R' = R + tau F(R) + sqrt(tau) chi, F = grad Psi / Psi,
 *    density q(R'|R) ~ exp(-|R' - R - tau F(R)|^2 / (2 tau));
 *  - learned: a 3-layer perceptron (tanh hidden layers, BF16 weights, FP32
 *    accumulation) maps the 3N coordinates to 3N mean offsets and N per-electron
 *    log-scales, R'_i = R_i + mu_i(R) + k sigma_i^2 F_i(R) + sigma_i chi_i with
 *    sigma_i = exp(s_i(R)) (the offset mu_i is in units of sigma_i), with density
 *    q(R'|R) ~ prod_i exp(-|R'_i - R_i - mu_i - k sigma_i^2 F_i|^2 / (2 sigma_i^2) - 3 s_i).
 *    k = 1 (the Langevin form: a drift-diffusion move with a learned,
 *    per-electron and position-dependent time step sigma_i^2 plus a learned
 *    offset) when a drift array is passed, k = 0 (the network alone) when it is NULL.
 * chi are standard normal variates from the counter-based Philox4x32-10
 * generator (Salmon, Moraes, Dror, Shaw, SC'11) keyed by (seed, step) and
 * indexed by (walker, coordinate); the same stream drives the acceptance draws.
 *
 * All arrays are device pointers; calls are asynchronous on `stream`.
 * Positions and log-densities are FP64 ([n_walk][n_elec][3] and [n_walk]).
 */
#ifndef MDET_VMC_H
#define MDET_VMC_H

#include <stdint.h>

#include "mdet.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 block: out[0..3] for counter ctr[0..3] and key key[0..1] (host, for tests). */
void mdet_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/*
 * Drift-diffusion proposal: R_new = R + tau * grad + sqrt(tau) * chi and
 * log_q_fwd = -|R_new - R - tau grad|^2 / (2 tau) (constants that cancel in
 * the acceptance ratio are dropped).
 */
mdet_status mdet_vmc_propose_drift(int64_t n_walk, int n_elec, const double* R, const double* grad, double tau,
                                   uint64_t seed, uint64_t step, double* R_new, double* log_q_fwd, void* stream);

/* Reverse drift-diffusion density: log_q_rev = -|R - R_new - tau grad_new|^2 / (2 tau). */
mdet_status mdet_vmc_reverse_drift(int64_t n_walk, int n_elec, const double* R, const double* R_new,
                                   const double* grad_new, double tau, double* log_q_rev, void* stream);

/*
 * Metropolis-Hastings acceptance of an all-electron move per walker:
 * accept with probability min(1, |Psi'/Psi|^2 q(R|R') / q(R'|R)), where
 * log|Psi| and sign come from mdet_evaluate. A move onto a node (sign 0) or with
 * a non-finite ratio is rejected. Accepted walkers get R, log|Psi|, sign, grad,
 * lap and e_local copied from the proposed state. A current state with
 * |Psi| = 0 (log alpha = +inf) accepts any finite proposal; a proposal with a
 * non-finite log|Psi| or drift is rejected. accept[w] = 1 / 0;
 * n_accept (device, may be null) is incremented by the number accepted.
 */
mdet_status mdet_vmc_accept(int64_t n_walk, int n_elec, uint64_t seed, uint64_t step, const double* log_q_fwd,
                            const double* log_q_rev, double* R, double* log_abs_psi, int8_t* sign, double* grad,
                            double* lap, double* e_local, const double* R_new, const double* log_abs_psi_new,
                            const int8_t* sign_new, const double* grad_new, const double* lap_new,
                            const double* e_local_new, int32_t* accept, uint32_t* n_accept, void* stream);

/*
 * Drift limiting (Umrigar, Nightingale and Runge, J. Chem. Phys. 99, 2865
 * (1993)), per electron i: F_bar_i = F_i (-1 + sqrt(1 + 2 a tau |F_i|^2)) / (a tau |F_i|^2).
 * Near a node |F| grows as the inverse distance to it and tau F overshoots;
 * the limited drift keeps tau |F_bar| below sqrt(2 tau / a). a = 0 copies F.
 * F and F_bar: [n_walk][n_elec][3] (may alias). Pass F_bar as the drift of
 * both the forward move and the reverse density: any drift that is a
 * function of the position keeps the acceptance exact.
 */
mdet_status mdet_vmc_limit_drift(int64_t n_walk, int n_elec, const double* F, double tau, double a, double* F_bar,
                                 void* stream);

/*
 * dst[w][:] = src[w][:] for the walkers with take[w] != 0 (rows of `width`
 * floats): keeps per-walker data such as the network output at the current
 * position in step with mdet_vmc_accept's accept flags.
 */
mdet_status mdet_vmc_select_rows(int64_t n_walk, int width, const int32_t* take, const float* src, float* dst,
                                 void* stream);

/* Sum of squared electron distances to the origin per walker (an observable for autocorrelation). */
mdet_status mdet_vmc_r2(int64_t n_walk, int n_elec, const double* R, double* r2, void* stream);

/* ---- the learned proposal ---------------------------------------------- */

/*
 * The perceptron's matrix product, exposed for testing and reuse (no paper
 * counterpart): D[m][n] = sum_k bf16(A[m][k]) bf16(B[n][k]) for m < M, n < N,
 * k < K on the tcgen05 tensor cores (operands rounded to BF16, nearest even;
 * FP32 accumulation in tensor memory). A is M x K row-major with leading
 * dimension lda, B is N x K row-major with ldb, D is M x N with ldd; all FP32
 * and on the device. accumulate = 0: D is overwritten (k_split is ignored);
 * 1: the product is added to D with FP32 atomics, the K range split over CTAs
 * of k_split (rounded up to 64) each. Asynchronous on `stream`. MDET_E_ARG on a
 * negative size, a null pointer with a nonzero size or a leading dimension
 * below the row length; MDET_E_CUDA on a launch error.
 */
mdet_status mdet_gemm_bf16(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                           float* D, int64_t ldd, int accumulate, int64_t k_split, void* stream);

typedef struct mdet_mlp mdet_mlp;

/*
 * A 3-layer perceptron n_in -> hidden -> hidden -> n_out with tanh after the
 * two hidden layers, for n_in = 3 n_elec and n_out = 4 n_elec. Master weights
 * are FP32 (Adam state alongside). Every product of the forward and backward
 * passes runs on the tcgen05 tensor cores (mdet_gemm_bf16 below): BF16 copies of
 * the weights, the activations and back-propagated deltas rounded to BF16 as
 * they enter a product, FP32 accumulation; the tanh derivatives and the bias
 * gradients use the unrounded FP32 values. Weights are drawn from U(-a, a) with
 * a = sqrt(6 / (fan_in + fan_out)) (Glorot) by Philox with `seed`, biases 0.
 * Parameter order everywhere: W1 [n_in][hidden], b1 [hidden], W2 [hidden][hidden],
 * b2 [hidden], W3 [hidden][n_out], b3 [n_out] (W[k][j]: input k, output j).
 * Head, per electron e and coordinate c: s_e = s0 + s_span * tanh(out[3N + e]),
 * mu_c = exp(s_e) * mu_max * tanh(out[c]) (offsets in units of the electron's step).
 */
mdet_status mdet_mlp_create(mdet_mlp** out, int device, int n_elec, int hidden, uint64_t seed, double mu_max,
                            double s0, double s_span, double coord_scale);
void mdet_mlp_destroy(mdet_mlp* m);
int64_t mdet_mlp_n_params(const mdet_mlp* m);
/* Host copies of the FP32 master parameters / their accumulated gradients, and parameter upload. */
mdet_status mdet_mlp_get_params(const mdet_mlp* m, float* host);
mdet_status mdet_mlp_set_params(mdet_mlp* m, const float* host);
mdet_status mdet_mlp_get_grads(const mdet_mlp* m, float* host);

/*
 * Forward pass for n_walk walkers at positions R: features x = R / coord_scale
 * (FP32), then the network; out [n_walk][4 n_elec] raw outputs (FP32, device).
 * The activations are kept for mdet_mlp_backward (n_walk <= the largest batch
 * seen; scratch grows synchronously on first use at a new size).
 */
mdet_status mdet_mlp_forward(mdet_mlp* m, int64_t n_walk, const double* R, float* out, void* stream);

/*
 * Backward pass of the last forward: given dL/d(out) [n_walk][4 n_elec]
 * (FP32, device), accumulates dL/d(params) into the gradient buffer.
 */
mdet_status mdet_mlp_backward(mdet_mlp* m, int64_t n_walk, const float* dout, void* stream);
mdet_status mdet_mlp_zero_grad(mdet_mlp* m, void* stream);

/* One Adam step (Kingma and Ba) on the master weights from the accumulated gradients. */
mdet_status mdet_mlp_adam(mdet_mlp* m, double lr, double beta1, double beta2, double eps, int64_t t,
                          void* stream);

/*
 * Training loss: mean over walkers of the negative log-likelihood of the
 * observed move R0 -> R1 under the network's Gaussian at R0 (out from
 * mdet_mlp_forward at R0), and dL/d(out) for mdet_mlp_backward. loss: device
 * scalar (overwritten).
 */
mdet_status mdet_mlp_nll_grad(const mdet_mlp* m, int64_t n_walk, const double* R0, const double* R1,
                              const float* out, float* dout, double* loss, void* stream);

/*
 * Training objectives that target mixing, for the learned move drawn by
 * mdet_vmc_propose_mlp, with alpha = |Psi'/Psi|^2 q(R|R') / q(R'|R) and
 * A = min(1, alpha):
 *  - speed_beta <= 0: the expected squared jump distance weighted by the
 *    exact Metropolis-Hastings acceptance (Pasarica and Gelman, Stat. Sinica
 *    2010), J = E[ A |R' - R|^2 ];
 *  - speed_beta > 0: the generalised speed measure (Titsias and Dellaportas,
 *    NeurIPS 2019), J = E[ min(0, log alpha) ] + speed_beta * H(q(.|R)) with the
 *    proposal entropy H = 3 sum_e s_e + const; each rejected walker costs
 *    log alpha, so walkers that never move dominate it.
 * The reparametrisation gradient needs d log|Psi(R')| / dR',
 * which is grad_new (grad Psi / Psi from mdet_evaluate at R'). Inputs: R,
 * R_new (drawn by mdet_vmc_propose_mlp), out (network at R), out_new (network
 * at R_new), log|Psi| at both points, the sign at R_new, drift and drift_new
 * (the drift arrays the forward move and the reverse density used, e.g.
 * limited by mdet_vmc_limit_drift; read only when langevin != 0 and then not
 * NULL) and grad_new. langevin selects the form of the move (k above) and must
 * match the one that drew R_new.
 * Outputs: dout, dout_new = dL/d(out), dL/d(out_new) for the loss
 * L = -J (J averaged over walkers), and objective[0] = J, objective[1] = the
 * mean of A (two device doubles, overwritten). With
 * jump_len2 > 0 the squared jump of electron e is divided by |R_e|^2 + jump_len2
 * (its squared distance from the origin at R, for a one-centre system: a jump
 * relative to the local length scale); jump_len2 <= 0 gives the plain |R' - R|^2. The
 * network input at R_new and the drift at R_new are held fixed (their
 * derivatives with respect to R_new are not followed), which biases the
 * gradient but not the sampler: every move is still judged by the exact
 * acceptance.
 */
mdet_status mdet_mlp_esjd_grad(const mdet_mlp* m, int64_t n_walk, const double* R, const double* R_new,
                               const float* out, const float* out_new, const double* log_abs_psi,
                               const double* log_abs_psi_new, const int8_t* sign_new, const double* drift,
                               const double* drift_new, const double* grad_new, int langevin, double jump_len2,
                               double speed_beta, float* dout, float* dout_new, double* objective, void* stream);

/*
 * Learned proposal: R_new = R + mu(out) + k sigma^2 drift + sigma chi and
 * log_q_fwd; drift = grad Psi / Psi at R ([n_walk][n_elec][3]) or NULL (k = 0).
 */
mdet_status mdet_vmc_propose_mlp(const mdet_mlp* m, int64_t n_walk, const double* R, const float* out,
                                 const double* drift, uint64_t seed, uint64_t step, double* R_new, double* log_q_fwd,
                                 void* stream);

/*
 * Reverse learned density log q(R | R_new) from the network output and the
 * drift at R_new (NULL for k = 0; the same choice as for the forward move).
 */
mdet_status mdet_vmc_reverse_mlp(const mdet_mlp* m, int64_t n_walk, const double* R, const double* R_new,
                                 const float* out_new, const double* drift_new, double* log_q_rev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MDET_VMC_H */

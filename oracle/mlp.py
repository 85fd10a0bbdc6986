"""Plain numpy FP64 reference of the learned proposal's perceptron and losses.

TEST INFRASTRUCTURE ONLY (gradient checks of the CUDA forward/backward and
of the training objectives).
Network: x = R / coord_scale (3N) -> tanh(W1^T x + b1) -> tanh(W2^T h1 + b2)
-> W3^T h2 + b3 (4N); head per electron e: s_e = s0 + s_span tanh(out[3N + e]),
sigma_e = exp(s_e), mean offset mu_c = sigma_e mu_max tanh(out[c]).
NLL loss = mean over walkers of sum_e |R1_e - R0_e - mu_e|^2 / (2 sigma_e^2) + 3 s_e.
The move R' = R + mu + k sigma^2 F + sigma chi (k = 1 in the Langevin form, F
the drift grad Psi / Psi at R) has the Gaussian density written in log_q.
Parameter vector order: W1 [n_in][H], b1, W2 [H][H], b2, W3 [H][n_out], b3.

Readings (the move and its objective are not in the paper): the acceptance
follows Metropolis-Hastings with both proposal densities; the objective is the
expected squared jump distance weighted by the acceptance (Pasarica and
Gelman, Stat. Sinica 2010) or the generalised speed measure (Titsias and
Dellaportas, NeurIPS 2019), with the noise chi held fixed
(reparametrisation); log|Psi| near the proposed point is its first-order
expansion with the drift there, and the network input and the drift at the
proposed point are held fixed.
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, H, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + n_in * H].reshape(n_in, H); o += n_in * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H * n_out].reshape(H, n_out); o += H * n_out
    b3 = p[o:o + n_out]; o += n_out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, R, n_elec, H, coord_scale, weights_bf16=True, acts_bf16=False):
    """Network output [B][4N] and the intermediates (x, h1, h2, W1, W2, W3).

    weights_bf16: the weights enter the products rounded to BF16 (the stored copy).
    acts_bf16: every product's other operand is rounded to BF16 too (x, h1, h2 here),
    which is the arithmetic of a BF16 x BF16 tensor-core product with FP32 accumulation;
    the tanh derivatives use the unrounded activations.
    """
    n_in, n_out = 3 * n_elec, 4 * n_elec
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    if weights_bf16:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    rnd = bf16_round if acts_bf16 else (lambda a: a)
    x = np.asarray(R, dtype=np.float64).reshape(len(R), n_in) / coord_scale
    x = x.astype(np.float32).astype(np.float64)
    h1 = np.tanh(rnd(x) @ W1 + b1)
    h2 = np.tanh(rnd(h1) @ W2 + b2)
    out = rnd(h2) @ W3 + b3
    return out, (x, h1, h2, W1, W2, W3)


def head(out, n_elec, mu_max, s0, s_span):
    """Mean offsets mu [B][3N] and log-scales s [B][N] from the raw outputs."""
    out = np.asarray(out, dtype=np.float64)
    s = s0 + s_span * np.tanh(out[:, 3 * n_elec:])
    mu = np.repeat(np.exp(s), 3, axis=1) * mu_max * np.tanh(out[:, :3 * n_elec])
    return mu, s


def log_q(R_to, R_from, out_from, n_elec, mu_max, s0, s_span, F_from=None):
    """log q(R_to | R_from) per walker, up to the constant -3N/2 log(2 pi)."""
    B = len(R_from)
    mu, s = head(out_from, n_elec, mu_max, s0, s_span)
    sig = np.repeat(np.exp(s), 3, axis=1)
    mean = np.asarray(R_from, dtype=np.float64).reshape(B, -1) + mu
    if F_from is not None:
        mean = mean + sig ** 2 * np.asarray(F_from, dtype=np.float64).reshape(B, -1)
    d = (np.asarray(R_to, dtype=np.float64).reshape(B, -1) - mean) / sig
    return -0.5 * (d ** 2).sum(1) - 3.0 * s.sum(1)


def nll_and_grad(p, R0, R1, n_elec, H, coord_scale, mu_max, s0, s_span, weights_bf16=True, acts_bf16=False):
    """Loss and its gradient with respect to the parameter vector (backpropagation).
    acts_bf16: as in forward, and in the backward products both operands (activations,
    deltas) are rounded to BF16 as well; the bias gradients sum the unrounded deltas."""
    B = len(R0)
    rnd = bf16_round if acts_bf16 else (lambda a: a)
    out, (x, h1, h2, W1, W2, W3) = forward(p, R0, n_elec, H, coord_scale, weights_bf16, acts_bf16)
    tm = np.tanh(out[:, :3 * n_elec])
    ts = np.tanh(out[:, 3 * n_elec:])
    s = s0 + s_span * ts
    sig = np.exp(s)
    sig3 = np.repeat(sig, 3, axis=1)
    mu = sig3 * mu_max * tm
    d = (np.asarray(R1) - np.asarray(R0)).reshape(B, 3 * n_elec) - mu
    iv = np.exp(-2 * s)
    d2 = (d.reshape(B, n_elec, 3) ** 2).sum(-1)
    dmu_s = (d * mu).reshape(B, n_elec, 3).sum(-1)
    loss = float(np.mean(np.sum(0.5 * d2 * iv + 3 * s, axis=1)))
    # d mu_c / d out_c = sigma_e mu_max (1 - tanh^2); d mu_c / d s_e = mu_c
    dmu = -d * np.repeat(iv, 3, axis=1)
    ds = 3 - (d2 + dmu_s) * iv
    dout = np.concatenate([dmu * sig3 * mu_max * (1 - tm ** 2), ds * s_span * (1 - ts ** 2)], axis=1) / B
    gW3 = rnd(h2).T @ rnd(dout)
    gb3 = dout.sum(0)
    dh2 = (rnd(dout) @ W3.T) * (1 - h2 ** 2)
    gW2 = rnd(h1).T @ rnd(dh2)
    gb2 = dh2.sum(0)
    dh1 = (rnd(dh2) @ W2.T) * (1 - h1 ** 2)
    gW1 = rnd(x).T @ rnd(dh1)
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g, dout


def esjd_terms(out, out_new, R, R_new0, chi, lp, lp_new0, F, F_new, sign_new, n_elec, mu_max, s0, s_span,
               langevin=True, jump_len2=0.0, G_new=None, speed_beta=0.0):
    """Per-walker objective and log alpha, as a function of the raw outputs at
    R (out) and at the proposed point (out_new). The objective is the
    acceptance-weighted squared jump A * D2, or with speed_beta > 0 the
    generalised speed measure min(0, log alpha) + speed_beta * 3 sum_e s_e
    (Titsias and Dellaportas, NeurIPS 2019); 0 for a walker whose sign at
    R_new0 is 0.

    The proposed point follows the outputs with the noise chi fixed:
    R' = R + mu(out) + k sigma(out)^2 F + sigma(out) chi. log|Psi(R')| is
    lp_new0 + G_new . (R' - R_new0) (first order around the evaluated point
    R_new0; G_new = grad Psi / Psi there, F_new when not given), the reverse
    density uses out_new and the drift F_new as given, and
    log alpha = 2 (log|Psi(R')| - lp) + log q(R | R') - log q(R' | R);
    A = min(1, exp(log alpha)), 0 where the sign at R_new0 is 0.
    D2 = sum_e w_e |R'_e - R_e|^2 with w_e = 1 / (|R_e|^2 + jump_len2) when
    jump_len2 > 0, else 1.
    """
    B = len(R)
    k = 1.0 if langevin else 0.0
    Rf = np.asarray(R, dtype=np.float64).reshape(B, -1)
    mu, s = head(out, n_elec, mu_max, s0, s_span)
    sig = np.repeat(np.exp(s), 3, axis=1)
    Ff = np.asarray(F, dtype=np.float64).reshape(B, -1)
    Fn = np.asarray(F_new, dtype=np.float64).reshape(B, -1)
    Gn = Fn if G_new is None else np.asarray(G_new, dtype=np.float64).reshape(B, -1)
    Rn = Rf + mu + k * sig ** 2 * Ff + sig * chi
    lpn = np.asarray(lp_new0) + (Gn * (Rn - np.asarray(R_new0, dtype=np.float64).reshape(B, -1))).sum(1)
    lqf = -0.5 * (chi ** 2).sum(1) - 3.0 * s.sum(1)
    lqr = log_q(Rf, Rn, out_new, n_elec, mu_max, s0, s_span, Fn if langevin else None)
    la = 2.0 * (lpn - np.asarray(lp)) + lqr - lqf
    A = np.where(np.asarray(sign_new) != 0, np.exp(np.minimum(la, 0.0)), 0.0)
    if speed_beta > 0:
        J = np.where(np.asarray(sign_new) != 0, np.minimum(la, 0.0) + speed_beta * 3.0 * s.sum(1), 0.0)
        return J, la
    jump = ((Rn - Rf).reshape(B, n_elec, 3) ** 2).sum(-1)
    if jump_len2 > 0:
        jump = jump / ((Rf.reshape(B, n_elec, 3) ** 2).sum(-1) + jump_len2)
    return A * jump.sum(1), la


def esjd_and_dout(out, out_new, R, R_new, lp, lp_new, F, F_new, sign_new, n_elec, mu_max, s0, s_span,
                  langevin=True, jump_len2=0.0, G_new=None, speed_beta=0.0, h=1e-6):
    """Objective J = mean_w of esjd_terms at the drawn move R -> R_new, and dL/d(out),
    dL/d(out_new) for L = -J by central differences of esjd_terms (FP64).
    Also returns log alpha per walker (differences straddling log alpha = 0,
    where A has a kink, are not meaningful)."""
    out = np.asarray(out, dtype=np.float64)
    out_new = np.asarray(out_new, dtype=np.float64)
    B = len(R)
    k = 1.0 if langevin else 0.0
    mu, s = head(out, n_elec, mu_max, s0, s_span)
    sig = np.repeat(np.exp(s), 3, axis=1)
    Rf = np.asarray(R, dtype=np.float64).reshape(B, -1)
    chi = (np.asarray(R_new, dtype=np.float64).reshape(B, -1) - Rf - mu
           - k * sig ** 2 * np.asarray(F, dtype=np.float64).reshape(B, -1)) / sig
    args = (R, R_new, chi, lp, lp_new, F, F_new, sign_new, n_elec, mu_max, s0, s_span, langevin, jump_len2, G_new,
            speed_beta)
    J, la = esjd_terms(out, out_new, *args)
    dout = np.zeros_like(out)
    dout_new = np.zeros_like(out_new)
    for j in range(out.shape[1]):
        for arr, grad, first in ((out, dout, True), (out_new, dout_new, False)):
            e = np.zeros_like(arr)
            e[:, j] = h
            if first:
                jp, jm = esjd_terms(arr + e, out_new, *args)[0], esjd_terms(arr - e, out_new, *args)[0]
            else:
                jp, jm = esjd_terms(out, arr + e, *args)[0], esjd_terms(out, arr - e, *args)[0]
            grad[:, j] = -(jp - jm) / (2 * h) / B
    return float(J.mean()), dout, dout_new, la

"""Comparison of a GPU evaluation with the oracle, quantity by quantity.

Criteria (the reading of "Psi ratios" and of the derivative targets):
- log|Psi|: |d log|Psi|| <= tol_psi * max(1, kappa), kappa = sum_k |c_k D_up D_dn| / |Psi|.
  This is the error of Psi~ measured against sum_k |c_k r_up r_dn| (the magnitude of
  the terms of Eq. 1), the most a correctly rounded FP64 sum of those terms can
  promise; kappa enters here only.
- grad Psi / Psi and Lap_i Psi / Psi: |d x| <= tol_der * max(|x|, rms of that
  walker's values of the same quantity), with no conditioning factor.
- E_L = -1/2 sum_i Lap_i + V: |d E_L| <= tol_der * 1/2 sum_i max(|Lap_i|, rms), the
  bound the Laplacian criterion implies.
- sign: exact on every walker with kappa < sign_cap (1e12: below that an FP64
  sum keeps the sign by a margin of 1e4 roundings).
Walkers with kappa >= kappa_cap (next to a node of Psi) are left out of the value
checks, counted in n_ill, and the comparison fails when there are more than max_ill.
"""
from __future__ import annotations

import numpy as np


def _der_errors(g, ref):
    gs = np.sqrt(np.mean(ref["grad"] ** 2, axis=(1, 2)))[:, None, None]
    e_grad = np.abs(g["grad"] - ref["grad"]) / np.maximum(np.abs(ref["grad"]), gs)
    ls = np.sqrt(np.mean(ref["lap"] ** 2, axis=1))[:, None]
    lap_scale = np.maximum(np.abs(ref["lap"]), ls)
    e_lap = np.abs(g["lap"] - ref["lap"]) / lap_scale
    e_el = np.abs(g["e_local"] - ref["e_local"]) / (0.5 * lap_scale.sum(axis=1))
    return e_grad.max(axis=(1, 2)), e_lap.max(axis=1), e_el


def compare(gpu: dict, ref: dict, idx=None, tol_psi=1e-10, tol_der=1e-8, kappa_cap=1e8, sign_cap=1e12, max_ill=0):
    idx = np.arange(len(ref["log_abs_psi"])) if idx is None else np.asarray(idx)
    g = {k: np.asarray(v)[idx] for k, v in gpu.items()}
    kappa = np.asarray(ref["kappa"])
    well = kappa < kappa_cap
    signed = kappa < sign_cap
    sign_ok = bool(np.all(np.asarray(g["sign"]).astype(int)[signed] == np.asarray(ref["sign"])[signed]))
    e_log = np.abs(g["log_abs_psi"] - ref["log_abs_psi"]) / np.maximum(1.0, kappa)
    e_grad, e_lap, e_el = _der_errors(g, ref)

    def mx(e):
        return float(e[well].max(initial=0.0))

    def p99(e):
        return float(np.percentile(e[well], 99)) if well.any() else 0.0

    rep = dict(sign_ok=sign_ok, n_ill=int((~well).sum()), n_unsigned=int((~signed).sum()),
               log=mx(e_log), grad=mx(e_grad), lap=mx(e_lap), e_local=mx(e_el),
               p99_log=p99(e_log), p99_grad=p99(e_grad), p99_lap=p99(e_lap),
               kappa_max=float(kappa.max(initial=0.0)), kappa_p99=float(np.percentile(kappa, 99)) if kappa.size else 0.0)
    rep["ok"] = bool(sign_ok and rep["n_ill"] <= max_ill and rep["log"] <= tol_psi and rep["grad"] <= tol_der
                     and rep["lap"] <= tol_der and rep["e_local"] <= tol_der)
    return rep


def walker_quantiles(gpu: dict, ref: dict, idx=None):
    """Per-walker worst relative error of each quantity (no conditioning factor),
    for reporting max / p50 / p99."""
    idx = np.arange(len(ref["log_abs_psi"])) if idx is None else np.asarray(idx)
    g = {k: np.asarray(v)[idx] for k, v in gpu.items()}
    e_psi = np.abs(np.expm1(g["log_abs_psi"] - ref["log_abs_psi"]))
    e_grad, e_lap, _ = _der_errors(g, ref)
    out = {}
    for name, e in (("psi", e_psi), ("grad", e_grad), ("lap", e_lap)):
        out[name] = dict(max=float(e.max()), p50=float(np.percentile(e, 50)), p99=float(np.percentile(e, 99)))
    return out

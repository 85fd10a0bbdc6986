"""Comparison of a GPU evaluation with the oracle, quantity by quantity.

Tolerances (FP64 path): log|Psi| within tol_psi * max(1, kappa) where kappa =
sum_k |c_k D_up D_dn| / |Psi| is the conditioning of the sum (the relative
error of Psi a correctly rounded FP64 sum can reach); sign exact; grad and
Laplacian within tol_der * max(|x|, rms of that walker's electrons) * max(1, kappa).
"""
from __future__ import annotations

import numpy as np


def compare(gpu: dict, ref: dict, idx=None, tol_psi=1e-10, tol_der=1e-8, kappa_cap=1e8):
    idx = np.arange(len(ref["log_abs_psi"])) if idx is None else np.asarray(idx)
    g = {k: np.asarray(v)[idx] for k, v in gpu.items()}
    kappa = np.asarray(ref["kappa"])
    well = kappa < kappa_cap
    kfac = np.maximum(1.0, kappa)
    sign_ok = np.all(np.asarray(g["sign"]).astype(int)[well] == np.asarray(ref["sign"])[well])
    e_log = np.abs(g["log_abs_psi"] - ref["log_abs_psi"]) / kfac
    gs = np.sqrt(np.mean(ref["grad"] ** 2, axis=(1, 2)))[:, None, None]
    e_grad = np.abs(g["grad"] - ref["grad"]) / np.maximum(np.abs(ref["grad"]), gs) / kfac[:, None, None]
    ls = np.sqrt(np.mean(ref["lap"] ** 2, axis=1))[:, None]
    e_lap = np.abs(g["lap"] - ref["lap"]) / np.maximum(np.abs(ref["lap"]), ls) / kfac[:, None]
    el_s = np.maximum(np.abs(ref["e_local"]), 1.0)
    e_el = np.abs(g["e_local"] - ref["e_local"]) / el_s / kfac
    rep = dict(sign_ok=bool(sign_ok), n_ill=int((~well).sum()),
               log=float(e_log[well].max(initial=0)), grad=float(e_grad[well].max(initial=0)),
               lap=float(e_lap[well].max(initial=0)), e_local=float(e_el[well].max(initial=0)),
               p99_log=float(np.percentile(e_log[well], 99)) if well.any() else 0.0,
               p99_grad=float(np.percentile(e_grad[well].max(axis=(1, 2)), 99)) if well.any() else 0.0,
               p99_lap=float(np.percentile(e_lap[well].max(axis=1), 99)) if well.any() else 0.0)
    rep["ok"] = bool(sign_ok and rep["log"] <= tol_psi and rep["grad"] <= tol_der and rep["lap"] <= tol_der
                     and rep["e_local"] <= tol_der)
    return rep


def walker_quantiles(gpu: dict, ref: dict, idx=None):
    """Per-walker worst relative error of each quantity (no conditioning factor),
    for reporting max / p50 / p99."""
    idx = np.arange(len(ref["log_abs_psi"])) if idx is None else np.asarray(idx)
    g = {k: np.asarray(v)[idx] for k, v in gpu.items()}
    e_psi = np.abs(np.expm1(g["log_abs_psi"] - ref["log_abs_psi"]))
    gs = np.sqrt(np.mean(ref["grad"] ** 2, axis=(1, 2)))[:, None, None]
    e_grad = (np.abs(g["grad"] - ref["grad"]) / np.maximum(np.abs(ref["grad"]), gs)).max(axis=(1, 2))
    ls = np.sqrt(np.mean(ref["lap"] ** 2, axis=1))[:, None]
    e_lap = (np.abs(g["lap"] - ref["lap"]) / np.maximum(np.abs(ref["lap"]), ls)).max(axis=1)
    out = {}
    for name, e in (("psi", e_psi), ("grad", e_grad), ("lap", e_lap)):
        out[name] = dict(max=float(e.max()), p50=float(np.percentile(e, 50)), p99=float(np.percentile(e, 99)))
    return out

"""Plain-Python reference of the norm-based truncation (Sec. 3).

TEST INFRASTRUCTURE ONLY (parity of mdet_truncate_norm).
Definition: the squared norm sum_k c_k^2 of a CI expansion given as products
(D^up_k, D^dn_k, c_k) splits over the distinct spin determinants,
N_i^up = sum of c_k^2 over the products whose up determinant is D_i^up (likewise
down), and sum_i N_i^up = sum_j N_j^dn = sum_k c_k^2. Distinct determinants with
N_i^sigma <= eps_sigma are removed; every product that uses a removed determinant
is dropped. Reading: all removals use the norms of the untruncated expansion,
nothing is renormalised, and eps < 0 removes nothing of that spin.
Sums are exact-rounded (math.fsum).
"""
from __future__ import annotations

import math


def norms(dets, coef):
    """{determinant (tuple of words): N} over the distinct determinants of one spin."""
    parts = {}
    for d, c in zip(dets, coef):
        parts.setdefault(tuple(int(x) for x in d), []).append(float(c) * float(c))
    return {k: math.fsum(v) for k, v in parts.items()}


def truncate(det_up, det_dn, coef, eps_up, eps_dn):
    """keep[k] (list of bool), the per-product norms of both determinants and the counts
    (kept products, distinct up / down dets among kept products, distinct up / down dets)."""
    det_up = [tuple(int(x) for x in (d if hasattr(d, "__len__") else [d])) for d in det_up]
    det_dn = [tuple(int(x) for x in (d if hasattr(d, "__len__") else [d])) for d in det_dn]
    nu, nd = norms(det_up, coef), norms(det_dn, coef)
    gone_u = {d for d, n in nu.items() if eps_up >= 0 and n <= eps_up}
    gone_d = {d for d, n in nd.items() if eps_dn >= 0 and n <= eps_dn}
    keep = [u not in gone_u and d not in gone_d for u, d in zip(det_up, det_dn)]
    kept_u = {u for u, k in zip(det_up, keep) if k}
    kept_d = {d for d, k in zip(det_dn, keep) if k}
    counts = dict(products=sum(keep), up=len(kept_u), dn=len(kept_d), up_all=len(nu), dn_all=len(nd))
    return keep, [nu[u] for u in det_up], [nd[d] for d in det_dn], counts

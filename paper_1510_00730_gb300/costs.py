"""Operation-count model of the paper's Sherman-Morrison chain (Sec. 5).

It is used to report the sequential chain (`mdet_sm_chain`) against the full
inversions it replaces, as the paper does. Host arithmetic only.
"""
from __future__ import annotations

import numpy as np


def inversion_flops(n: int) -> int:
    """FP operations of a full n x n inversion (LU then inverse), about 2 n^3 (Sec. 5)."""
    return 2 * n ** 3


def substitution_flops(n: int) -> int:
    """FP operations of one Sherman-Morrison column substitution, 5 n^2 + 2 n + 3 (Sec. 5)."""
    return 5 * n * n + 2 * n + 3


def fixed_reference_substitutions(*degree_counts) -> float:
    """Average number of column substitutions per determinant if every determinant were
    reached from one fixed reference, one substitution per excited orbital: the mean
    excitation degree over the determinants of all the given histograms (count of
    determinants per degree, index = degree)."""
    num = den = 0.0
    for h in degree_counts:
        h = np.asarray(h, dtype=np.float64)
        num += float((np.arange(len(h)) * h).sum())
        den += float(h.sum())
    return num / den if den else 0.0

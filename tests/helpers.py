"""Independent checking tools used by the oracle pins (no oracle arithmetic here)."""
from __future__ import annotations

import itertools

import numpy as np


def perm_parity(p) -> int:
    """Sign of a permutation given as a sequence of distinct integers (by inversion count)."""
    p = list(p)
    inv = sum(1 for i in range(len(p)) for j in range(i + 1, len(p)) if p[i] > p[j])
    return -1 if inv % 2 else 1


def leibniz_det(a) -> float:
    """Determinant by the Leibniz permutation expansion (brute force, n <= 7)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    if n == 0:
        return 1.0
    tot = 0.0
    for p in itertools.permutations(range(n)):
        term = float(perm_parity(p))
        for i in range(n):
            term *= a[i, p[i]]
        tot += term
    return tot


def richardson_d1(f, x0: float, h: float) -> float:
    """First derivative by central differences with one Richardson step (error O(h^4))."""
    d = lambda hh: (f(x0 + hh) - f(x0 - hh)) / (2 * hh)
    return (4 * d(h / 2) - d(h)) / 3


def richardson_d2(f, x0: float, h: float) -> float:
    """Second derivative by central differences with one Richardson step (error O(h^4))."""
    f0 = f(x0)
    d = lambda hh: (f(x0 + hh) - 2 * f0 + f(x0 - hh)) / (hh * hh)
    return (4 * d(h / 2) - d(h)) / 3


def rel_err(a, b, floor=1e-300):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)

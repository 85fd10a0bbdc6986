"""Norm-based truncation (Sec. 3): the reference definition pinned by the
paper's norm identity and by hand-worked cases, and the library's host routine
(mdet_truncate_norm) against it, bit-exact on the keep decisions."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import truncation as otr
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth


def _hand_case():
    # up determinants a, b, c; down determinants x, y, z (one word each)
    a, b, c, x, y, z = 0b0011, 0b0101, 0b1001, 0b0011, 0b0110, 0b1100
    det_up = [[a], [a], [b], [c]]
    det_dn = [[x], [y], [x], [z]]
    coef = [0.9, 0.1, 0.05, 0.01]
    return det_up, det_dn, coef


def test_hand_worked_norms_and_removals():
    det_up, det_dn, coef = _hand_case()
    # N_a = 0.81 + 0.01, N_b = 0.0025, N_c = 1e-4; N_x = 0.81 + 0.0025, N_y = 0.01, N_z = 1e-4
    keep, nu, nd, cnt = otr.truncate(det_up, det_dn, coef, 1e-3, 5e-3)
    assert nu == pytest.approx([0.82, 0.82, 0.0025, 1e-4], rel=1e-15)
    assert nd == pytest.approx([0.8125, 0.01, 0.8125, 1e-4], rel=1e-15)
    assert keep == [True, True, True, False]
    assert cnt == dict(products=3, up=2, dn=2, up_all=3, dn_all=3)
    # a larger down threshold removes y as well, and with it the product (a, y)
    keep, _, _, cnt = otr.truncate(det_up, det_dn, coef, 1e-3, 2e-2)
    assert keep == [True, False, True, False]
    assert cnt == dict(products=2, up=2, dn=1, up_all=3, dn_all=3)
    # eps < 0 keeps everything; an infinite threshold removes everything
    assert otr.truncate(det_up, det_dn, coef, -1.0, -1.0)[0] == [True] * 4
    assert otr.truncate(det_up, det_dn, coef, math.inf, -1.0)[0] == [False] * 4


def test_norm_decomposition_identity():
    """Sec. 3: sum_i N_i^up = sum_j N_j^dn = sum_k c_k^2."""
    wl = synth.chlorine_like_100k(n_walk=1)
    nu = otr.norms(wl.det_up, wl.ci_coef)
    nd = otr.norms(wl.det_dn, wl.ci_coef)
    total = math.fsum(float(c) ** 2 for c in wl.ci_coef)
    assert math.fsum(nu.values()) == pytest.approx(total, rel=1e-14)
    assert math.fsum(nd.values()) == pytest.approx(total, rel=1e-14)
    assert len(nu) == len(np.unique(wl.det_up, axis=0)) and len(nd) == len(np.unique(wl.det_dn, axis=0))


def test_reference_is_order_independent():
    wl = synth.oxygen_like_1k(n_walk=1)
    perm = np.random.default_rng(0).permutation(len(wl.ci_coef))
    k1, _, _, c1 = otr.truncate(wl.det_up, wl.det_dn, wl.ci_coef, 1e-6, 1e-6)
    k2, _, _, c2 = otr.truncate(wl.det_up[perm], wl.det_dn[perm], wl.ci_coef[perm], 1e-6, 1e-6)
    assert c1 == c2
    assert [k1[i] for i in perm] == k2


def _midpoint_thresholds(values, n=5):
    """Thresholds between consecutive distinct norms (geometric midpoints), so no
    decision sits on a rounding boundary."""
    v = np.unique(np.asarray(values))
    v = v[v > 0]
    idx = np.linspace(1, len(v) - 1, n).astype(int)
    return [float(math.sqrt(v[i - 1] * v[i])) for i in idx]


@pytest.mark.parametrize("name", ["oxygen_like_1k", "chlorine_like_100k"])
def test_library_matches_reference(name):
    wl = synth.WORKLOADS[name]()
    _, nu_ref, nd_ref, _ = otr.truncate(wl.det_up, wl.det_dn, wl.ci_coef, -1.0, -1.0)
    keep, nu, nd, cnt = pkg.truncate_norm(wl.det_up, wl.det_dn, wl.ci_coef, -1.0, -1.0)
    assert keep.all() and cnt["products"] == len(wl.ci_coef)
    np.testing.assert_allclose(nu, nu_ref, rtol=1e-14)
    np.testing.assert_allclose(nd, nd_ref, rtol=1e-14)
    for eu, ed in zip(_midpoint_thresholds(nu_ref), _midpoint_thresholds(nd_ref)[::-1]):
        k_ref, _, _, c_ref = otr.truncate(wl.det_up, wl.det_dn, wl.ci_coef, eu, ed)
        k, _, _, c = pkg.truncate_norm(wl.det_up, wl.det_dn, wl.ci_coef, eu, ed)
        assert np.array_equal(k, np.asarray(k_ref)), (eu, ed)
        assert c == c_ref


def test_library_edge_cases():
    det_up, det_dn, coef = _hand_case()
    keep, nu, nd, cnt = pkg.truncate_norm(det_up, det_dn, coef, 1e-3, 5e-3)
    assert keep.tolist() == [True, True, True, False]
    assert cnt == dict(products=3, up=2, dn=2, up_all=3, dn_all=3)
    keep, _, _, cnt = pkg.truncate_norm(np.zeros((0, 1), np.uint64), np.zeros((0, 1), np.uint64),
                                        np.zeros(0), 1e-3, 1e-3)
    assert keep.size == 0 and cnt == dict(products=0, up=0, dn=0, up_all=0, dn_all=0)
    with pytest.raises(ValueError):
        pkg.truncate_norm(det_up, det_dn[:2], coef, 0.0, 0.0)

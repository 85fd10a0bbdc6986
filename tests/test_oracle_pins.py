"""Pins of the FP64 oracle against facts fixed outside it (no GPU needed).

Each test states which passage of the paper or which piece of mathematics it
checks. Together they are meant to catch a dropped term, a wrong sign, a wrong
index or a transposed operand anywhere in the oracle.
"""
from __future__ import annotations

import math
from itertools import combinations

import numpy as np
import pytest

import oracle
from paper_1510_00730_gb300 import synth
from tests.helpers import leibniz_det, perm_parity, richardson_d1, richardson_d2


def _one_shell_workload(l, alpha, coef=1.0):
    wl = synth.oxygen_like_1k(n_walk=1)
    wl.shell_l = np.array([l], np.int32)
    wl.shell_center = np.array([0], np.int32)
    wl.shell_nprim = np.array([1], np.int32)
    wl.alpha = np.array([alpha])
    wl.coef = np.array([coef])
    return wl


# --------------------------------------------------------------------------- AOs
@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_ao_values_norms_by_exact_quadrature(l):
    """Orbital values (Sec. 2): for one normalised primitive x^a y^b z^c e^{-alpha r^2}
    the squared norm is prod (2a-1)!! / (2l-1)!! (1 for the x^l component).
    Gauss-Hermite quadrature is exact for this integrand, so a wrong power,
    exponent or component order shows up."""
    alpha = 0.7
    norm = (2 * alpha / math.pi) ** 0.75 * (4 * alpha) ** (l / 2) / math.sqrt(synth._dfact(2 * l - 1))
    wl = _one_shell_workload(l, alpha, norm)
    t, w = np.polynomial.hermite.hermgauss(12)
    s = 1.0 / math.sqrt(2 * alpha)           # e^{-2 alpha x^2} = e^{-t^2} with x = s t
    X, Y, Zc = np.meshgrid(t * s, t * s, t * s, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]) * s ** 3
    pts = np.stack([X.ravel(), Y.ravel(), Zc.ravel()], axis=1)
    ao = oracle.ao_eval(wl, pts)[:, 0, :]   # [pts][n_ao]
    # the quadrature weight already contains e^{-2 alpha r^2}; divide it out of chi^2
    g = np.exp(-2 * alpha * (pts ** 2).sum(1))
    comps = [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]
    for mu, (a, b, c) in enumerate(comps):
        integral = float(np.sum(W.ravel() * ao[:, mu] ** 2 / g))
        expect = synth._dfact(2 * a - 1) * synth._dfact(2 * b - 1) * synth._dfact(2 * c - 1) / synth._dfact(2 * l - 1)
        assert abs(integral - expect) < 1e-12 * max(1.0, expect), (l, (a, b, c), integral, expect)


def test_ao_component_order_and_center():
    """Component order xx, xy, xz, yy, yz, zz (Sec. 8(b) boundary convention) and
    the value of an s function at its centre (= sum of contraction weights)."""
    wl = _one_shell_workload(2, 0.5, 1.0)
    p = np.array([[0.3, -0.7, 1.1]])
    v = oracle.ao_eval(wl, p)[0, 0]
    e = math.exp(-0.5 * (0.09 + 0.49 + 1.21))
    x, y, z = p[0]
    np.testing.assert_allclose(v, [x * x * e, x * y * e, x * z * e, y * y * e, y * z * e, z * z * e], rtol=1e-15)
    wl0 = _one_shell_workload(0, 3.0, 0.25)
    assert oracle.ao_eval(wl0, np.zeros((1, 3)))[0, 0, 0] == 0.25


def test_ao_derivatives_vs_finite_differences():
    """Gradient and Laplacian of every AO (Sec. 2) against Richardson central
    differences; two shells of each l = 0..3 with exponents in [0.1, 10] so the
    difference steps resolve every function."""
    wl = synth.oxygen_like_1k(n_walk=1)
    rng = np.random.default_rng(3)
    (wl.shell_l, wl.shell_center, wl.shell_nprim, wl.alpha, wl.coef) = synth.make_basis(rng, (2, 2, 2, 2), 0.1, 10.0)
    worst_g = worst_l = 0.0
    for _ in range(6):
        p0 = rng.normal(size=3) * 0.8
        ao0 = oracle.ao_eval(wl, p0[None])[0]
        scale = np.abs(ao0[0]) + 1e-12
        for d in range(3):
            def f(t, d=d):
                q = p0.copy(); q[d] = t
                return oracle.ao_eval(wl, q[None])[0, 0]
            fd = richardson_d1(f, p0[d], 2e-3)
            worst_g = max(worst_g, float(np.max(np.abs(fd - ao0[1 + d]) / (np.abs(ao0[1 + d]) + scale))))
        lap = np.zeros(wl.n_ao)
        for d in range(3):
            def f(t, d=d):
                q = p0.copy(); q[d] = t
                return oracle.ao_eval(wl, q[None])[0, 0]
            lap += richardson_d2(f, p0[d], 4e-3)
        worst_l = max(worst_l, float(np.max(np.abs(lap - ao0[4]) / (np.abs(ao0[4]) + scale))))
    assert worst_g < 1e-7, worst_g
    assert worst_l < 1e-5, worst_l


def test_mo_is_linear_combination_of_aos():
    """phi_m = sum_mu B[mu, m] chi_mu for value and derivatives (Sec. 2)."""
    wl = synth.oxygen_like_1k(n_walk=3)
    pts = wl.R.reshape(-1, 3)
    ao = oracle.ao_eval(wl, pts)
    mo = oracle.mo_eval(wl, pts)
    np.testing.assert_allclose(mo, ao @ wl.mo_coef, rtol=1e-12, atol=1e-12 * np.abs(ao).max())


# ------------------------------------------------------------------ determinants
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_det_matches_leibniz(n):
    """LU with partial pivoting (Sec. 2.2, dgetrf route) equals the Leibniz
    expansion the paper hard-codes for n <= 5."""
    rng = np.random.default_rng(n)
    for _ in range(5):
        a = rng.normal(size=(n, n))
        la, sg = oracle.det(a)
        ref = leibniz_det(a)
        assert sg == (1 if ref > 0 else -1)
        assert abs(sg * math.exp(la) - ref) <= 1e-13 * max(1.0, abs(ref))


def test_det_vandermonde_closed_form():
    """det V(x) = prod_{i<j} (x_j - x_i) for a 9 x 9 Vandermonde matrix."""
    x = np.array([0.3, -1.2, 0.7, 2.1, -0.4, 1.5, -2.2, 0.05, 1.1])
    V = np.vander(x, increasing=True)
    ref_sign, ref_log = 1, 0.0
    for i in range(9):
        for j in range(i + 1, 9):
            d = x[j] - x[i]
            ref_sign *= 1 if d > 0 else -1
            ref_log += math.log(abs(d))
    la, sg = oracle.det(V)
    assert sg == ref_sign
    assert abs(la - ref_log) < 1e-12


def test_det_permutation_and_singular():
    p = [3, 0, 4, 1, 2]
    P = np.eye(5)[p]
    la, sg = oracle.det(P)
    assert sg == perm_parity(p) and abs(la) < 1e-15
    a = np.random.default_rng(0).normal(size=(4, 4))
    a[2] = a[0]
    la, sg = oracle.det(a)
    assert sg == 0 or la < -30


def test_inverse_property():
    a = np.random.default_rng(1).normal(size=(9, 9))
    np.testing.assert_allclose(oracle.inverse(a) @ a, np.eye(9), atol=1e-12)


def test_sherman_morrison_ratio_identity():
    """Eq. 4: replacing column k of S by S[:,k] + u changes the determinant by
    the factor 1 + (S^-1 u)_k (the ratio the paper's threshold tests)."""
    rng = np.random.default_rng(5)
    for k in range(9):
        S = rng.normal(size=(9, 9))
        u = rng.normal(size=9)
        S2 = S.copy(); S2[:, k] += u
        l1, s1 = oracle.det(S)
        l2, s2 = oracle.det(S2)
        ratio = s1 * s2 * math.exp(l2 - l1)
        assert abs(ratio - (1 + (oracle.inverse(S) @ u)[k])) < 1e-12 * max(1, abs(ratio))


# ------------------------------------------------------------- wavefunction level
def _slater(mo_vals, occ, rows):
    return mo_vals[np.ix_(rows, occ)]


def _occ(bits_row):
    occ = []
    for q, w in enumerate(bits_row):
        for b in range(64):
            if (int(w) >> b) & 1:
                occ.append(64 * q + b)
    return occ


def test_single_determinant_is_plain_determinant():
    """N_det = 1 (Table 2, first row): Psi = c D_up D_dn, checked with Leibniz
    determinants of the 4 x 4 Slater matrices."""
    wl = synth.oxygen_like_1k(n_walk=5)
    k = 17
    du, dd, c = wl.det_up[k:k + 1], wl.det_dn[k:k + 1], np.array([-0.37])
    o = oracle.evaluate(wl, det_up=du, det_dn=dd, ci=c)
    for w in range(wl.n_walk):
        phi = oracle.mo_eval(wl, wl.R[w])[:, 0, :]
        up = leibniz_det(_slater(phi, _occ(du[0]), list(range(4))))
        dn = leibniz_det(_slater(phi, _occ(dd[0]), list(range(4, 8))))
        psi = -0.37 * up * dn
        assert o["sign"][w] == np.sign(psi)
        assert abs(o["log_abs_psi"][w] - math.log(abs(psi))) < 1e-12


def test_exchange_antisymmetry():
    """Psi changes sign when two same-spin electrons are exchanged (each Slater
    determinant is antisymmetric), but not in general for an up/down swap."""
    wl = synth.oxygen_like_1k(n_walk=6)
    o = oracle.evaluate(wl)
    R2 = wl.R.copy(); R2[:, [0, 2]] = R2[:, [2, 0]]
    o2 = oracle.evaluate(wl, R=R2)
    assert np.all(o2["sign"] == -o["sign"])
    np.testing.assert_allclose(o2["log_abs_psi"], o["log_abs_psi"], atol=1e-12)
    np.testing.assert_allclose(o2["grad"][:, [2, 0]], o["grad"][:, [0, 2]], rtol=1e-10, atol=1e-12)
    R3 = wl.R.copy(); R3[:, [5, 7]] = R3[:, [7, 5]]
    o3 = oracle.evaluate(wl, R=R3)
    assert np.all(o3["sign"] == -o["sign"])
    R4 = wl.R.copy(); R4[:, [0, 4]] = R4[:, [4, 0]]
    o4 = oracle.evaluate(wl, R=R4)
    assert np.max(np.abs(o4["log_abs_psi"] - o["log_abs_psi"])) > 1e-3


def test_gradient_and_laplacian_vs_finite_differences():
    """grad Psi / Psi and Lap_i Psi / Psi (Eqs. 5-7) against Richardson central
    differences of Psi itself."""
    wl = synth.oxygen_like_1k(n_walk=3)
    o = oracle.evaluate(wl)
    for w in range(wl.n_walk):
        base = wl.R[w]
        l0 = o["log_abs_psi"][w]
        s0 = o["sign"][w]

        def psi_rel(i, d, t):
            R = base.copy(); R[i, d] = t
            q = oracle.evaluate(wl, R=R[None], n_threads=1)
            return q["sign"][0] * s0 * math.exp(q["log_abs_psi"][0] - l0)

        g = o["grad"][w]
        lap = o["lap"][w]
        gscale = np.sqrt(np.mean(g ** 2))
        lscale = np.sqrt(np.mean(lap ** 2))
        for i in (0, 3, 4, 7):
            lap_fd = 0.0
            for d in range(3):
                f = lambda t: psi_rel(i, d, t)
                gfd = richardson_d1(f, base[i, d], 1e-3)
                assert abs(gfd - g[i, d]) <= 1e-6 * max(abs(g[i, d]), gscale), (w, i, d, gfd, g[i, d])
                lap_fd += richardson_d2(f, base[i, d], 2e-3)
            assert abs(lap_fd - lap[i]) <= 1e-4 * max(abs(lap[i]), lscale), (w, i, lap_fd, lap[i])


def test_fci_cauchy_binet_closed_form():
    """Full CI (Sec. 1: N_det = N_det^up * N_det^dn = C(M, N)^2): with
    C_IJ = det U[I, :N_up] det U[J, :N_dn] for an orthogonal U, Cauchy-Binet
    gives Psi = det(Phi_up U_up) det(Phi_dn U_dn), i.e. one determinant of the
    rotated orbitals phi' = phi U. Pins the ascending-column convention, every
    sign and index of the product sum, and the derivatives."""
    M, N = 10, 4
    wl = synth.oxygen_like_1k(n_walk=4)
    wl.mo_coef = wl.mo_coef[:, :M].copy()
    rng = np.random.default_rng(11)
    U, _ = np.linalg.qr(rng.normal(size=(M, M)))
    subsets = list(combinations(range(M), N))
    assert len(subsets) == math.comb(M, N) == 210
    bits = np.array([[sum(1 << m for m in s)] for s in subsets], dtype=np.uint64)
    minors = np.array([np.linalg.det(U[list(s), :N]) for s in subsets])
    I, J = np.meshgrid(np.arange(len(subsets)), np.arange(len(subsets)), indexing="ij")
    det_up = bits[I.ravel()]
    det_dn = bits[J.ravel()]
    ci = minors[I.ravel()] * minors[J.ravel()]
    assert ci.shape[0] == 44100
    o = oracle.evaluate(wl, det_up=det_up, det_dn=det_dn, ci=ci)
    aufbau = np.array([[0b1111]], dtype=np.uint64)
    o1 = oracle.evaluate(wl, det_up=aufbau, det_dn=aufbau, ci=np.array([1.0]), mo_coef=wl.mo_coef @ U)
    assert np.all(o["sign"] == o1["sign"])
    np.testing.assert_allclose(o["log_abs_psi"], o1["log_abs_psi"], atol=1e-10)
    np.testing.assert_allclose(o["grad"], o1["grad"], rtol=1e-8, atol=1e-9 * np.abs(o1["grad"]).max())
    np.testing.assert_allclose(o["lap"], o1["lap"], rtol=1e-8, atol=1e-9 * np.abs(o1["lap"]).max())


def test_brute_force_tiny_expansion():
    """Eq. 1 by brute force on every product of a 2 up / 2 down system in 5 MOs
    (100 products): Leibniz determinants for values and, for derivatives,
    Leibniz determinants of the Slater matrices with row i replaced by the
    derivative row (each row depends on one electron only)."""
    wl = synth.tiny()
    assert wl.n_det == 100
    o = oracle.evaluate(wl)
    ne = 4
    for w in range(wl.n_walk):
        phi = oracle.mo_eval(wl, wl.R[w])   # [e][5][m]
        psi = 0.0
        G = np.zeros((ne, 4))
        for k in range(wl.n_det):
            ou, od = _occ(wl.det_up[k]), _occ(wl.det_dn[k])
            Su = phi[np.ix_([0, 1], [0], ou)][:, 0, :]
            Sd = phi[np.ix_([2, 3], [0], od)][:, 0, :]
            Du, Dd = leibniz_det(Su), leibniz_det(Sd)
            c = wl.ci_coef[k]
            psi += c * Du * Dd
            for i in range(ne):
                for mu in range(4):
                    if i < 2:
                        S = Su.copy(); S[i] = phi[i, 1 + mu, ou]
                        G[i, mu] += c * leibniz_det(S) * Dd
                    else:
                        S = Sd.copy(); S[i - 2] = phi[i, 1 + mu, od]
                        G[i, mu] += c * Du * leibniz_det(S)
        assert o["sign"][w] == np.sign(psi)
        assert abs(o["log_abs_psi"][w] - math.log(abs(psi))) < 1e-11
        np.testing.assert_allclose(o["grad"][w], G[:, :3] / psi, rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(o["lap"][w], G[:, 3] / psi, rtol=1e-9, atol=1e-11)


def test_product_sum_equals_bilinear_form():
    """Eq. 1 (sum over products) equals Eq. 2 (D_up^T C D_dn over distinct spin
    determinants with a dense C built from the product list)."""
    wl = synth.oxygen_like_1k(n_walk=4)
    o = oracle.evaluate(wl)
    ku = {tuple(r): i for i, r in enumerate(np.unique(wl.det_up, axis=0).tolist())}
    kd = {tuple(r): i for i, r in enumerate(np.unique(wl.det_dn, axis=0).tolist())}
    ups = np.array(list(ku.keys()), dtype=np.uint64)
    dns = np.array(list(kd.keys()), dtype=np.uint64)
    Cm = np.zeros((len(ku), len(kd)))
    for k in range(wl.n_det):
        Cm[ku[tuple(wl.det_up[k].tolist())], kd[tuple(wl.det_dn[k].tolist())]] += wl.ci_coef[k]
    lu, su, _ = oracle.spin_dets(wl, 0, ups)
    ld, sd, _ = oracle.spin_dets(wl, 1, dns)
    for w in range(wl.n_walk):
        mu, md = lu[w].max(), ld[w].max()
        Du = su[w] * np.exp(lu[w] - mu)
        Dd = sd[w] * np.exp(ld[w] - md)
        psi = Du @ Cm @ Dd
        assert np.sign(psi) == o["sign"][w]
        assert abs(math.log(abs(psi)) + mu + md - o["log_abs_psi"][w]) < 1e-11 * o["kappa"][w]


def test_local_energy_hydrogenic_closed_form():
    """E_L = -1/2 Lap Psi / Psi + V: for one electron in the 1s orbital
    e^{-alpha r^2} of a nucleus of charge Z, E_L = 3 alpha - 2 alpha^2 r^2 - Z/r."""
    alpha, Z = 0.6, 2.0
    wl = _one_shell_workload(0, alpha)
    wl.n_up, wl.n_dn = 1, 0
    wl.Z = np.array([Z])
    wl.mo_coef = np.ones((1, 1))
    R = np.array([[[0.3, -0.4, 0.5]], [[1.1, 0.2, -0.3]]])
    o = oracle.evaluate(wl, R=R, det_up=np.array([[1]], np.uint64), det_dn=np.zeros((1, 1), np.uint64),
                        ci=np.array([1.0]))
    r2 = (R ** 2).sum(-1)[:, 0]
    np.testing.assert_allclose(o["e_local"], 3 * alpha - 2 * alpha ** 2 * r2 - Z / np.sqrt(r2), rtol=1e-13)
    np.testing.assert_allclose(o["grad"][:, 0], -2 * alpha * R[:, 0], rtol=1e-13)


# ------------------------------------------------------- conditioning of the CI sum
# kappa = sum_k |c_k D_up D_dn| / |Psi| (the factor by which a relative rounding
# of each product of Eq. 1 can grow in the sum); the parity tests scale the
# log|Psi| tolerance by it, so it gets pins of its own.
def test_kappa_single_determinant_is_one():
    """N_det = 1: the sum has one term, so sum |c D D| = |Psi| and kappa = 1 exactly."""
    wl = synth.oxygen_like_1k(n_walk=7)
    o = oracle.evaluate(wl, det_up=wl.det_up[5:6], det_dn=wl.det_dn[5:6], ci=np.array([-2.5]))
    assert np.all(o["kappa"] == 1.0), o["kappa"]


def _two_product_case():
    """Two products with distinct up and down determinants and coefficients of
    opposite sign, at walkers where the two terms partly cancel."""
    wl = synth.oxygen_like_1k(n_walk=40, seed=77)
    ks = [0, 9]
    du, dd, c = wl.det_up[ks], wl.det_dn[ks], np.array([0.8, -0.55])
    assert not np.array_equal(du[0], du[1]) and not np.array_equal(dd[0], dd[1])
    terms = np.empty((wl.n_walk, 2))
    for w in range(wl.n_walk):
        phi = oracle.mo_eval(wl, wl.R[w])[:, 0, :]
        for q in range(2):
            up = leibniz_det(_slater(phi, _occ(du[q]), list(range(4))))
            dn = leibniz_det(_slater(phi, _occ(dd[q]), list(range(4, 8))))
            terms[w, q] = c[q] * up * dn
    return wl, du, dd, c, terms


def test_kappa_two_products_closed_form():
    """kappa = (|t1| + |t2|) / |t1 + t2| with t_q = c_q D_up,q D_dn,q from Leibniz
    determinants of the (pinned) orbital values; at least some walkers have
    terms of opposite sign, so a numerator without |.|, or the reciprocal, fails."""
    wl, du, dd, c, t = _two_product_case()
    want = np.abs(t).sum(1) / np.abs(t.sum(1))
    assert (want > 1.5).sum() >= 5, want
    o = oracle.evaluate(wl, det_up=du, det_dn=dd, ci=c)
    np.testing.assert_allclose(o["kappa"], want, rtol=1e-9)
    np.testing.assert_array_equal(o["sign"], np.sign(t.sum(1)))


def test_kappa_fci_cauchy_binet():
    """Full CI with C_IJ = m_I m_J (m the N x N minors of an orthogonal U, as in the
    Cauchy-Binet pin above): sum_IJ |C_IJ D_I D_J| factorises into
    (sum_I |m_I D_up,I|) (sum_J |m_J D_dn,J|), and Psi = det(Phi_up U_:N) det(Phi_dn U_:N).
    The determinants here are numpy's LU (an independent library routine)."""
    M, N = 10, 4
    wl = synth.oxygen_like_1k(n_walk=5)
    wl.mo_coef = wl.mo_coef[:, :M].copy()
    U, _ = np.linalg.qr(np.random.default_rng(11).normal(size=(M, M)))
    subsets = list(combinations(range(M), N))
    bits = np.array([[sum(1 << m for m in s)] for s in subsets], dtype=np.uint64)
    minors = np.array([np.linalg.det(U[list(s), :N]) for s in subsets])
    I, J = np.meshgrid(np.arange(len(subsets)), np.arange(len(subsets)), indexing="ij")
    o = oracle.evaluate(wl, det_up=bits[I.ravel()], det_dn=bits[J.ravel()], ci=minors[I.ravel()] * minors[J.ravel()])
    for w in range(wl.n_walk):
        phi = oracle.mo_eval(wl, wl.R[w])[:, 0, :]
        su = sum(abs(m * np.linalg.det(phi[:4][:, list(s)])) for m, s in zip(minors, subsets))
        sd = sum(abs(m * np.linalg.det(phi[4:][:, list(s)])) for m, s in zip(minors, subsets))
        psi = np.linalg.det(phi[:4] @ U[:, :N]) * np.linalg.det(phi[4:] @ U[:, :N])
        assert abs(o["kappa"][w] - su * sd / abs(psi)) <= 1e-9 * su * sd / abs(psi), (w, o["kappa"][w])


# ------------------------------------------------------------ potential energy
# V of E_L (Sec. 4): electron-nucleus attraction, electron-electron and
# nucleus-nucleus repulsion. Each pin below is a hand-evaluated configuration.
def test_potential_two_electrons_one_nucleus():
    """r1 = (0, 0, 1), r2 = (0, 3, 1), Z = 2 at the origin:
    V = -2/1 - 2/sqrt(10) + 1/3 (the electron pair enters once, with a + sign)."""
    v = oracle.potential([[0, 0, 1.0], [0, 3.0, 1.0]], [2.0], [[0, 0, 0]])
    assert abs(v - (-2.0 - 2.0 / math.sqrt(10.0) + 1.0 / 3.0)) < 1e-15


def test_potential_nucleus_pair():
    """No electron: V = Z_A Z_B / R_AB = 3 * 5 / 2.5; one electron midway between
    them adds -3/1.25 - 5/1.25."""
    X = [[0, 0, 0], [1.5, 2.0, 0]]
    assert abs(oracle.potential(np.zeros((0, 3)), [3.0, 5.0], X) - 6.0) < 1e-15
    v = oracle.potential([[0.75, 1.0, 0]], [3.0, 5.0], X)
    assert abs(v - (6.0 - 3.0 / 1.25 - 5.0 / 1.25)) < 1e-14


def test_potential_three_electrons_count_pairs():
    """Three electrons on a 3-4-5 right triangle, no nuclei: 1/3 + 1/4 + 1/5
    (three pairs, each once); four electrons on a unit square: 4 + 2/sqrt(2)."""
    v = oracle.potential([[0, 0, 0], [3.0, 0, 0], [0, 4.0, 0]])
    assert abs(v - (1 / 3 + 1 / 4 + 1 / 5)) < 1e-15
    v4 = oracle.potential([[0, 0, 0], [1.0, 0, 0], [1.0, 1.0, 0], [0, 1.0, 0]])
    assert abs(v4 - (4.0 + 2.0 / math.sqrt(2.0))) < 1e-14


def test_local_energy_two_electrons_two_nuclei_closed_form():
    """E_L of Psi = e^{-alpha r1^2} e^{-alpha r2^2} (one up and one down electron in
    the same 1s Gaussian on nucleus A) next to a second nucleus B:
    E_L = sum_i (3 alpha - 2 alpha^2 r_i^2) - sum_iA Z_A / |r_i - X_A| + 1 / r12 + Z_A Z_B / R_AB,
    which pins the kinetic term, all three potential sums and their signs in
    evaluate itself."""
    alpha, ZA, ZB = 0.45, 2.0, 1.0
    wl = _one_shell_workload(0, alpha)
    wl.n_up, wl.n_dn = 1, 1
    wl.Z = np.array([ZA, ZB])
    XB = np.array([0.3, -0.2, 1.4])
    wl.nuc_xyz = np.array([[0.0, 0.0, 0.0], XB])
    wl.mo_coef = np.ones((1, 1))
    R = np.array([[[0.3, -0.4, 0.5], [-0.6, 0.1, 0.9]], [[1.1, 0.2, -0.3], [0.2, 0.2, 0.2]]])
    one = np.array([[1]], np.uint64)
    o = oracle.evaluate(wl, R=R, det_up=one, det_dn=one, ci=np.array([1.0]))
    for w in range(R.shape[0]):
        r1, r2 = R[w]
        kin = sum(3 * alpha - 2 * alpha ** 2 * (r @ r) for r in (r1, r2))
        ven = -sum(ZA / np.linalg.norm(r) + ZB / np.linalg.norm(r - XB) for r in (r1, r2))
        want = kin + ven + 1.0 / np.linalg.norm(r1 - r2) + ZA * ZB / np.linalg.norm(XB)
        assert abs(o["e_local"][w] - want) < 1e-13 * max(1.0, abs(want)), (w, o["e_local"][w], want)


def test_local_energy_is_kinetic_plus_potential_many_electrons():
    """For the 8-electron expansion, E_L + 1/2 sum_i Lap_i Psi / Psi (the kinetic
    part, pinned by finite differences above) equals V by brute force over every
    electron, pair and nucleus: 28 electron pairs."""
    wl = synth.oxygen_like_1k(n_walk=3)
    o = oracle.evaluate(wl)
    for w in range(wl.n_walk):
        r = wl.R[w]
        v = -sum(wl.Z[A] / np.linalg.norm(r[i] - wl.nuc_xyz[A]) for i in range(8) for A in range(len(wl.Z)))
        v += sum(1.0 / np.linalg.norm(r[i] - r[j]) for i, j in combinations(range(8), 2))
        assert abs(o["e_local"][w] + 0.5 * o["lap"][w].sum() - v) < 1e-12 * max(1.0, abs(v))


# ------------------------------------------------ row-replaced cross-check mode
@pytest.mark.parametrize("name,n_walk", [("tiny", 6), ("oxygen_like_1k", 16)])
def test_row_replaced_mode_matches_cofactor_mode(name, n_walk):
    """The two derivative routes of the oracle: cofactors from the inverse (mode 0,
    Eq. 8 read with (S^-1)_{a i}) and determinants of the Slater matrix with row i
    replaced by d_mu phi(r_i) (mode 1, the definition of a derivative of a
    determinant that is linear in row i) agree to rounding."""
    wl = getattr(synth, name)(n_walk=n_walk)
    o0 = oracle.evaluate(wl, mode=0)
    o1 = oracle.evaluate(wl, mode=1)
    np.testing.assert_array_equal(o0["sign"], o1["sign"])
    np.testing.assert_allclose(o1["log_abs_psi"], o0["log_abs_psi"], rtol=0, atol=1e-13)
    for k in ("grad", "lap"):
        a, b = o0[k], o1[k]
        scale = np.sqrt(np.mean(a.reshape(n_walk, -1) ** 2, axis=1)).reshape((-1,) + (1,) * (a.ndim - 1))
        err = np.abs(a - b) / np.maximum(np.abs(a), scale)
        assert err.max() < 1e-10, (k, err.max())

"""Host-side logic of the library (no GPU): the C ABI surface, the encoding and
ordering of Sec. 2.1, the sparse C matrix, excitation records and phases, and
input validation. Contexts here are created with device = -1 (no device)."""
from __future__ import annotations

import math
import os
import re
from itertools import combinations

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import binding, synth
from tests.helpers import perm_parity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _host_ctx(wl):
    return pkg.Context.from_workload(wl, device=binding.NO_DEVICE)


def test_library_exports_every_declared_symbol():
    """Every function declared in include/*.h is exported by libmdet.so."""
    L = pkg.load_library()
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(mdet_\w+)\s*\(", txt, flags=re.M))
    assert len(names) >= 14, names
    for n in sorted(names):
        assert hasattr(L, n), n


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    """Rows of a fixture under tests/golden (the paper's printed values), comments skipped."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_paper_encoding_examples():
    """Sec. 2.1: the Hartree-Fock determinant of Cl is (511, 255), and the
    up+down excitation 7 -> 12 is (2495, 2239) (tests/golden/encoding_sec2_1.txt)."""
    rows = {r[0]: r[1:] for r in _golden("encoding_sec2_1.txt")}
    hf_up = synth.occ_to_bits(range(9), 1)[0]
    hf_dn = synth.occ_to_bits(range(8), 1)[0]
    assert [hf_up, hf_dn] == [int(x) for x in rows["hf"][:2]]
    assert [format(hf_up, "b"), format(hf_dn, "b")] == rows["hf"][2:]
    ex_up = synth.occ_to_bits([0, 1, 2, 3, 4, 5, 7, 8, 11], 1)[0]
    ex_dn = synth.occ_to_bits([0, 1, 2, 3, 4, 5, 7, 11], 1)[0]
    assert [ex_up, ex_dn] == [int(x) for x in rows["ex_7_to_12"][:2]]
    assert [format(ex_up, "b"), format(ex_dn, "b")] == rows["ex_7_to_12"][2:]
    # the library reads the same strings as a degree-1 excitation of the reference
    wl = synth.chlorine_like_100k(n_walk=1)
    wl.mo_coef = wl.mo_coef[:, :19].copy()
    wl.det_up = np.array([[hf_up], [ex_up]], np.uint64)
    wl.det_dn = np.array([[hf_dn], [ex_dn]], np.uint64)
    wl.ci_coef = np.array([0.96, -0.05])
    ctx = _host_ctx(wl)
    for spin, (hf, ex) in enumerate(((hf_up, ex_up), (hf_dn, ex_dn))):
        dets, deg, ph = ctx.spin_dets(spin)
        assert int(dets[0, 0]) == hf and int(dets[1, 0]) == ex
        assert list(deg) == [0, 1]
        # column of MO 7 (index 6) takes MO 12 (index 11): the ascending order moves it past MOs 8, 9 (up) / 8 (down)
        assert ph[1] == (1 if spin == 0 else -1)


def test_table1_ordering():
    """Table 1 / Eq. 3: 4 electrons in 8 orbitals sort as 15, 23, 27, 29, 30, 39, 43, 45, ...
    (tests/golden/table1_omega_order.txt: decimal, binary and occupied orbitals)."""
    table = _golden("table1_omega_order.txt")
    for idx, dec, binary, occ in table:
        assert int(binary, 2) == int(dec) == sum(1 << (int(c) - 1) for c in occ)
    vals = [sum(1 << m for m in s) for s in combinations(range(8), 4)]
    rng = np.random.default_rng(0)
    vals = np.array(vals, np.uint64)[rng.permutation(len(vals))]
    order = pkg.omega_sort(vals[:, None])
    got = [int(v) for v in vals[order]]
    assert got[:len(table)] == [int(r[1]) for r in table]
    assert got == sorted(got)


def test_sec5_operation_counts_reproduce_the_paper():
    """Sec. 5's cost model (tests/golden/sec5_costs.txt): for a 9 x 9 matrix a full inversion
    costs 1.71 times two Sherman-Morrison substitutions, and with the Hartree-Fock determinants
    as a fixed reference the up and down determinants of Table 4
    (tests/golden/table4_excitation_degrees.txt) would need 3.46 substitutions on average."""
    from paper_1510_00730_gb300 import costs
    want = {r[0]: float(r[1]) for r in _golden("sec5_costs.txt")}
    ratio = costs.inversion_flops(9) / (2 * costs.substitution_flops(9))
    assert round(ratio, 2) == want["inversion_over_two_substitutions_n9"]
    t4 = np.array([[int(x) for x in r] for r in _golden("table4_excitation_degrees.txt")])
    assert list(t4[:, 0]) == list(range(9))
    avg = costs.fixed_reference_substitutions(t4[:, 2], t4[:, 3])
    assert round(avg, 2) == want["fixed_reference_substitutions"]
    # the printed total of Table 4's product column is the 10^6-determinant wave function
    assert abs(int(t4[:, 1].sum()) - 1_000_000) <= 1_000


def test_omega_key_is_xor_of_words_unsigned():
    """Eq. 3 with N_int = 2: the key is the xor of the words compared as an
    unsigned integer (the -2^63 shift only emulates that in Fortran); equal
    keys are ordered by the words from the last to the first."""
    d = np.array([[0b1111, 0], [0b0111, 1 << 63], [0b0110, 0b1001], [0b1001, 0b0110], [0, 0b1111]], np.uint64)
    order = pkg.omega_sort(d)
    keys = [int(d[i, 0]) ^ int(d[i, 1]) for i in order]
    assert keys == sorted(keys)
    assert int(d[order[-1], 1]) == 1 << 63  # largest unsigned key sorts last
    tied = [i for i in order if (int(d[i, 0]) ^ int(d[i, 1])) == 0b1111]
    assert [int(d[i, 1]) for i in tied] == sorted(int(d[i, 1]) for i in tied)


def test_ci_matrix_column_major_and_complete():
    """Sec. 2.1: C in coordinate format over the distinct determinants, ordered by
    N_up * j + i (column by column), exactly one entry per product."""
    wl = synth.oxygen_like_1k(n_walk=1)
    ctx = _host_ctx(wl)
    st = ctx.stats()
    row, col, val = ctx.ci_matrix()
    assert st["n_det"] == wl.n_det == len(val)
    key = col.astype(np.int64) * st["n_det_up"] + row
    assert np.all(np.diff(key) > 0)
    up, _, _ = ctx.spin_dets(0)
    dn, _, _ = ctx.spin_dets(1)
    assert len(np.unique(up, axis=0)) == len(up) == st["n_det_up"]
    got = {(int(up[r, 0]), int(dn[c, 0])): v for r, c, v in zip(row, col, val)}
    want = {(int(a[0]), int(b[0])): v for a, b, v in zip(wl.det_up, wl.det_dn, wl.ci_coef)}
    assert got == want


def test_excitation_records_and_phase():
    """Each distinct determinant is stored as an excitation of the reference (the
    spin part of the largest |c_k| product); its phase is the parity of the
    permutation that sorts the substituted columns ascending (checked by brute
    force); the list is grouped by degree with the reference first."""
    wl = synth.chlorine_like_100k(n_walk=1)
    ctx = _host_ctx(wl)
    kref = int(np.argmax(np.abs(wl.ci_coef)))
    for spin, src in ((0, wl.det_up), (1, wl.det_dn)):
        dets, deg, ph = ctx.spin_dets(spin)
        assert np.array_equal(dets[0], src[kref])
        assert deg[0] == 0 and ph[0] == 1
        assert np.all(np.diff(deg) >= 0)

        def occ(w):
            return [64 * q + b for q in range(len(w)) for b in range(64) if (int(w[q]) >> b) & 1]
        ref = occ(dets[0])
        for t in range(0, len(dets), 7):
            o = occ(dets[t])
            holes = [a for a, m in enumerate(ref) if m not in o]
            parts = sorted(set(o) - set(ref))
            assert len(holes) == deg[t]
            cols = list(ref)
            for a, p in zip(holes, parts):
                cols[a] = p
            assert ph[t] == perm_parity(cols)


def test_excitation_ratio_identity_against_oracle():
    """The table-method identity used by the kernels (Sec. 5; Eq. 4 for one
    column): D_I / D_ref = eps_I det T[h, p] with T = S_ref^-1 Phi, checked in
    numpy with the library's excitation records against oracle determinants."""
    wl = synth.oxygen_like_1k(n_walk=3)
    ctx = _host_ctx(wl)
    for spin in (0, 1):
        dets, deg, ph = ctx.spin_dets(spin)
        lg, sg, _ = oracle.spin_dets(wl, spin, dets)
        n = wl.n_up if spin == 0 else wl.n_dn
        e0 = 0 if spin == 0 else wl.n_up
        ref = [b for b in range(64) if (int(dets[0, 0]) >> b) & 1]
        for w in range(wl.n_walk):
            phi = oracle.mo_eval(wl, wl.R[w])[e0:e0 + n, 0, :]
            T = np.linalg.solve(phi[:, ref], phi)
            for t in range(len(dets)):
                o = [b for b in range(64) if (int(dets[t, 0]) >> b) & 1]
                h = [a for a, m in enumerate(ref) if m not in o]
                p = sorted(set(o) - set(ref))
                r = ph[t] * (np.linalg.det(T[np.ix_(h, p)]) if h else 1.0)
                want = sg[w, t] * sg[w, 0] * math.exp(lg[w, t] - lg[w, 0])
                assert abs(r - want) <= 1e-9 * max(1.0, abs(want)), (spin, w, t, r, want)


@pytest.mark.parametrize("bad", ["popcount", "beyond_mo", "duplicate", "degree"])
def test_input_validation(bad):
    wl = synth.oxygen_like_1k(n_walk=1) if bad != "degree" else synth.chlorine_like_100k(n_walk=1)
    du, dd, c = wl.det_up.copy(), wl.det_dn.copy(), wl.ci_coef.copy()
    if bad == "popcount":
        du[5, 0] |= np.uint64(1 << 19) if not (int(du[5, 0]) >> 19) & 1 else np.uint64(1 << 18)
    elif bad == "beyond_mo":
        du[5, 0] = np.uint64((int(du[5, 0]) & ~1) | (1 << 25)) if int(du[5, 0]) & 1 else np.uint64((int(du[5, 0]) & ~2) | (1 << 25))
    elif bad == "duplicate":
        du[7], dd[7] = du[3], dd[3]
    elif bad == "degree":
        du[9, 0] = np.uint64(sum(1 << m for m in range(4)) | sum(1 << m for m in range(20, 25)))  # degree 5
    ctx = pkg.Context(device=binding.NO_DEVICE)
    ctx.set_system(wl.n_up, wl.n_dn, wl.Z, wl.nuc_xyz)
    ctx.set_orbitals(wl.shell_l, wl.shell_center, wl.shell_nprim, wl.alpha, wl.coef, wl.mo_coef)
    with pytest.raises(pkg.MdetError) as ei:
        ctx.set_ci_expansion(du, dd, c)
    assert ei.value.status == 5  # MDET_E_INPUT


def test_call_order_and_no_device_errors():
    wl = synth.oxygen_like_1k(n_walk=1)
    ctx = pkg.Context(device=binding.NO_DEVICE)
    with pytest.raises(pkg.MdetError) as ei:
        ctx.set_ci_expansion(wl.det_up, wl.det_dn, wl.ci_coef)
    assert ei.value.status == 2  # MDET_E_STATE
    with pytest.raises(pkg.MdetError):
        ctx.set_system(3, 4, wl.Z, wl.nuc_xyz)  # n_up < n_dn
    ctx = _host_ctx(wl)
    with pytest.raises(pkg.MdetError) as ei:
        ctx.evaluate_host(wl.R)
    assert ei.value.status == 7  # MDET_E_NODEVICE


def test_unique_counts_follow_generator():
    """The distinct-determinant counts the library finds equal the ones the
    workload was drawn with (N_det^sigma ~ 0.9 N_det^0.6, Sec. 4 fit)."""
    wl = synth.chlorine_like_100k(n_walk=1)
    st = _host_ctx(wl).stats()
    assert (st["n_det_up"], st["n_det_dn"]) == wl.meta["n_unique"] == (900, 900)
    assert st["max_degree"] == [4, 4]
    assert sum(st["degree_hist"][0]) == 900


def test_uneven_batch_generator_ranges():
    """The 64-expansion uneven workload follows its recipe: 8-34 electrons split
    as evenly as possible, 40-160 AOs, N_MO = max(round(0.73 N_AO), N_up + 4),
    10^3-10^6 determinants, 256-4,096 walkers."""
    wls = synth.batched_uneven()
    assert len(wls) == 64
    for wl in wls:
        ne = wl.n_up + wl.n_dn
        assert 8 <= ne <= 34 and wl.n_up - wl.n_dn in (0, 1)
        assert 40 <= wl.n_ao <= 160
        assert wl.n_mo == min(wl.n_ao, 255, max(int(round(0.73 * wl.n_ao)), wl.n_up + 4))
        assert 1000 <= wl.n_det <= 1_000_000
        assert 256 <= wl.n_walk <= 4096
    nd = np.log10([wl.n_det for wl in wls])
    assert nd.min() < 3.6 and nd.max() > 5.4   # spans the decades

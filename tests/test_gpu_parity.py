"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs (criteria in tests/parity.py). FP64 path: log|Psi| within 1e-10
times the conditioning kappa of the determinant sum, grad Psi / Psi and
Lap Psi / Psi within 1e-8 relative to max(|x|, the walker's rms), no kappa.
Mixed path (double-float FP32 for orbitals, ratios and cofactors; FP64 LU and
contraction): 1e-9 on log|Psi| (times kappa) and 1e-6 on the derivatives, and
the 99th percentile over walkers below 1e-5 relative."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth
from tests.parity import compare, walker_quantiles

PRECISIONS = [pytest.param(pkg.PRECISION_FP64, id="fp64"), pytest.param(pkg.PRECISION_MIXED, id="mixed")]
TOL = {pkg.PRECISION_FP64: dict(tol_psi=1e-10, tol_der=1e-8), pkg.PRECISION_MIXED: dict(tol_psi=1e-9, tol_der=1e-6)}

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_double_float_exp_and_product():
    """The mixed path's double-float exp (Cody-Waite reduction + Taylor series)
    and product against CUDA's FP64 exp and FP64 arithmetic. For -50 <= t <= 0
    the relative error is below 2e-14 plus exp's conditioning |t| times the
    rounding of t to double-float (2^-48); below -50 the low word runs into
    FP32's subnormal range, so the bound is absolute, (2e-14 + 87 * 2^-48) exp(-50),
    far below any AO value that matters next to the others of its row."""
    from paper_1510_00730_gb300.binding import selftest_df32
    x = -torch.cat([torch.logspace(-8, math.log10(87.0), 20000, dtype=torch.float64),
                    torch.rand(20000, dtype=torch.float64) * 87.0, torch.zeros(1, dtype=torch.float64)]).to("cuda:0")
    y_df, y_ref, prod = selftest_df32(x)
    err = (y_df - y_ref).abs()
    hi = x >= -50.0
    bound = 2e-14 + x[hi].abs() * 2.0 ** -48
    rel = (err[hi] / y_ref[hi].abs() / bound).max().item()
    assert rel < 1.0, rel
    assert err[~hi].max().item() < (2e-14 + 87.0 * 2.0 ** -48) * math.exp(-50.0)
    xn = x.cpu().numpy()
    want = xn * np.roll(xn, -1) + xn
    got = prod.cpu().numpy()
    scale = np.abs(xn * np.roll(xn, -1)) + np.abs(xn) + 1e-300
    assert np.max(np.abs(got - want) / scale) < 1e-13


def test_coulomb_inverse_square_root():
    """The epilogue's 1/r in the Coulomb sums of E_L (an FP32 estimate refined by two
    Newton-Raphson steps in FP64) against CUDA's FP64 1.0 / sqrt. A step squares the
    estimate's relative error (below 2^-21), so what remains are the roundings of the last
    step, and the reference's own two: within 8 * 2^-53 relative over squared distances
    from 1e-12 to 1e12. Arguments outside the estimate's range take 1.0 / sqrt itself and
    must agree exactly."""
    from paper_1510_00730_gb300.binding import selftest_inv_r
    x = torch.cat([torch.logspace(-12, 12, 40000, dtype=torch.float64),
                   torch.rand(40000, dtype=torch.float64) * 100.0 + 1e-3]).to("cuda:0")
    y, ref = selftest_inv_r(x)
    rel = ((y - ref).abs() / ref).max().item()
    assert rel <= 8 * 2.0 ** -53, rel
    special = torch.tensor([0.0, 1e-300, 2.0 ** -100, 2.0 ** 100, 1e300, math.inf], dtype=torch.float64,
                           device="cuda:0")
    ys, refs = selftest_inv_r(special)
    assert torch.equal(ys, refs)


def _gpu_eval(ctx, R):
    Rt = torch.from_numpy(np.ascontiguousarray(R)).to("cuda:0")
    out = ctx.evaluate(Rt)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.fixture(scope="module")
def o2100():
    wl = synth.oxygen_like_1k(n_walk=2100, seed=123)
    return wl, oracle.evaluate(wl)


@pytest.fixture(scope="module")
def o1k():
    wl = synth.oxygen_like_1k(n_walk=64)
    return wl, oracle.evaluate(wl)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_oxygen_like_1k_all_walkers(o1k, prec):
    wl, ref = o1k
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    got = _gpu_eval(ctx, wl.R)
    rep = compare(got, ref, **TOL[prec])
    assert rep["ok"], rep
    q = walker_quantiles(got, ref)
    assert all(q[k]["p99"] < 1e-5 for k in q), q
    assert np.all(got["status"] & (pkg.WS_REF_SINGULAR | pkg.WS_NONFINITE) == 0)


def test_fp64_per_determinant_ratios(o1k):
    """Every distinct spin determinant: D_I / D_ref from the table method equals
    the oracle's ratio of full LU determinants. The k x k determinant of table
    entries cancels terms as large as the permanent of |T[h, p]|, and T itself
    carries the conditioning of the reference Slater matrix, so the absolute
    bound is 1e-14 (about 90 ulps) * cond(S_ref) * max(per|T[h,p]|, |r|, 1)."""
    from itertools import permutations
    wl, _ = o1k
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    _gpu_eval(ctx, wl.R)
    r_up, r_dn, ld0, sg0 = ctx.ratios(wl.n_walk)
    for spin, r in ((0, r_up), (1, r_dn)):
        dets, _, _ = ctx.spin_dets(spin)
        lg, sg, _ = oracle.spin_dets(wl, spin, dets)
        want = sg * sg[:, :1] * np.exp(lg - lg[:, :1])
        n, e0 = (wl.n_up, 0) if spin == 0 else (wl.n_dn, wl.n_up)
        ref_occ = [b for b in range(64) if (int(dets[0, 0]) >> b) & 1]
        occs = [[b for b in range(64) if (int(d[0]) >> b) & 1] for d in dets]
        holes = [[a for a, m in enumerate(ref_occ) if m not in o] for o in occs]
        parts = [sorted(set(o) - set(ref_occ)) for o in occs]
        for w in range(wl.n_walk):
            phi = oracle.mo_eval(wl, wl.R[w])[e0:e0 + n, 0, :]
            cond = np.linalg.cond(phi[:, ref_occ])
            T = np.abs(np.linalg.solve(phi[:, ref_occ], phi))
            for t in range(len(dets)):
                M = T[np.ix_(holes[t], parts[t])]
                k = M.shape[0]
                per = sum(np.prod([M[i, q[i]] for i in range(k)]) for q in permutations(range(k))) if k else 1.0
                bound = 1e-14 * max(cond, 1.0) * max(per, abs(want[w, t]), 1.0)
                assert abs(r[w, t] - want[w, t]) <= bound, (spin, w, t, r[w, t], want[w, t], bound)
        assert np.all(np.abs(ld0[:, spin] - lg[:, 0]) < 1e-11)
        assert np.all(sg0[:, spin] == sg[:, 0])


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n_walk", [1, 31, 77, 130, 257])
def test_ragged_walker_counts(n_walk, prec):
    """Walker counts that are not multiples of the 32/128-walker tiles."""
    wl = synth.oxygen_like_1k(n_walk=n_walk, seed=4242 + n_walk)
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    rep = compare(_gpu_eval(ctx, wl.R), ref, **TOL[prec])
    assert rep["ok"], rep


@pytest.mark.parametrize("chunks", [1, 2, 3, 4])
def test_mixed_walker_chunks(chunks):
    """Mixed precision with the batch cut into chunks pipelined over two streams
    (ragged: 900 walkers = 3.5 tiles of 256)."""
    wl = synth.oxygen_like_1k(n_walk=900, seed=99)
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    ctx.set_walker_chunks(chunks)
    rep = compare(_gpu_eval(ctx, wl.R), ref, **TOL[pkg.PRECISION_MIXED])
    assert rep["ok"], rep
    assert ctx.last_chunks == chunks


@pytest.mark.parametrize("prec,chunks,blocks,esc", [(pkg.PRECISION_MIXED, 8, 0, False), (pkg.PRECISION_MIXED, 5, 3, False),
                                                    (pkg.PRECISION_MIXED, 3, 1, False), (pkg.PRECISION_MIXED, 3, 0, True),
                                                    (pkg.PRECISION_FP64, 1, 2, False)])
def test_persistent_contraction_grids(o2100, prec, chunks, blocks, esc):
    """The contraction on persistent grids whose warps draw work items from a
    counter: 8, 5 and 3 pipelined chunks of a ragged 2,100-walker batch, grids of 1
    to 3 blocks (every warp takes many items) and the FP64 path with a capped grid.
    The mixed fallback tolerance is tightened to 1e-7, so that every walker meets
    the test tolerances: the refinement then re-evaluates tens of walkers flagged by
    the pipelined chunks, by full LU or (esc) by the FP64 ratio table first. Stage
    times come back for every stage."""
    wl, ref = o2100
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    ctx.set_tuning(walker_chunks=chunks, spmm_blocks=blocks)
    if prec == pkg.PRECISION_MIXED:
        ctx.set_fallback(1e-7, 512)
        ctx.set_escalation(pkg.Context.ESCALATE_ALWAYS if esc else pkg.Context.ESCALATE_AUTO)
    ctx.set_profiling(True)
    got = _gpu_eval(ctx, wl.R)
    rep = compare(got, ref, **TOL[prec])
    assert rep["ok"], rep
    assert ctx.last_chunks == chunks
    assert bool(((got["status"] & pkg.WS_ESCALATED) != 0).any()) == esc
    # 6 kernels per chunk; the fallback: FP64 full LU 5; the mixed refinement 10, or 14 with
    # the FP64 table (this small expansion escalates only when forced)
    assert ctx.last_kernels == 6 * chunks + (5 if prec == pkg.PRECISION_FP64 else (14 if esc else 10))
    prof = ctx.profile()
    assert all(v > 0 for k, v in prof.items() if k != "zero"), prof
    # mode 2: the contraction kernels time themselves (global-timer stamps, no events); the
    # results and the kernel count are unchanged, the other stages read zero, no timeline
    ctx.set_profiling(2)
    got = _gpu_eval(ctx, wl.R)
    assert compare(got, ref, **TOL[prec])["ok"]
    assert ctx.last_kernels == 6 * chunks + (5 if prec == pkg.PRECISION_FP64 else (14 if esc else 10))
    prof2 = ctx.profile()
    assert all(v == 0 for k, v in prof2.items() if k != "contract"), prof2
    assert 0.2 * prof["contract"] < prof2["contract"] < 5.0 * prof["contract"], (prof, prof2)
    with pytest.raises(RuntimeError):
        ctx.timeline()
    ctx.set_profiling(False)


def test_fp64_grow_and_shrink_batch(o1k):
    """One context, batches of varying size (scratch grows once, stale columns ignored)."""
    wl, ref = o1k
    ctx = pkg.Context.from_workload(wl, device=0)
    for n in (8, 64, 5, 40):
        rep = compare(_gpu_eval(ctx, wl.R[:n]), {k: v[:n] for k, v in ref.items()})
        assert rep["ok"], (n, rep)


def test_empty_batch_is_noop(o1k):
    wl, _ = o1k
    ctx = pkg.Context.from_workload(wl, device=0)
    out = ctx.evaluate(torch.empty(0, wl.n_elec, 3, dtype=torch.float64, device="cuda:0"))
    torch.cuda.synchronize()
    assert out["log_abs_psi"].numel() == 0


@pytest.mark.parametrize("prec", PRECISIONS)
def test_single_determinant(prec):
    """N_det = 1: the plain Slater determinant product (Table 2, first row)."""
    wl = synth.oxygen_like_1k(n_walk=32)
    k = 11
    wl.det_up, wl.det_dn, wl.ci_coef = wl.det_up[k:k + 1], wl.det_dn[k:k + 1], np.array([0.5])
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    rep = compare(_gpu_eval(ctx, wl.R), ref, **TOL[prec])
    assert rep["ok"], rep


@pytest.mark.parametrize("prec", PRECISIONS)
def test_fci_expansion_all_degrees(prec):
    """Full CI of 4 up / 4 down electrons in 10 MOs (210 x 210 = 44,100 products,
    excitation degrees 0..4 in both spins)."""
    from itertools import combinations
    wl = synth.oxygen_like_1k(n_walk=40)
    wl.mo_coef = wl.mo_coef[:, :10].copy()
    subsets = list(combinations(range(10), 4))
    bits = np.array([[sum(1 << m for m in s)] for s in subsets], np.uint64)
    rng = np.random.default_rng(9)
    cu = rng.normal(size=len(subsets))
    I, J = np.meshgrid(np.arange(210), np.arange(210), indexing="ij")
    wl.det_up, wl.det_dn = bits[I.ravel()], bits[J.ravel()]
    wl.ci_coef = cu[I.ravel()] * cu[J.ravel()] + 0.1 * rng.normal(size=I.size)
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    assert ctx.stats()["max_degree"] == [4, 4]
    rep = compare(_gpu_eval(ctx, wl.R), ref, **TOL[prec])
    assert rep["ok"], rep


def test_host_api_matches_device_api(o1k):
    wl, _ = o1k
    ctx = pkg.Context.from_workload(wl, device=0)
    dev = _gpu_eval(ctx, wl.R)
    host = ctx.evaluate_host(wl.R)
    # the contraction accumulates with atomics, so two runs agree to rounding, not bitwise
    for k in ("log_abs_psi", "grad", "lap", "e_local"):
        np.testing.assert_allclose(host[k], dev[k], rtol=1e-9, atol=1e-9)
    assert np.array_equal(host["sign"], dev["sign"])


def test_coincident_same_spin_electrons_flagged():
    """Two up electrons at the same point: every up Slater matrix is singular
    (Psi = 0 on this node). Rounding may leave a tiny nonzero pivot, so the
    walker is flagged singular or ill-conditioned; its neighbours are unaffected."""
    wl = synth.oxygen_like_1k(n_walk=8)
    R = wl.R.copy()
    R[3, 1] = R[3, 0]
    ref = oracle.evaluate(wl, R=R)
    assert ref["sign"][3] == 0
    ctx = pkg.Context.from_workload(wl, device=0)
    got = _gpu_eval(ctx, R)
    assert got["status"][3] & (pkg.WS_REF_SINGULAR | pkg.WS_REF_ILLCOND)
    assert not np.any(got["status"][[0, 1, 2, 4, 5, 6, 7]] & (pkg.WS_REF_SINGULAR | pkg.WS_REF_ILLCOND))
    keep = [i for i in range(8) if i != 3]
    rep = compare({k: v[keep] for k, v in got.items()}, {k: v[keep] for k, v in ref.items()})
    assert rep["ok"], rep


@pytest.mark.slow
@pytest.mark.parametrize("prec", PRECISIONS)
def test_chlorine_like_100k_sampled(prec):
    """10^5 determinants, 4,096 walkers on the GPU; 32 sampled walkers checked."""
    wl = synth.chlorine_like_100k()
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    got = _gpu_eval(ctx, wl.R)
    idx = np.random.default_rng(1).choice(wl.n_walk, 32, replace=False)
    ref = oracle.evaluate(wl, R=wl.R[idx])
    rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL[prec])
    assert rep["ok"], rep
    assert np.all(np.isfinite(got["log_abs_psi"]))


@pytest.fixture(scope="module")
def cl750():
    wl = synth.chlorine_like_750k()
    idx = np.random.default_rng(2).choice(wl.n_walk, 64, replace=False)
    return wl, idx, oracle.evaluate(wl, R=wl.R[idx])


@pytest.mark.slow
@pytest.mark.parametrize("prec", PRECISIONS)
def test_chlorine_like_750k_full_size_sampled(cl750, prec):
    """The full 750k-determinant, 8,192-walker workload in the launch
    configuration the benchmark times; 64 sampled walkers checked against the
    oracle, every walker finite, 99th percentile of the relative errors < 1e-5.
    No sampled walker is left out for its conditioning (n_ill == 0), and on the
    FP64 path every sampled walker's gradient and Laplacian is within 1e-8 of the
    oracle's with no conditioning factor."""
    wl, idx, ref = cl750
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    got = _gpu_eval(ctx, wl.R)
    assert np.all(np.isfinite(got["log_abs_psi"]))
    assert np.all(got["status"] & (pkg.WS_REF_SINGULAR | pkg.WS_NONFINITE) == 0)
    sub = {k: v[idx] for k, v in got.items()}
    rep = compare(sub, ref, **TOL[prec])
    assert rep["ok"], rep
    assert rep["n_ill"] == 0 and rep["n_unsigned"] == 0, rep
    if prec == pkg.PRECISION_FP64:
        assert rep["grad"] <= 1e-8 and rep["lap"] <= 1e-8, rep
    q = walker_quantiles(sub, ref)
    assert all(q[k]["p99"] < 1e-5 for k in q), q


@pytest.mark.parametrize("impl,ec", [(0, 4), (0, 6), (0, 8), (1, 4), (1, 8), (2, 4)])
@pytest.mark.parametrize("name", ["oxygen_like_1k", "chlorine_like_100k"])
def test_mixed_orbital_products(name, impl, ec):
    """Every orbital product of the mixed path against the oracle: exact BF16
    digit products on the tcgen05 tensor cores (mo_impl 2, the default), the same
    digits on warp-level mma.sync (0) and the compensated dot product on the CUDA
    cores (1), with the electron blocks of the last two; the 10^5 expansion on 32
    sampled walkers."""
    wl = synth.WORKLOADS[name]()
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    assert ctx.tuning()["mo_impl"] == 2
    ctx.set_tuning(mo_ec=ec, mo_impl=impl)
    assert ctx.tuning()["mo_impl"] == impl
    got = _gpu_eval(ctx, wl.R)
    idx = np.arange(wl.n_walk) if wl.n_walk <= 64 else np.random.default_rng(2).choice(wl.n_walk, 32, replace=False)
    ref = oracle.evaluate(wl, R=wl.R[idx])
    rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL[pkg.PRECISION_MIXED])
    assert rep["ok"], rep


@pytest.mark.slow
@pytest.mark.parametrize("prec", PRECISIONS)
def test_exchange_antisymmetry_full_size(cl750, prec):
    """A property that holds at any size, checked on every walker of the
    full-size workload in the bench's launch configuration: exchanging two
    same-spin electrons (an up pair and a down pair) flips the sign of Psi,
    keeps log|Psi| and permutes the gradients and Laplacians (Eq. 1: each spin
    factor is a determinant)."""
    wl = cl750[0] if isinstance(cl750, tuple) else cl750
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    a = _gpu_eval(ctx, wl.R)
    for i, j in ((0, 3), (wl.n_up + 1, wl.n_up + 6)):
        Rs = wl.R.copy()
        Rs[:, [i, j]] = Rs[:, [j, i]]
        b = _gpu_eval(ctx, Rs)
        perm = np.arange(wl.n_elec)
        perm[[i, j]] = perm[[j, i]]
        ok = (a["status"] & (pkg.WS_REF_SINGULAR | pkg.WS_PSI_ZERO | pkg.WS_NONFINITE)) == 0
        assert ok.mean() > 0.99
        assert np.all(b["sign"][ok] == -a["sign"][ok])
        d_log = np.abs(b["log_abs_psi"] - a["log_abs_psi"])[ok]
        gs = np.sqrt(np.mean(a["grad"] ** 2, axis=(1, 2)))[:, None, None]
        d_grad = (np.abs(b["grad"] - a["grad"][:, perm]) / np.maximum(np.abs(a["grad"][:, perm]), gs)).max(axis=(1, 2))[ok]
        ls = np.sqrt(np.mean(a["lap"] ** 2, axis=1))[:, None]
        d_lap = (np.abs(b["lap"] - a["lap"][:, perm]) / np.maximum(np.abs(a["lap"][:, perm]), ls)).max(axis=1)[ok]
        tol = 1e-9 if prec == pkg.PRECISION_FP64 else 1e-7
        for name, d in (("log", d_log), ("grad", d_grad), ("lap", d_lap)):
            assert np.percentile(d, 99) <= tol, (name, np.percentile(d, 99), d.max())
            assert d.max() <= 1e3 * tol, (name, d.max())


@pytest.mark.parametrize("name", ["oxygen_like_1k", "chlorine_like_100k"])
def test_mixed_double_float_contraction(name):
    """The optional double-float contraction of the mixed path (contract_impl = 1)
    against the oracle; the 10^5 expansion on 32 sampled walkers."""
    wl = synth.WORKLOADS[name]()
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    ctx.set_tuning(contract_impl=1)
    assert ctx.tuning()["contract_impl"] == 1
    got = _gpu_eval(ctx, wl.R)
    idx = np.arange(wl.n_walk) if wl.n_walk <= 64 else np.random.default_rng(3).choice(wl.n_walk, 32, replace=False)
    ref = oracle.evaluate(wl, R=wl.R[idx])
    rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL[pkg.PRECISION_MIXED])
    assert rep["ok"], rep


@pytest.mark.slow
def test_mixed_double_float_contraction_full_size(cl750):
    wl, idx, ref = cl750
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    ctx.set_tuning(contract_impl=1)
    got = _gpu_eval(ctx, wl.R)
    rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL[pkg.PRECISION_MIXED])
    assert rep["ok"], rep


def test_binding_refuses_mismatched_buffers(o1k):
    """Buffers of the wrong shape, dtype, layout or device are refused before any
    kernel runs (the kernels would otherwise read or write out of bounds)."""
    wl, _ = o1k
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    R = torch.from_numpy(wl.R).to("cuda:0")
    with pytest.raises(ValueError):
        ctx.evaluate(R.float())
    with pytest.raises(ValueError):
        ctx.evaluate(R[:, :4])
    with pytest.raises(ValueError):
        ctx.evaluate(R.cpu())
    with pytest.raises(ValueError):
        ctx.evaluate(R.transpose(0, 1).contiguous().transpose(0, 1))
    out = ctx.alloc_outputs(wl.n_walk - 1)
    with pytest.raises(ValueError):
        ctx.evaluate(R, out=out)
    with pytest.raises(ValueError):
        ctx.evaluate_host(wl.R, out=dict(log_abs_psi=np.empty(3)))
    good = ctx.evaluate(R)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(good["log_abs_psi"].cpu().numpy()))

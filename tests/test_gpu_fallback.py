"""Stability control: walkers whose reference Slater matrix is too
ill-conditioned for the ratio table are re-evaluated by full LU of every
determinant (the paper's O(N^3) fallback, Sec. 2.2), in FP64 on the GPU."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _eval(ctx, R):
    out = ctx.evaluate(torch.from_numpy(np.ascontiguousarray(R)).to("cuda:0"))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


ESC = pkg.Context.ESCALATE_ALWAYS
NO_ESC = pkg.Context.ESCALATE_NEVER
MODES = [(pkg.PRECISION_FP64, None), (pkg.PRECISION_MIXED, NO_ESC), (pkg.PRECISION_MIXED, ESC)]


@pytest.mark.parametrize("prec,mode", MODES)
def test_forced_fallback_for_every_walker_matches_oracle(prec, mode):
    """With a tiny tolerance every walker goes through the full-LU path (mixed:
    directly, or after the FP64 re-evaluation); at most `cap` of them are
    re-evaluated, the rest keep the table result and are flagged."""
    wl = synth.oxygen_like_1k(n_walk=40, seed=31)
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    if mode is not None:
        ctx.set_escalation(mode)
    ctx.set_fallback(1e-30, max_walkers=32)
    got = _eval(ctx, wl.R)
    fb = (got["status"] & pkg.WS_FALLBACK) != 0
    assert fb.sum() == 32
    assert np.all(got["status"][~fb] & pkg.WS_REF_ILLCOND)
    # with escalation the full-LU path is reached through the FP64 re-evaluation
    esc = (got["status"] & pkg.WS_ESCALATED) != 0
    assert np.array_equal(esc, fb) if mode == ESC else not esc.any()
    rep = compare(got, ref, tol_psi=1e-10, tol_der=1e-8) if prec == pkg.PRECISION_FP64 else \
        compare(got, ref, tol_psi=1e-9, tol_der=1e-6)
    assert rep["ok"], rep
    # the re-evaluated walkers carry FP64 accuracy in both precisions
    rep_fb = compare({k: v[fb] for k, v in got.items()}, {k: v[fb] for k, v in ref.items()},
                     tol_psi=1e-10, tol_der=1e-8)
    assert rep_fb["ok"], rep_fb


def test_forced_fallback_on_full_ci():
    from itertools import combinations
    wl = synth.oxygen_like_1k(n_walk=10)
    wl.mo_coef = wl.mo_coef[:, :9].copy()
    subsets = list(combinations(range(9), 4))
    bits = np.array([[sum(1 << m for m in s)] for s in subsets], np.uint64)
    rng = np.random.default_rng(4)
    I, J = np.meshgrid(np.arange(len(subsets)), np.arange(len(subsets)), indexing="ij")
    wl.det_up, wl.det_dn = bits[I.ravel()], bits[J.ravel()]
    wl.ci_coef = rng.normal(size=I.size)
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    ctx.set_fallback(1e-30, max_walkers=64)
    got = _eval(ctx, wl.R)
    assert np.all(got["status"] & pkg.WS_FALLBACK)
    rep = compare(got, ref, tol_psi=1e-10, tol_der=1e-8)
    assert rep["ok"], rep


@pytest.mark.parametrize("prec", [pkg.PRECISION_FP64, pkg.PRECISION_MIXED])
def test_ill_conditioned_reference_walkers_are_caught(prec):
    """A small expansion where some walkers have a reference Slater matrix with
    cond_1 near 1e8 and strong cancellation in the derivative sums: with the
    default tolerance every walker meets the oracle (the bad ones through the
    fallback, flagged), and the flagged set contains the worst-conditioned one."""
    wls = synth.batched_uneven(n_exp=6, walkers=(40, 300), n_det_range=(300, 20000), elec_range=(4, 20),
                               ao_range=(20, 60), seed=555)
    rng = np.random.default_rng(3)
    new_R = [synth.make_walkers(rng, wl.n_walk, wl.n_elec) for wl in wls]
    wl, R = wls[1], new_R[1]       # walker 2 has cond_1(S_ref_up) = 8e7
    idx = np.arange(12)
    ref = oracle.evaluate(wl, R=R[idx])
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    got = {k: v[idx] for k, v in _eval(ctx, R).items()}
    assert got["status"][2] & pkg.WS_FALLBACK
    tol = dict(tol_psi=1e-10, tol_der=1e-8) if prec == pkg.PRECISION_FP64 else dict(tol_psi=1e-9, tol_der=1e-6)
    rep = compare(got, ref, **tol)
    assert rep["ok"], rep


def _walker_errors(got, ref):
    """Per-walker worst relative error over log|Psi|, the gradient and the
    Laplacian (the gradient and Laplacian relative to max(|x|, the walker's rms))."""
    e_log = np.abs(got["log_abs_psi"] - ref["log_abs_psi"])
    gs = np.sqrt(np.mean(ref["grad"] ** 2, axis=(1, 2)))[:, None, None]
    e_grad = (np.abs(got["grad"] - ref["grad"]) / np.maximum(np.abs(ref["grad"]), gs)).max(axis=(1, 2))
    ls = np.sqrt(np.mean(ref["lap"] ** 2, axis=1))[:, None]
    e_lap = (np.abs(got["lap"] - ref["lap"]) / np.maximum(np.abs(ref["lap"]), ls)).max(axis=1)
    return np.maximum(e_log, np.maximum(e_grad, e_lap))


@pytest.fixture(scope="module")
def o2100_fb():
    # 2,100 walkers: among them references with cond_1 up to 1e6 and CI sums that
    # cancel by up to 2e4, the cases an estimate without the CI-sum conditioning missed
    wl = synth.oxygen_like_1k(n_walk=2100, seed=123)
    return wl, oracle.evaluate(wl)


@pytest.mark.parametrize("prec", [pkg.PRECISION_FP64, pkg.PRECISION_MIXED])
def test_error_estimate_bounds_the_error(o2100_fb, prec):
    """With re-evaluation off (infinite tolerance, estimates still computed), every
    walker's error against the oracle stays below its l1 estimate (plus 1e-12 for
    the oracle's own rounding). The estimate is a worst-case bound, typically
    10^3-10^4 above the error, but not a vacuous one: the median walker sits two
    orders of magnitude below the path's default tolerance."""
    wl, ref = o2100_fb
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    default_tol = ctx.fallback[0]
    ctx.set_fallback(1e30, 1)
    got = _eval(ctx, wl.R)
    _, est = ctx.error_estimates(wl.n_walk)
    err = _walker_errors(got, ref)
    ratio = err / (est[:, 0] + 1e-12)
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 1.0, (worst, err[worst], est[worst], ref["kappa"][worst])
    assert np.median(err) <= np.median(est[:, 0]) <= default_tol / 100
    ctx.close()


@pytest.mark.parametrize("prec,mode", MODES)
def test_default_tolerance_meets_each_path_target(o2100_fb, prec, mode):
    """With the default fallback (1e-8 FP64, 1e-5 mixed) every walker of the
    2,100-walker set is within its path's target of the oracle: the ones the
    estimate flags are re-evaluated (mixed: by full LU, or by the FP64 table and
    then full LU for those still above the tolerance), the others are bounded by it."""
    wl, ref = o2100_fb
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    if mode is not None:
        ctx.set_escalation(mode)
    tol, cap = ctx.fallback
    assert tol == (1e-8 if prec == pkg.PRECISION_FP64 else 1e-5)
    got = _eval(ctx, wl.R)
    fb = (got["status"] & pkg.WS_FALLBACK) != 0
    esc = (got["status"] & pkg.WS_ESCALATED) != 0
    assert 0 < fb.sum() <= cap
    if mode == ESC:  # escalation resolves some walkers before the full-LU path
        assert esc.sum() > fb.sum() and not (fb & ~esc).any()
    else:
        assert not esc.any()
    err = _walker_errors(got, ref)
    assert err[~fb].max() <= tol, (int(np.flatnonzero(~fb)[np.argmax(err[~fb])]), err[~fb].max())
    # the re-evaluated walkers: the FP64 LU result, at the FP64 tolerances of the parity tests
    idx = np.flatnonzero(fb)
    rep = compare({k: v[idx] for k, v in got.items()}, {k: np.asarray(v)[idx] for k, v in ref.items()},
                  tol_psi=1e-10, tol_der=1e-8)
    assert rep["ok"], rep
    ctx.close()


def test_escalated_walkers_carry_fp64_table_results(o2100_fb):
    """Mixed walkers re-evaluated by the FP64 ratio table (and not by full LU)
    agree with an FP64 context's table result for the same walkers within the
    two FP64 estimates; without flagged walkers nothing is escalated."""
    wl, ref = o2100_fb
    mixed = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    mixed.set_escalation(ESC)
    got = _eval(mixed, wl.R)
    only = ((got["status"] & pkg.WS_ESCALATED) != 0) & ((got["status"] & pkg.WS_FALLBACK) == 0)
    assert only.any()
    fp64 = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    fp64.set_fallback(1e30, 1)  # table results with their estimates, nothing re-evaluated
    want = _eval(fp64, wl.R)
    _, est = fp64.error_estimates(wl.n_walk)
    d = _walker_errors({k: v[only] for k, v in got.items()}, {k: v[only] for k, v in want.items()})
    assert np.all(d <= 2 * est[only, 0] + 1e-13), (d.max(), est[only, 0])
    mixed.set_fallback(1e30, 256)  # estimates only: no walker exceeds the tolerance
    got2 = _eval(mixed, wl.R)
    assert not (got2["status"] & (pkg.WS_ESCALATED | pkg.WS_FALLBACK)).any()
    mixed.close()
    fp64.close()


def test_escalation_mode_is_validated():
    wl = synth.oxygen_like_1k(n_walk=8)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    with pytest.raises(pkg.MdetError):
        ctx.set_escalation(3)
    ctx.set_escalation(pkg.Context.ESCALATE_AUTO)
    ctx.close()

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


@pytest.mark.parametrize("prec", [pkg.PRECISION_FP64, pkg.PRECISION_MIXED])
def test_forced_fallback_for_every_walker_matches_oracle(prec):
    """With a tiny tolerance every walker goes through the full-LU path; at most
    `cap` of them are re-evaluated, the rest keep the table result and are flagged."""
    wl = synth.oxygen_like_1k(n_walk=40, seed=31)
    ref = oracle.evaluate(wl)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    ctx.set_fallback(1e-30, max_walkers=32)
    got = _eval(ctx, wl.R)
    fb = (got["status"] & pkg.WS_FALLBACK) != 0
    assert fb.sum() == 32
    assert np.all(got["status"][~fb] & pkg.WS_REF_ILLCOND)
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

"""Batched evaluation of uneven independent expansions (one device): direct
batch launches, the CUDA-graph batch, the autotuner and every tile shape,
each checked against the FP64 oracle on sampled walkers."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = dict(tol_psi=1e-9, tol_der=1e-6)


@pytest.fixture(scope="module")
def small_batch():
    wls = synth.batched_uneven(n_exp=6, walkers=(40, 300), n_det_range=(300, 20000), elec_range=(4, 20),
                               ao_range=(20, 60), seed=555)
    refs = []
    for wl in wls:
        idx = np.arange(min(6, wl.n_walk))
        refs.append((idx, oracle.evaluate(wl, R=wl.R[idx])))
    return wls, refs


def _to_host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("prec", [pkg.PRECISION_FP64, pkg.PRECISION_MIXED])
def test_batch_evaluate_matches_oracle(small_batch, prec):
    wls, refs = small_batch
    ctxs = [pkg.Context.from_workload(wl, device=0, precision=prec) for wl in wls]
    Rs = [torch.from_numpy(wl.R).to("cuda:0") for wl in wls]
    outs = pkg.batch_evaluate(ctxs, Rs, n_streams=3)
    torch.cuda.synchronize()
    for wl, (idx, ref), out in zip(wls, refs, outs):
        got = {k: v[idx] for k, v in _to_host(out).items()}
        rep = compare(got, ref, **TOL)
        assert rep["ok"], (wl.name, rep)


def test_graph_batch_replays_match_oracle(small_batch):
    """Two replays of the captured graph, the second with refilled walker
    buffers, checked against the oracle on sampled walkers and against
    evaluating each context on its own (same computation up to the order of
    the atomic sums)."""
    wls, refs = small_batch
    ctxs = [pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED) for wl in wls]
    Rs = [torch.from_numpy(wl.R).to("cuda:0") for wl in wls]
    batch = pkg.Batch(ctxs, Rs, n_streams=4)
    rng = np.random.default_rng(3)
    for rep_i in range(2):
        if rep_i:
            new_R = [synth.make_walkers(rng, wl.n_walk, wl.n_elec) for wl in wls]
            for R, nr in zip(Rs, new_R):
                R.copy_(torch.from_numpy(nr))
            refs = [(idx, oracle.evaluate(wl, R=nr[idx])) for wl, nr, (idx, _) in zip(wls, new_R, refs)]
        outs = batch.launch()
        torch.cuda.synchronize()
        for wl, c, R, out, (idx, ref) in zip(wls, ctxs, Rs, outs, refs):
            got = _to_host(out)
            rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL)
            assert rep["ok"], (rep_i, wl.name, rep)
            single = _to_host(c.evaluate(R.clone()))
            torch.cuda.synchronize()
            np.testing.assert_allclose(got["log_abs_psi"], single["log_abs_psi"], rtol=0, atol=1e-7)
            np.testing.assert_array_equal(got["sign"], single["sign"])
    batch.close()


def test_autotune_picks_valid_shapes_and_stays_correct(small_batch):
    wls, refs = small_batch
    wl, (idx, ref) = wls[0], refs[0]
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    R = torch.from_numpy(wl.R).to("cuda:0")
    t = ctx.autotune(R, budget_ms=100.0)
    assert t["spmm_chunk"] in (256, 512, 1024, 2048)
    assert t["mo_ec"] in (4, 6, 8)
    assert t["walker_chunks"] in (1, 2, 3, 4)
    assert t["trials"] >= 1 and t["best_ms"] > 0
    got = {k: v[idx] for k, v in _to_host(ctx.evaluate(R)).items()}
    torch.cuda.synchronize()
    rep = compare(got, ref, **TOL)
    assert rep["ok"], rep


@pytest.mark.parametrize("chunk,ec", [(64, 4), (256, 8), (2048, 6), (8192, 4)])
def test_every_tile_shape_is_correct(small_batch, chunk, ec):
    wls, refs = small_batch
    wl, (idx, ref) = wls[1], refs[1]
    for prec in (pkg.PRECISION_FP64, pkg.PRECISION_MIXED):
        ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
        ctx.set_tuning(spmm_chunk=chunk, mo_ec=ec, walker_chunks=2)
        got = {k: v[idx] for k, v in _to_host(ctx.evaluate(torch.from_numpy(wl.R).to("cuda:0"))).items()}
        rep = compare(got, ref, **(TOL if prec == pkg.PRECISION_MIXED else dict(tol_psi=1e-10, tol_der=1e-8)))
        assert rep["ok"], (chunk, ec, prec, rep)


@pytest.mark.slow
def test_full_uneven_64_graph_batch_sampled():
    """The 64-expansion uneven workload (8-34 electrons, 40-160 AOs, 10^3-10^6
    determinants, 256-4,096 walkers each) as one graph launch; two sampled
    walkers per expansion checked against the oracle."""
    wls = synth.batched_uneven()
    ctxs = [pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED) for wl in wls]
    Rs = [torch.from_numpy(wl.R).to("cuda:0") for wl in wls]
    batch = pkg.Batch(ctxs, Rs, n_streams=8)
    outs = batch.launch()
    torch.cuda.synchronize()
    for wl, out in zip(wls, outs):
        got = _to_host(out)
        assert np.all(np.isfinite(got["log_abs_psi"][(got["status"] & pkg.WS_REF_SINGULAR) == 0]))
        idx = np.array([0, wl.n_walk - 1])
        ref = oracle.evaluate(wl, R=wl.R[idx])
        rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL)
        assert rep["ok"], (wl.name, rep)
    batch.close()

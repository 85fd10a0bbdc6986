"""The allocation-free entry point mdet_psi_tilde_noalloc, checked through the C
ABI against mdet_evaluate on two calls in a row.

It serves callers that cannot allocate device memory at call time (a pooled
or custom allocator owning the GPU's memory, or a runtime that forbids
allocation after start-up): the intermediate v = C r_dn lives in the
library's static device scratch. This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _walker_minor(r_up, r_dn, ld, dev):
    """[n_walk][n] host ratios of both spins -> [n_up + n_dn][ld] device, walker-minor."""
    n_walk = r_up.shape[0]
    r = np.zeros((r_up.shape[1] + r_dn.shape[1], ld))
    r[:, :n_walk] = np.concatenate([r_up, r_dn], axis=1).T
    return torch.from_numpy(r).to(dev)


def test_noalloc_psi_tilde_matches_evaluate_twice():
    wl = synth.chlorine_like_100k(n_walk=300)
    dev = torch.device("cuda", 0)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    rng = np.random.default_rng(17)
    batches = [wl.R, synth.make_walkers(rng, 200, wl.n_elec)]   # two calls of different sizes
    for R in batches:
        n = R.shape[0]
        out = ctx.evaluate(torch.from_numpy(np.ascontiguousarray(R)).to(dev))
        torch.cuda.synchronize()
        log_ref = out["log_abs_psi"].cpu().numpy()
        sign_ref = out["sign"].cpu().numpy().astype(int)
        r_up, r_dn, log_d0, sign_d0 = ctx.ratios(n)
        ld = (n + 127) // 128 * 128
        r = _walker_minor(r_up, r_dn, ld, dev)
        psi_t = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        ctx.psi_tilde_noalloc(r, ld, psi_t)
        torch.cuda.synchronize()
        pt = psi_t.cpu().numpy()
        log_na = np.log(np.abs(pt)) + log_d0.sum(axis=1)
        sign_na = np.sign(pt).astype(int) * sign_d0[:, 0] * sign_d0[:, 1]
        assert np.all(sign_na == sign_ref)
        # same tolerance as the FP64 parity tests: 1e-10 relative on Psi
        assert np.max(np.abs(log_na - log_ref)) < 1e-10


def test_noalloc_rejects_sizes_beyond_scratch():
    wl = synth.chlorine_like_100k(n_walk=1)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    n_up = ctx.stats()["n_det_up"]
    ld = (pkg.Context.NOALLOC_SCRATCH_DOUBLES // (n_up + 1) // 128 + 1) * 128   # one tile too many
    dev = torch.device("cuda", 0)
    r = torch.zeros((n_up + ctx.stats()["n_det_dn"], ld), dtype=torch.float64, device=dev)
    psi_t = torch.zeros(ld, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.MdetError, match="static scratch") as ei:
        ctx.psi_tilde_noalloc(r, ld, psi_t)
    assert ei.value.status == 1   # MDET_E_ARG, rejected before any GPU work

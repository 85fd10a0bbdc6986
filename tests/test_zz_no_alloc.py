"""The allocation-free entry point mdet_psi_tilde_noalloc, checked through the C
ABI against mdet_evaluate on two calls in a row.

It serves callers that cannot allocate device memory at call time (a pooled
or custom allocator owning the GPU's memory, or a runtime that forbids
allocation after start-up): the intermediate v = C r_dn lives in the
library's static device scratch. This file is collected last on purpose.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRECISIONS = [pytest.param(pkg.PRECISION_FP64, id="fp64"), pytest.param(pkg.PRECISION_MIXED, id="mixed")]


def _walker_minor(r_up, r_dn, ld, dev, pad_value=0.0):
    """[n_walk][n] host ratios of both spins -> [n_up + n_dn][ld] device, walker-minor;
    the columns beyond n_walk hold pad_value."""
    n_walk = r_up.shape[0]
    r = np.full((r_up.shape[1] + r_dn.shape[1], ld), pad_value)
    r[:, :n_walk] = np.concatenate([r_up, r_dn], axis=1).T
    return torch.from_numpy(r).to(dev)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_noalloc_psi_tilde_matches_evaluate_twice(prec):
    """Two calls in a row of different sizes, the second on a non-default stream
    with a leading dimension one 128-walker tile wider than needed and NaN in the
    padding columns (which the call must not read into any walker's result).
    mdet_evaluate's ratios go in; its log|Psi| and sign must come back, to the
    1e-10 relative tolerance of the FP64 parity tests. On the mixed path the
    walkers that the stability fallback re-evaluated in FP64 are left out: their
    final Psi no longer comes from these ratios."""
    wl = synth.chlorine_like_100k(n_walk=300)
    dev = torch.device("cuda", 0)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    rng = np.random.default_rng(17)
    side = torch.cuda.Stream(dev)
    cases = [(wl.R, 0, None, 0.0), (synth.make_walkers(rng, 200, wl.n_elec), 128, side, float("nan"))]
    for R, extra, stream, pad in cases:
        n = R.shape[0]
        out = ctx.evaluate(torch.from_numpy(np.ascontiguousarray(R)).to(dev))
        torch.cuda.synchronize()
        log_ref = out["log_abs_psi"].cpu().numpy()
        sign_ref = out["sign"].cpu().numpy().astype(int)
        status = out["status"].cpu().numpy()
        r_up, r_dn, log_d0, sign_d0 = ctx.ratios(n)
        ld = (n + 127) // 128 * 128 + extra
        r = _walker_minor(r_up, r_dn, ld, dev, pad)
        psi_t = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        ctx.psi_tilde_noalloc(r, ld, psi_t, stream=stream)
        torch.cuda.synchronize()
        pt = psi_t.cpu().numpy()
        assert np.all(np.isfinite(pt))
        keep = (status & (pkg.WS_FALLBACK | pkg.WS_ESCALATED)) == 0
        assert keep.sum() > 0.9 * n
        log_na = np.log(np.abs(pt)) + log_d0.sum(axis=1)
        sign_na = np.sign(pt).astype(int) * sign_d0[:, 0] * sign_d0[:, 1]
        assert np.all(sign_na[keep] == sign_ref[keep])
        assert np.max(np.abs(log_na - log_ref)[keep]) < 1e-10
    ctx.close()


def test_noalloc_rejects_sizes_beyond_scratch():
    """One 128-walker tile more than the static scratch holds, through the
    binding; then, directly through the C ABI (the binding checks r's shape
    first), a leading dimension so large that (n_det_up + 1) * ld would overflow
    a 64-bit integer. Both come back as MDET_E_ARG before any GPU work, and the
    caller's current device is the same afterwards."""
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
    huge = (2 ** 62 // 128) * 128
    L = pkg.load_library()
    st = L.mdet_psi_tilde_noalloc(ctx._h, 1, C.c_void_p(r.data_ptr()), huge, C.c_void_p(psi_t.data_ptr()), None)
    assert st == 1
    assert torch.cuda.current_device() == 0
    ctx.close()

"""The paper's sequential Sherman-Morrison chain (Sec. 2.2, mdet_sm_chain)
against the oracle's full-LU determinant ratios and against the table method,
with the inversion and substitution counts of Table 3."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _chain_vs_oracle(wl, walkers):
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    R = torch.from_numpy(wl.R).to("cuda:0")
    out = ctx.alloc_outputs(R.shape[0])
    ctx.evaluate(R, out=out)
    r, n_inv, n_subst = ctx.sm_chain(R.shape[0])
    torch.cuda.synchronize()
    r = r.cpu().numpy()
    st = ctx.stats()
    r_tab_up, r_tab_dn, _, _ = ctx.ratios(R.shape[0])
    errs, errs_tab = [], []
    for spin, r_tab in ((0, r_tab_up), (1, r_tab_dn)):
        dets, _, _ = ctx.spin_dets(spin)
        off = 0 if spin == 0 else st["n_det_up"]
        chain = r[off:off + len(dets), :R.shape[0]].T  # [walker][det]
        lg, sg, _ = oracle.spin_dets(wl, spin, dets, R=wl.R[walkers])
        want = sg * sg[:, :1] * np.exp(lg - lg[:, :1])
        scale = np.maximum(np.abs(want), 1.0)
        errs.append((np.abs(chain[walkers] - want) / scale).ravel())
        errs_tab.append((np.abs(chain[walkers] - r_tab[walkers]) / scale).ravel())
    ctx.close()
    return np.concatenate(errs), np.concatenate(errs_tab), n_inv.cpu().numpy(), n_subst.cpu().numpy()


def test_sm_chain_oxygen_like_1k():
    wl = synth.oxygen_like_1k()
    err, err_tab, n_inv, n_subst = _chain_vs_oracle(wl, np.arange(wl.n_walk))
    assert np.percentile(err, 99) <= 1e-9 and err.max() <= 1e-7, (np.percentile(err, 99), err.max())
    assert err_tab.max() <= 1e-7
    assert (n_inv >= 2).all() and (n_subst > 0).all()


def test_sm_chain_chlorine_like_100k(capsys):
    """Sampled walkers of the 10^5-product expansion (two-word determinants,
    degrees up to 4); reports the Table 3 analogue."""
    wl = synth.chlorine_like_100k(n_walk=512)
    walkers = np.arange(0, 512, 64)
    err, err_tab, n_inv, n_subst = _chain_vs_oracle(wl, walkers)
    with capsys.disabled():
        print("\nSM chain, chlorine-like 1e5 (%d + %d distinct dets): N_inv %.2f, N_subst %.0f per walker-step; "
              "error vs oracle p50 %.1e p99 %.1e max %.1e" % (
                  *[len(np.unique(d, axis=0)) for d in (wl.det_up, wl.det_dn)], n_inv.mean(), n_subst.mean(),
                  np.median(err), np.percentile(err, 99), err.max()))
    assert np.percentile(err, 99) <= 1e-7, np.percentile(err, 99)
    assert (n_inv >= 2).all()


def test_sm_chain_arguments():
    wl = synth.oxygen_like_1k()
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    with pytest.raises(pkg.MdetError):
        ctx.sm_chain(8)  # no evaluation yet
    R = torch.from_numpy(wl.R[:16]).to("cuda:0")
    ctx.evaluate(R, out=ctx.alloc_outputs(16))
    with pytest.raises(pkg.MdetError):
        ctx.sm_chain(32)  # more walkers than were evaluated
    r, n_inv, _ = ctx.sm_chain(16)
    torch.cuda.synchronize()
    assert (n_inv.cpu().numpy() >= 2).all()
    ctx.close()

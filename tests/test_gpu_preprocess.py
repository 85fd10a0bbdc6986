"""Expansion preprocessing on the GPU (mdet_set_ci_expansion_device) against
the host path: identical distinct determinants, excitation records, C in the
paper's column-major order and identical evaluations, including multi-word
determinants, shuffled product order and invalid inputs (which must come back
as errors from the device checks)."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pair(wl, prec=pkg.PRECISION_FP64):
    host = pkg.Context.from_workload(wl, device=0, precision=prec)
    dev = pkg.Context.from_workload(wl, device=0, precision=prec, on_device=True)
    return host, dev


def _same_state(a, b):
    sa, sb = a.stats(), b.stats()
    assert sa == sb
    for sp in (0, 1):
        for x, y in zip(a.spin_dets(sp), b.spin_dets(sp)):
            assert np.array_equal(x, y)
    for x, y in zip(a.ci_matrix(), b.ci_matrix()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("name", ["oxygen_like_1k", "chlorine_like_100k"])
def test_device_preprocessing_matches_host(name):
    wl = synth.WORKLOADS[name]()
    assert name != "chlorine_like_100k" or wl.det_up.shape[1] == 2  # two 64-bit words per determinant
    host, dev = _pair(wl)
    _same_state(host, dev)
    R = torch.from_numpy(wl.R[:257]).to("cuda:0")
    oa, ob = host.alloc_outputs(R.shape[0]), dev.alloc_outputs(R.shape[0])
    host.evaluate(R, out=oa)
    dev.evaluate(R, out=ob)
    torch.cuda.synchronize()
    # the problems are identical (checked above); evaluations differ only by the order of FP64
    # atomic additions, which two runs of one context share
    for k in ("log_abs_psi", "grad", "lap", "e_local"):
        np.testing.assert_allclose(ob[k].cpu().numpy(), oa[k].cpu().numpy(), rtol=1e-9, atol=1e-9)
    assert torch.equal(oa["sign"], ob["sign"])
    host.close()
    dev.close()


def test_device_preprocessing_shuffled_and_uneven():
    """Products in random order, the reference not first, single-word and wide
    expansions from the uneven generator."""
    wls = synth.batched_uneven(n_exp=4, walkers=(32, 64), n_det_range=(2000, 60000), elec_range=(6, 30),
                               ao_range=(40, 160), seed=99)
    for wl in wls:
        perm = np.random.default_rng(3).permutation(len(wl.ci_coef))
        wl = synth.subset_products(wl, np.ones(len(perm), bool))
        wl.det_up, wl.det_dn, wl.ci_coef = wl.det_up[perm], wl.det_dn[perm], wl.ci_coef[perm]
        host, dev = _pair(wl, pkg.PRECISION_MIXED)
        _same_state(host, dev)
        host.close()
        dev.close()


TOL = {pkg.PRECISION_FP64: dict(tol_psi=1e-10, tol_der=1e-8), pkg.PRECISION_MIXED: dict(tol_psi=1e-9, tol_der=1e-6)}


@pytest.mark.parametrize("prec", [pkg.PRECISION_FP64, pkg.PRECISION_MIXED])
@pytest.mark.parametrize("name", ["oxygen_like_1k", "chlorine_like_100k"])
def test_device_preprocessed_context_matches_oracle(name, prec):
    """A context whose expansion went through the device preprocessing, with the
    products in shuffled order (so the sort, the deduplication and the reference
    search do real work), against the oracle's evaluation of the same expansion:
    all walkers of the 1k workload, 32 sampled walkers of the 10^5 one (two
    64-bit words per determinant)."""
    wl = synth.WORKLOADS[name]()
    perm = np.random.default_rng(5).permutation(len(wl.ci_coef))
    wl.det_up, wl.det_dn, wl.ci_coef = wl.det_up[perm], wl.det_dn[perm], wl.ci_coef[perm]
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec, on_device=True)
    out = ctx.evaluate(torch.from_numpy(np.ascontiguousarray(wl.R)).to("cuda:0"))
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    idx = np.arange(wl.n_walk) if wl.n_walk <= 64 else np.random.default_rng(8).choice(wl.n_walk, 32, replace=False)
    ref = oracle.evaluate(wl, R=wl.R[idx])
    rep = compare({k: v[idx] for k, v in got.items()}, ref, **TOL[prec])
    assert rep["ok"], rep
    ctx.close()


def test_device_preprocessing_rejects_invalid_input():
    wl = synth.oxygen_like_1k()
    ctx = pkg.Context(0, pkg.PRECISION_FP64)
    ctx.set_system(wl.n_up, wl.n_dn, wl.Z, wl.nuc_xyz)
    ctx.set_orbitals(wl.shell_l, wl.shell_center, wl.shell_nprim, wl.alpha, wl.coef, wl.mo_coef)
    bad = wl.det_up.copy()
    bad[17, 0] ^= 1 << 19  # one electron more or less in product 17
    with pytest.raises(pkg.MdetError, match="product 17") as e:
        ctx.set_ci_expansion(bad, wl.det_dn, wl.ci_coef, on_device=True)
    assert e.value.status == 5  # MDET_E_INPUT
    dup_u = np.concatenate([wl.det_up, wl.det_up[4:5]])
    dup_d = np.concatenate([wl.det_dn, wl.det_dn[4:5]])
    with pytest.raises(pkg.MdetError, match="repeat the same"):
        ctx.set_ci_expansion(dup_u, dup_d, np.concatenate([wl.ci_coef, [0.1]]), on_device=True)
    cf = wl.ci_coef.copy()
    cf[3] = np.nan
    with pytest.raises(pkg.MdetError, match="not finite"):
        ctx.set_ci_expansion(wl.det_up, wl.det_dn, cf, on_device=True)
    # the context is still usable afterwards
    ctx.set_ci_expansion(wl.det_up, wl.det_dn, wl.ci_coef, on_device=True)
    assert ctx.stats()["n_det"] == len(wl.ci_coef)
    ctx.close()


def test_device_preprocessing_time_750k(capsys):
    """Host and device preprocessing of the 750k-product expansion (reported)."""
    wl = synth.chlorine_like_750k()
    times = {}
    for on_dev in (False, True, True):
        ctx = pkg.Context(0, pkg.PRECISION_MIXED)
        ctx.set_system(wl.n_up, wl.n_dn, wl.Z, wl.nuc_xyz)
        ctx.set_orbitals(wl.shell_l, wl.shell_center, wl.shell_nprim, wl.alpha, wl.coef, wl.mo_coef)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_ci_expansion(wl.det_up, wl.det_dn, wl.ci_coef, on_device=on_dev)
        torch.cuda.synchronize()
        times["device" if on_dev else "host"] = time.perf_counter() - t0  # the second device run is warm
        ctx.close()
    with capsys.disabled():
        print("\npreprocessing of 750,000 products: host %.3f s, device %.3f s" % (times["host"], times["device"]))
    assert times["device"] > 0

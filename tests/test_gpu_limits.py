"""The library's size limits against the oracle: 32 electrons per spin (the
largest Slater matrices, whole-warp pivoting in the reference LU and the
largest per-walker shared-memory epilogue) and 255 molecular orbitals (four
64-bit words per determinant, the widest AO->MO product), in both
precisions, on ragged walker counts."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {pkg.PRECISION_FP64: dict(tol_psi=1e-10, tol_der=1e-8), pkg.PRECISION_MIXED: dict(tol_psi=1e-9, tol_der=1e-6)}


def _limit_workloads():
    # 32 + 32 electrons in 48 MOs over 52 AOs (s/p/d), degrees up to 4, 40 walkers
    wa = synth.make_workload("max_spin", 151000790, 32, 32, 64, (10, 8, 3), (0.05, 50.0), 48, 1500, 4, 40)
    # 4 + 4 electrons in 255 MOs over 300 AOs (s/p/d/f), 3,000 products, 37 walkers
    wb = synth.make_workload("max_mo", 151000791, 4, 4, 8, (40, 30, 25, 2), (0.05, 500.0), 255, 3000, 4, 37)
    return [wa, wb]


@pytest.fixture(scope="module")
def limits():
    return [(wl, oracle.evaluate(wl)) for wl in _limit_workloads()]


@pytest.mark.parametrize("prec", [pkg.PRECISION_FP64, pkg.PRECISION_MIXED])
@pytest.mark.parametrize("which", [0, 1])
def test_size_limits_match_oracle(limits, prec, which):
    wl, ref = limits[which]
    assert (wl.n_up == 32) if which == 0 else (wl.n_mo == 255 and wl.det_up.shape[1] == 4)
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    out = ctx.evaluate(torch.from_numpy(wl.R).to("cuda:0"))
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    rep = compare(got, ref, **TOL[prec])
    assert rep["ok"], rep
    ctx.close()


def test_limits_are_enforced():
    """One electron or one MO beyond the limits is refused with MDET_E_ARG."""
    wl = synth.oxygen_like_1k()
    ctx = pkg.Context(0, pkg.PRECISION_FP64)
    with pytest.raises(pkg.MdetError) as e:
        ctx.set_system(33, 4, wl.Z, wl.nuc_xyz)
    assert e.value.status == 1
    ctx.close()


def test_measured_fp64_rate_is_plausible():
    """The FP64 FMA throughput probe behind the contraction's roofline: positive,
    repeatable within 10 %, and within a factor of 4 of GB300's nominal 1.25 TFLOP/s."""
    a, ms, mhz = pkg.measure_fp64_rate(0, fma_per_thread=1 << 16, reps=3)
    b, _, _ = pkg.measure_fp64_rate(0, fma_per_thread=1 << 16, reps=3)
    assert ms > 0 and 500 < mhz < 3000, (ms, mhz)
    assert 0.3 < a < 5.0, a
    assert abs(a - b) <= 0.1 * max(a, b), (a, b)

"""The tcgen05 BF16 GEMM behind the learned proposal's perceptron (mdet_gemm_bf16).

Small integers are exact in BF16, their products exact in FP32, and every sum here
stays below 2^24, so with integer operands the tensor cores must return the exact
integer product whatever the accumulation order: the comparison is bit for bit. With
random FP32 operands the reference is the FP64 product of the same operands rounded
to BF16, within FP32 accumulation: K * 2^-23 of sum |a b| per entry.
Shapes cover a ragged M over 128-row tiles, N from 16 to two 256-wide tiles, K over
64-wide chunks with a ragged tail, and the K range split over CTAs (atomic path).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1510_00730_gb300 as pkg
from oracle.mlp import bf16_round

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _int_operands(rng, M, N, K, lo=-8, hi=8):
    return rng.integers(lo, hi + 1, size=(M, K)), rng.integers(lo, hi + 1, size=(N, K))


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 80, 100), (77, 256, 256), (513, 300, 64), (5, 68, 51),
                                   (260, 200, 1000)])
def test_integer_products_are_exact(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a, b = _int_operands(rng, M, N, K)
    want = a @ b.T  # int64, |entries| <= 64 K < 2^24
    A = torch.tensor(a, dtype=torch.float32, device=DEV)
    B = torch.tensor(b, dtype=torch.float32, device=DEV)
    D = pkg.gemm_bf16(A, B)
    torch.cuda.synchronize()
    assert np.array_equal(D.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("k_split", [64, 256, 1000])
def test_split_k_accumulates_exactly(k_split):
    """accumulate=1 adds into D with the K range split over CTAs; integer sums stay exact."""
    rng = np.random.default_rng(11)
    M, N, K = 200, 96, 2100
    a, b = _int_operands(rng, M, N, K, -4, 4)
    d0 = rng.integers(-100, 101, size=(M, N))
    A = torch.tensor(a, dtype=torch.float32, device=DEV)
    B = torch.tensor(b, dtype=torch.float32, device=DEV)
    D = torch.tensor(d0, dtype=torch.float32, device=DEV)
    pkg.gemm_bf16(A, B, D, accumulate=True, k_split=k_split)
    torch.cuda.synchronize()
    assert np.array_equal(D.cpu().numpy().astype(np.int64), d0 + a @ b.T)


def test_strided_operands_and_output():
    """Leading dimensions larger than the rows: padding is never read or written."""
    rng = np.random.default_rng(12)
    M, N, K = 130, 40, 70
    a, b = _int_operands(rng, M, N, K)
    A = torch.full((M, K + 9), float("nan"), dtype=torch.float32, device=DEV)
    B = torch.full((N, K + 3), float("nan"), dtype=torch.float32, device=DEV)
    A[:, :K] = torch.tensor(a, dtype=torch.float32, device=DEV)
    B[:, :K] = torch.tensor(b, dtype=torch.float32, device=DEV)
    D = torch.full((M, N + 5), -7.0, dtype=torch.float32, device=DEV)
    pkg.gemm_bf16(A[:, :K], B[:, :K], D[:, :N])
    torch.cuda.synchronize()
    d = D.cpu().numpy()
    assert np.array_equal(d[:, :N].astype(np.int64), a @ b.T)
    assert np.all(d[:, N:] == -7.0)


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (300, 68, 51), (64, 200, 8192)])
def test_random_operands_within_fp32_accumulation(M, N, K):
    rng = np.random.default_rng(K)
    a = rng.normal(size=(M, K)).astype(np.float32)
    b = rng.normal(size=(N, K)).astype(np.float32)
    ab, bb = bf16_round(a), bf16_round(b)
    want = ab @ bb.T
    bound = K * 2.0 ** -23 * (np.abs(ab) @ np.abs(bb).T)
    A = torch.tensor(a, device=DEV)
    B = torch.tensor(b, device=DEV)
    D = pkg.gemm_bf16(A, B).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(D - want) <= bound), np.max(np.abs(D - want) / bound)
    # and the operands really were rounded to BF16: the unrounded product is much farther away
    exact = a.astype(np.float64) @ b.T.astype(np.float64)
    assert np.abs(D - exact).max() > 10.0 * np.abs(D - want).max()


def test_empty_sum_and_refusals():
    A = torch.zeros(4, 0, dtype=torch.float32, device=DEV)
    B = torch.zeros(3, 0, dtype=torch.float32, device=DEV)
    D = torch.full((4, 3), 5.0, dtype=torch.float32, device=DEV)
    pkg.gemm_bf16(A, B, D)  # K = 0 overwrites with zeros
    torch.cuda.synchronize()
    assert float(D.abs().max()) == 0.0
    L = pkg.load_library()
    x = torch.zeros(16, dtype=torch.float32, device=DEV)
    p = x.data_ptr()
    assert L.mdet_gemm_bf16(-1, 2, 2, p, 2, p, 2, p, 2, 0, 64, None) == 1  # negative size
    assert L.mdet_gemm_bf16(2, 2, 4, p, 3, p, 4, p, 2, 0, 64, None) == 1  # lda below K
    assert L.mdet_gemm_bf16(2, 2, 4, None, 4, p, 4, p, 2, 0, 64, None) == 1  # null operand
    assert L.mdet_gemm_bf16(0, 2, 4, None, 4, None, 4, None, 2, 0, 64, None) == 0  # nothing to do

"""Pins for oracle.gemm: brute force, closed forms and planted mistakes."""
import numpy as np
import pytest

import synthetic
from oracle import gemm as og


def _ops(M, N, K, seed=0):
    a, b = synthetic.operands_bf16(M, N, K, seed)
    return og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (8, 4, 16), (13, 11, 9)])
def test_library_matmul_matches_triple_loop(M, N, K):
    a, b = _ops(M, N, K)
    c_loop = og.gemm_f64_loops(a, b)
    c = og.gemm_f64(a, b)
    # BF16 products are exact in float64; sums of <= 16 terms of magnitude <= 1
    # differ at most by float64 rounding-order effects.
    assert np.max(np.abs(c - c_loop)) <= K * 2.0 ** -52


def test_identity_gives_b_exactly():
    K = 64
    a = np.eye(K)
    _, b = _ops(K, 24, K)
    assert np.array_equal(og.gemm_f64(a, b), b)
    ok, ratio = og.check(b.astype(np.float32), a, b)
    assert ok and ratio == 0.0


def test_all_ones_gives_k():
    for K in (1, 7, 128, 4096):
        a = np.ones((3, K))
        b = np.ones((K, 5))
        assert np.all(og.gemm_f64(a, b) == K)


def test_rank_one_outer_product_exact():
    M, N, K = 17, 19, 33
    a_full, b = _ops(M, N, K)
    a = np.zeros_like(a_full)
    a[:, 5] = a_full[:, 5]
    c = og.gemm_f64(a, b)
    assert np.array_equal(c, np.outer(a[:, 5], b[5, :]))
    # the float32 product of two BF16 numbers is exact, so a float32 C passes with ratio 0
    ok, ratio = og.check(c.astype(np.float32), a, b)
    assert ok and ratio == 0.0


def test_bound_value():
    assert og.bound(4096) == 4096 * 2.0 ** -24
    assert og.bound(128, bf16_out=True) == 128 * 2.0 ** -24 + 2.0 ** -8


def test_float32_accumulation_within_bound():
    M, N, K = 32, 48, 512
    a, b = _ops(M, N, K)
    # sequential float32 accumulation: a legal summation order
    c32 = np.zeros((M, N), dtype=np.float32)
    for k in range(K):
        c32 += (a[:, k:k + 1].astype(np.float32) * b[k:k + 1, :].astype(np.float32))
    ok, ratio = og.check(c32, a, b)
    assert ok and 0 < ratio <= og.bound(K)


@pytest.mark.parametrize("mistake", ["dropped_term", "sign", "transposed", "wrong_index"])
def test_planted_mistakes_fail(mistake):
    M, N, K = 24, 24, 40
    a, b = _ops(M, N, K)
    if mistake == "dropped_term":
        c = a[:, :-1] @ b[:-1, :]
    elif mistake == "sign":
        c = a @ b
        c[3, 4] = -c[3, 4]
    elif mistake == "transposed":
        c = (a @ b).T                       # C^T in place of C (M == N here)
    else:
        c = a @ np.roll(b, 1, axis=0)
    ok, _ = og.check(c.astype(np.float32), a, b)
    assert not ok


def test_sampled_rows_cols_match_full():
    M, N, K = 40, 36, 64
    a, b = _ops(M, N, K)
    rows = np.array([0, 7, 39])
    cols = np.array([1, 35])
    cr, sr, cc, sc = og.sampled_rows_cols(a, b, rows, cols)
    full = og.gemm_f64(a, b)
    assert np.array_equal(cr, full[rows, :]) and np.array_equal(cc, full[:, cols])
    assert np.array_equal(sr, og.abs_sum(a, b)[rows, :])


def test_zero_scale_requires_exactness():
    a = np.zeros((2, 3))
    b = np.ones((3, 2))
    ok, _ = og.check(np.array([[0.0, 0.0], [0.0, 1e-30]], dtype=np.float32), a, b)
    assert not ok

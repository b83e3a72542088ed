"""O-GEMM: the plain definition C = A B of the BF16 NN GEMM (Sec. 2.2: A is
M x K, B is K x N, C is M x N), evaluated in float64, and the acceptance test
for a float32 result.

Test infrastructure only (see the package docstring).

Acceptance: for a float32 result C of the product of BF16 operands,

    max_ij |C_ij - C64_ij| / S_ij <= K * 2**-24,   S_ij = sum_k |a_ik| |b_kj|,

with exact equality required where S_ij == 0.  The bound is the classical
a-priori bound for recursive summation with unit roundoff 2**-24 and holds for
any summation order, so it covers split-K (partial sums added in another
order) and zero padding (extra exact zeros).  A BF16 output adds 2**-8
relative to the bound.
"""
from __future__ import annotations

import numpy as np


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Decode bfloat16 bit patterns (uint16) to float64 (bfloat16 = top half of float32)."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def gemm_f64_loops(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Textbook triple loop, float64, for tiny shapes: C[i][j] = sum_k a[i][k] * b[k][j]."""
    M, K = a.shape
    K2, N = b.shape
    assert K == K2
    c = np.zeros((M, N), dtype=np.float64)
    for i in range(M):
        for j in range(N):
            s = 0.0
            for k in range(K):
                s += float(a[i, k]) * float(b[k, j])
            c[i, j] = s
    return c


def gemm_f64(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """C = A B with float64 inputs and float64 accumulation (library matmul as one step)."""
    return np.asarray(a, dtype=np.float64) @ np.asarray(b, dtype=np.float64)


def abs_sum(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """S_ij = sum_k |a_ik| |b_kj|, the scale of the error bound."""
    return np.abs(np.asarray(a, dtype=np.float64)) @ np.abs(np.asarray(b, dtype=np.float64))


def error_ratio(c: np.ndarray, c64: np.ndarray, s: np.ndarray) -> tuple[float, bool]:
    """(max_ij |c - c64| / S_ij over S_ij > 0, exact-where-S-is-zero flag)."""
    c = np.asarray(c, dtype=np.float64)
    err = np.abs(c - c64)
    pos = s > 0
    ratio = float(np.max(err[pos] / s[pos])) if np.any(pos) else 0.0
    exact_zero = bool(np.all(err[~pos] == 0.0))
    return ratio, exact_zero


def bound(K: int, bf16_out: bool = False) -> float:
    b = K * 2.0 ** -24
    if bf16_out:
        b += 2.0 ** -8
    return b


def check(c: np.ndarray, a: np.ndarray, b: np.ndarray, bf16_out: bool = False) -> tuple[bool, float]:
    """Accept c as the product of a and b (float64 views of the BF16 operands)."""
    c64 = gemm_f64(a, b)
    s = abs_sum(a, b)
    ratio, exact_zero = error_ratio(c, c64, s)
    K = a.shape[1]
    return (ratio <= bound(K, bf16_out) and exact_zero), ratio


def sampled_rows_cols(a: np.ndarray, b: np.ndarray, rows: np.ndarray, cols: np.ndarray):
    """float64 reference for whole rows ``rows`` and whole columns ``cols`` of C
    (for shapes too large to form C64 in full): returns (C64[rows, :], S[rows, :],
    C64[:, cols], S[:, cols])."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ar = a[rows, :]
    bc = b[:, cols]
    return ar @ b, np.abs(ar) @ np.abs(b), a @ bc, np.abs(a) @ np.abs(bc)

"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This module holds input generation only: no GEMM, no planning, no statistics.
Both the CPU oracle (in tests) and the CUDA path consume the arrays it returns,
so the two sides see bit-identical operands.

Counter-based stream (one per operand), element ``idx`` of operand ``tag``:

    key  = mix(seed * 4 + tag)                       tag: A = 1, B = 2
    r    = mix(key + (idx + 1) * 0x9E3779B97F4A7C15)  (mod 2**64)
    u    = (r >> 40) * 2**-24                         24-bit uniform in [0, 1)

``mix`` is the SplitMix64 output function (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014).

BF16 operands: x = 2u - 1 (exact in float32), rounded to bfloat16 with
round-to-nearest-even.  The workloads draw U[-1, 1) rounded to BF16; the
rounding can produce exactly +1.0, which is accepted.

FP8 workload inputs: N(0, 1) float32 by the Box-Muller transform, element i
from the draws 2i (u1) and 2i+1 (u2):
z = sqrt(-2 ln(1 - u1)) * cos(2 pi u2), evaluated in float64, then rounded to
float32.

GEMM operands for a shape (M, N, K) are the contiguous prefixes of the
streams: A = stream_A[:M*K] viewed as M x K row-major, B = stream_B[:K*N]
viewed as K x N row-major.  Every shape of a sweep therefore reads the same
two buffers.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
TAG_A = 1
TAG_B = 2


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, tag: int) -> np.uint64:
    return _mix(np.array([(seed * 4 + tag) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]


def uniform24(seed: int, tag: int, n: int, start: int = 0) -> np.ndarray:
    """u[idx] for idx in [start, start+n): float64 multiples of 2**-24 in [0, 1)."""
    key = stream_key(seed, tag)
    idx = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = key + (idx + np.uint64(1)) * GOLDEN_GAMMA
    r = _mix(ctr)
    return (r >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); returns uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def bf16_uniform_stream(seed: int, tag: int, n: int) -> np.ndarray:
    """First n elements of a U[-1, 1) BF16 operand stream, as uint16 bit patterns."""
    x = (2.0 * uniform24(seed, tag, n) - 1.0).astype(np.float32)   # exact
    return f32_to_bf16_bits(x)


def normal_stream_f32(seed: int, tag: int, n: int) -> np.ndarray:
    """First n elements of an N(0, 1) float32 operand stream (Box-Muller)."""
    u = uniform24(seed, tag, 2 * n)
    u1 = 1.0 - u[0::2]                      # in (0, 1]
    u2 = u[1::2]
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z[:n].astype(np.float32)


def operands_bf16(M: int, N: int, K: int, seed: int = 0):
    """(A bits M x K, B bits K x N) as uint16 arrays, prefixes of the seed's streams."""
    a = bf16_uniform_stream(seed, TAG_A, M * K).reshape(M, K)
    b = bf16_uniform_stream(seed, TAG_B, K * N).reshape(K, N)
    return a, b


def grid_values(start: int, step: int, count: int) -> list[int]:
    return [start + i * step for i in range(count)]


def poisson_arrivals(rate_per_s: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times in ns of a Poisson process (exponential gaps from the stream, tag 3)."""
    u = uniform24(seed, 3, n)
    gaps = -np.log(1.0 - u) / rate_per_s
    return np.round(np.cumsum(gaps) * 1e9).astype(np.int64)


def uniform_cells(n: int, counts=(32, 32, 32), seed: int = 0) -> np.ndarray:
    """n grid-cell indices (a, b, c), each drawn uniformly (stream tag 4)."""
    u = uniform24(seed, 4, 3 * n).reshape(n, 3)
    return np.floor(u * np.array(counts)).astype(np.int64)

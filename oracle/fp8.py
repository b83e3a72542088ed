"""FP8 e4m3 block-scaled GEMM reference (the precision variant of the GEMM
path; the paper itself measures BF16 only, Sec. 2.2, so these definitions come
from the formats, not from the paper).

Test infrastructure only (see the package docstring).

e4m3 ("E4M3FN"): 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits, no
infinities, S.1111.111 is NaN; the largest finite magnitude is 448 and the
smallest normal 2**-6, subnormals are multiples of 2**-9.

Block quantisation of a float32 matrix X with 128 x 128 blocks (ragged blocks
at the edges hold fewer elements):
  amax  = max |x| over the block (exact)
  s     = amax / 448 in float32 (IEEE division); s = 1 when amax == 0
  q     = e4m3(x / s): the float32 quotient (IEEE division) rounded to the
          nearest e4m3 value, ties to even, magnitudes above 448 saturated
          to 448 (satfinite)
The scales are stored as float32 arrays sA[M/128][K/128] and sB[K/128][N/128]
(ceil-divided).  The dequantised operand is float64(q) * float64(s).
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0
BLOCK = 128


def e4m3_round(v: np.ndarray) -> np.ndarray:
    """Nearest e4m3 value of float32 inputs (ties to even, satfinite), as float64."""
    v = np.asarray(v, dtype=np.float32).astype(np.float64)
    a = np.abs(v)
    out = np.zeros_like(a)
    nz = a > 0
    e = np.floor(np.log2(a[nz]))
    # exponent of the binade, clamped to the normal range's bottom for subnormals
    e = np.maximum(e, -6.0)
    # guard against log2 rounding at exact powers of two
    e = np.where(2.0 ** e > a[nz], e - 1, e)
    e = np.where(2.0 ** (e + 1) <= a[nz], e + 1, e)
    e = np.maximum(e, -6.0)
    quantum = 2.0 ** (e - 3)
    r = np.rint(a[nz] / quantum) * quantum       # rint = round half to even; exact
    out[nz] = np.minimum(r, E4M3_MAX)
    return np.copysign(out, v)


def e4m3_bits(r: np.ndarray) -> np.ndarray:
    """Encode values that are exactly representable in e4m3 to their byte."""
    r = np.asarray(r, dtype=np.float64)
    sign = (np.signbit(r)).astype(np.uint8) << 7
    a = np.abs(r)
    bits = np.zeros(a.shape, dtype=np.uint8)
    sub = (a > 0) & (a < 2.0 ** -6)
    bits[sub] = np.rint(a[sub] / 2.0 ** -9).astype(np.uint8)
    nor = a >= 2.0 ** -6
    e = np.floor(np.log2(a[nor]))
    e = np.where(2.0 ** e > a[nor], e - 1, e)
    man = np.rint((a[nor] / 2.0 ** e - 1.0) * 8.0)
    bits[nor] = ((e + 7).astype(np.uint8) << 3) | man.astype(np.uint8)
    return bits | sign


def e4m3_decode(bits: np.ndarray) -> np.ndarray:
    b = np.asarray(bits, dtype=np.uint8)
    s = np.where(b & 0x80, -1.0, 1.0)
    e = ((b >> 3) & 0xF).astype(np.int64)
    m = (b & 0x7).astype(np.float64)
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * 2.0 ** (e - 7).astype(np.float64))
    nan = (e == 15) & ((b & 0x7) == 7)
    val = np.where(nan, np.nan, val)
    return s * val


def quantize_blocks(x: np.ndarray, block: int = BLOCK):
    """Block-quantise a float32 matrix: returns (q bytes uint8, scales float32)."""
    x = np.asarray(x, dtype=np.float32)
    R, C = x.shape
    br, bc = -(-R // block), -(-C // block)
    scales = np.ones((br, bc), dtype=np.float32)
    q = np.zeros((R, C), dtype=np.uint8)
    for i in range(br):
        for j in range(bc):
            blk = x[i * block:(i + 1) * block, j * block:(j + 1) * block]
            amax = np.float32(np.max(np.abs(blk))) if blk.size else np.float32(0)
            s = np.float32(amax / np.float32(E4M3_MAX)) if amax > 0 else np.float32(1.0)
            quot = (blk / s).astype(np.float32)          # IEEE float32 division
            q[i * block:(i + 1) * block, j * block:(j + 1) * block] = e4m3_bits(e4m3_round(quot))
            scales[i, j] = s
    return q, scales


def dequantize(q: np.ndarray, scales: np.ndarray, block: int = BLOCK) -> np.ndarray:
    v = e4m3_decode(q)
    s = np.repeat(np.repeat(scales.astype(np.float64), block, axis=0), block, axis=1)
    return v * s[: v.shape[0], : v.shape[1]]


def gemm_blockscaled_f64(qa, sa, qb, sb, block: int = BLOCK) -> np.ndarray:
    """C = dequant(A) @ dequant(B) in float64: the exact product of the quantised operands."""
    return dequantize(qa, sa, block) @ dequantize(qb, sb, block)

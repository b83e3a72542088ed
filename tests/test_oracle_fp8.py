"""Pins for oracle.fp8: the e4m3 format, rounding, saturation and block scaling."""
import numpy as np
import pytest

import synthetic
from oracle import fp8


def test_decode_encode_roundtrip_all_bytes():
    b = np.arange(256, dtype=np.uint8)
    nan = ((b & 0x7F) == 0x7F)
    v = fp8.e4m3_decode(b)
    assert np.all(np.isnan(v[nan]))
    keep = ~nan & (b != 0x80)                     # -0 encodes as +0's magnitude with sign kept
    assert np.array_equal(fp8.e4m3_bits(v[keep]), b[keep])
    assert fp8.e4m3_decode(np.array([0x7E], dtype=np.uint8))[0] == 448.0
    assert fp8.e4m3_decode(np.array([0x01], dtype=np.uint8))[0] == 2.0 ** -9
    assert fp8.e4m3_decode(np.array([0x38], dtype=np.uint8))[0] == 1.0
    assert fp8.e4m3_decode(np.array([0x08], dtype=np.uint8))[0] == 2.0 ** -6


def test_round_ties_to_even_and_saturate():
    x = np.array([1.0625, 1.1875, 1.0624, 500.0, -1e9, 464.0, 2.0 ** -10, 3 * 2.0 ** -10, 0.0],
                 dtype=np.float32)
    r = fp8.e4m3_round(x)
    assert r.tolist() == [1.0, 1.25, 1.0, 448.0, -448.0, 448.0, 0.0, 2.0 ** -8, 0.0]


def test_round_is_nearest_on_every_representable_neighbourhood():
    vals = np.unique(np.abs(fp8.e4m3_decode(np.arange(0, 0x7F, dtype=np.uint8))))
    rng = np.random.default_rng(1)
    x = rng.uniform(-448, 448, 20000).astype(np.float32)
    r = fp8.e4m3_round(x)
    # brute force: nearest representable value, ties to the even mantissa
    for xi, ri in zip(x[:2000], r[:2000]):
        d = np.abs(vals - abs(float(xi)))
        best = vals[d == d.min()]
        if len(best) == 2:
            best = [v for v in best if fp8.e4m3_bits(np.array([v]))[0] % 2 == 0]
        assert abs(ri) == best[0]


def test_matches_torch_cast_in_range():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(0, 30, 50000), rng.uniform(-448, 448, 50000),
                        rng.normal(0, 1e-3, 20000)]).astype(np.float32)
    t = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(fp8.e4m3_bits(fp8.e4m3_round(x)), t)


def test_block_quantization_scales_and_amax():
    x = synthetic.normal_stream_f32(0, 1, 300 * 260).reshape(300, 260)
    q, s = fp8.quantize_blocks(x)
    assert s.shape == (3, 3) and q.shape == x.shape
    d = fp8.e4m3_decode(q)
    for i in range(3):
        for j in range(3):
            blk = d[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]
            assert np.max(np.abs(blk)) == 448.0                       # amax maps to the top code
            assert s[i, j] == np.float32(np.max(np.abs(x[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]))
                                         / np.float32(448.0))
    # quantisation error: half an e4m3 ulp relative (2**-4) of each value, times the scale
    rel = np.abs(fp8.dequantize(q, s) - x) / np.maximum(np.abs(x), 1e-30)
    big = np.abs(x) > np.repeat(np.repeat(s, 128, 0), 128, 1)[:300, :260] * 2.0 ** -6
    assert np.max(rel[big]) <= 2.0 ** -4 + 1e-7


def test_zero_block_scale_is_one():
    q, s = fp8.quantize_blocks(np.zeros((128, 256), dtype=np.float32))
    assert np.all(s == 1.0) and np.all(q == 0)


def test_blockscaled_gemm_exact_on_representable_inputs():
    # e4m3 values whose every 128 x 128 block holds +-448: scale 1, quantisation exact,
    # so the block-scaled product equals the plain float64 product of the inputs
    rng = np.random.default_rng(4)
    a = fp8.e4m3_decode(rng.integers(0, 0x7E, size=(256, 384)).astype(np.uint8))
    b = fp8.e4m3_decode(rng.integers(0, 0x7E, size=(384, 256)).astype(np.uint8))
    a[::128, ::128] = 448.0
    b[::128, ::128] = -448.0
    qa, sa = fp8.quantize_blocks(a.astype(np.float32))
    qb, sb = fp8.quantize_blocks(b.astype(np.float32))
    assert np.all(sa == 1.0) and np.all(sb == 1.0)
    assert np.array_equal(fp8.dequantize(qa, sa), a)
    assert np.array_equal(fp8.gemm_blockscaled_f64(qa, sa, qb, sb), a @ b)

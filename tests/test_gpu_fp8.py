"""GPU parity of the FP8 e4m3 path: the block quantiser (bit-exact against the
oracle, codes and scales) and the block-scaled GEMM (against the float64
product of the dequantised operands)."""
import numpy as np
import pytest

import synthetic
from oracle import fp8 as of
from oracle import gemm as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Observed FP8 GEMM error is reported per shape; the test bound is the FP32
# accumulation bound K * 2^-24 (the e4m3 products are exact in FP32) with a factor
# 4 for the per-block scale product and promotion, which the paper leaves open.
FP8_BOUND_FACTOR = 4.0


@pytest.fixture(scope="module")
def rg():
    from paper_2605_29752_gb300 import rg as _rg
    return _rg


@pytest.fixture(scope="module")
def ctx(rg):
    h = rg.rg_init(0)
    yield h
    rg.rg_destroy(h)


def quantize(rg, ctx, x):
    R, Cc = x.shape
    X = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Q = torch.zeros((R, Cc), dtype=torch.uint8, device="cuda")
    S = torch.zeros((-(-R // 128), -(-Cc // 128)), dtype=torch.float32, device="cuda")
    rg.rg_fp8_quantize(ctx, X, R, Cc, Cc, Q, Cc, S)
    rg.rg_check(ctx)
    return Q, S


@pytest.mark.parametrize("shape", [(300, 260), (128, 128), (1024, 1536), (1, 16)])
def test_quantizer_bit_exact(rg, ctx, shape):
    x = synthetic.normal_stream_f32(0, 1, shape[0] * shape[1]).reshape(shape)
    x[0, 0] = 0.0
    Q, S = quantize(rg, ctx, x)
    q_ref, s_ref = of.quantize_blocks(x)
    assert np.array_equal(S.cpu().numpy(), s_ref)
    assert np.array_equal(Q.cpu().numpy(), q_ref)


def test_quantizer_zero_block_and_saturation(rg, ctx):
    x = np.zeros((256, 128), np.float32)
    x[128:, :] = np.linspace(-3e4, 3e4, 128 * 128, dtype=np.float32).reshape(128, 128)
    Q, S = quantize(rg, ctx, x)
    q_ref, s_ref = of.quantize_blocks(x)
    assert S.cpu().numpy()[0, 0] == 1.0
    assert np.array_equal(Q.cpu().numpy(), q_ref) and np.array_equal(S.cpu().numpy(), s_ref)


def _gemm(rg, ctx, M, N, K, seed=0):
    a = synthetic.normal_stream_f32(seed, 1, M * K).reshape(M, K)
    b = synthetic.normal_stream_f32(seed, 2, K * N).reshape(K, N)
    qa, sa = quantize(rg, ctx, a)
    qb, sb = quantize(rg, ctx, b)
    C = torch.full((M, N), float("nan"), device="cuda")
    rg.rg_gemm_fp8(ctx, M, N, K, qa, K, sa, qb, N, sb, C, N)
    rg.rg_check(ctx)
    return C.cpu().numpy(), (qa.cpu().numpy(), sa.cpu().numpy(), qb.cpu().numpy(), sb.cpu().numpy())


@pytest.mark.parametrize("shape", [(128, 128, 128), (512, 512, 512), (300, 272, 400), (1024, 512, 2048),
                                   (512, 1536, 1024)])
def test_gemm_fp8_against_dequantized_f64(rg, ctx, shape):
    M, N, K = shape
    c, (qa, sa, qb, sb) = _gemm(rg, ctx, M, N, K)
    A = of.dequantize(qa, sa)
    B = of.dequantize(qb, sb)
    c64 = A @ B
    s = np.abs(A) @ np.abs(B)
    ratio, exact_zero = og.error_ratio(c, c64, s)
    print(f"fp8 {shape}: max |C - C64| / sum|a||b| = {ratio:.3e} (K * 2^-24 = {K * 2.0 ** -24:.3e})")
    assert not np.any(np.isnan(c)) and exact_zero
    assert ratio <= FP8_BOUND_FACTOR * K * 2.0 ** -24


def test_gemm_fp8_exact_on_representable_inputs(rg, ctx):
    # e4m3 values in {0, +-0.5, +-1, +-2} and +-448 in every block: scales are 1, products and
    # their sums are exact in FP32, so C must equal the exact product bit for bit
    M, N, K = 256, 384, 512
    rng = np.random.default_rng(3)
    vals = np.array([0.0, 0.5, -0.5, 1.0, -1.0, 2.0, -2.0], np.float32)
    a = vals[rng.integers(0, 7, size=(M, K))]
    b = vals[rng.integers(0, 7, size=(K, N))]
    a[::128, ::128] = 448.0
    b[::128, ::128] = 448.0
    qa, sa = quantize(rg, ctx, a)
    qb, sb = quantize(rg, ctx, b)
    assert torch.all(sa == 1.0) and torch.all(sb == 1.0)
    C = torch.full((M, N), float("nan"), device="cuda")
    rg.rg_gemm_fp8(ctx, M, N, K, qa, K, sa, qb, N, sb, C, N)
    rg.rg_check(ctx)
    exact = a.astype(np.float64) @ b.astype(np.float64)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), exact)


def test_gemm_fp8_full_size_sampled(rg, ctx):
    M = N = K = 4096
    c, (qa, sa, qb, sb) = _gemm(rg, ctx, M, N, K, seed=1)
    A = of.dequantize(qa, sa)
    B = of.dequantize(qb, sb)
    rs = np.random.default_rng(0)
    rows = rs.choice(M, 8, replace=False)
    cols = rs.choice(N, 8, replace=False)
    cr, sr, cc, sc = og.sampled_rows_cols(A, B, rows, cols)
    for got, ref, s in ((c[rows, :], cr, sr), (c[:, cols], cc, sc)):
        ratio, exact_zero = og.error_ratio(got, ref, s)
        assert exact_zero and ratio <= FP8_BOUND_FACTOR * K * 2.0 ** -24, ratio


def test_gemm_fp8_alignment_errors(rg, ctx):
    q = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    s = torch.ones((1, 1), device="cuda")
    C = torch.zeros((64, 64), device="cuda")
    with pytest.raises(rg.RGError) as e:
        rg.rg_gemm_fp8(ctx, 64, 64, 40, q, 40, s, q, 64, s, C, 64)
    assert e.value.code == rg.RG_ERR_ALIGN


def test_fp8_sweep_small_grid(rg, ctx):
    """rg_sweep_fp8 times every cell of a grid (here {256, 512}^3) and the surface statistics accept it."""
    Mx = 512
    x = synthetic.normal_stream_f32(0, 1, Mx * Mx).reshape(Mx, Mx)
    qa, sa = quantize(rg, ctx, x)
    qb, sb = quantize(rg, ctx, x)
    C = torch.zeros(Mx * Mx, device="cuda")
    g = rg.make_grid((256, 256, 2))
    opts = rg.rg_sweep_opts_default()
    opts.reps = 2
    t = rg.rg_sweep_fp8(ctx, g, qa, sa, qb, sb, C, opts)
    assert t.shape == (8,) and np.all(t > 0) and np.all(t < 10 ** 8)
    tf, r, mean = rg.rg_surface_stats(g, t)
    assert mean > 0 and np.all(tf > 0)

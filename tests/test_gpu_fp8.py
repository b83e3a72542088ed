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
    assert t.shape == (8,) and np.all(t > 0) and np.all(t < 10 ** 8)       # the default 128x256 variant
    tf, r, mean = rg.rg_surface_stats(g, t)
    assert mean > 0 and np.all(tf > 0)


def _check_fp8(c, qa, sa, qb, sb, K, c0=None):
    A = of.dequantize(qa, sa)
    B = of.dequantize(qb, sb)
    c64 = A @ B
    s = np.abs(A) @ np.abs(B)
    if c0 is not None:
        c64 = c64 + c0.astype(np.float64)
        s = s + np.abs(c0.astype(np.float64))
    ratio, exact_zero = og.error_ratio(c, c64, s)
    assert not np.any(np.isnan(c)) and exact_zero
    assert ratio <= FP8_BOUND_FACTOR * (K + (1 if c0 is not None else 0)) * 2.0 ** -24, ratio
    return ratio


def _operands(rg, ctx, M, N, K, seed):
    a = synthetic.normal_stream_f32(seed, 1, M * K).reshape(M, K)
    b = synthetic.normal_stream_f32(seed, 2, K * N).reshape(K, N)
    qa, sa = quantize(rg, ctx, a)
    qb, sb = quantize(rg, ctx, b)
    return qa, sa, qb, sb


def _run_ex(rg, ctx, M, N, K, ops, v, beta=0, c0=None, pads=(0, 0, 0)):
    qa, sa, qb, sb = ops
    C = torch.from_numpy(c0.copy()).cuda() if c0 is not None else torch.full((M, N), float("nan"), device="cuda")
    rg.rg_gemm_fp8_ex(ctx, M, N, K, qa, K, sa, sa.shape[1], qb, N, sb, sb.shape[1], C, N, v, beta, *pads)
    rg.rg_check(ctx)
    return C.cpu().numpy()


FP8_VARIANTS = list(range(64, 76))          # 128x256, 128x128, 256x256 cta_group::2 pair; split-K 1/2/4/8


@pytest.mark.parametrize("v", FP8_VARIANTS)
def test_fp8_every_variant_ragged_and_deterministic(rg, ctx, v):
    M, N, K = 300, 272, 400                  # partial tiles in M, N and K for both tiles
    ops = _operands(rg, ctx, M, N, K, seed=5)
    c = _run_ex(rg, ctx, M, N, K, ops, v)
    _check_fp8(c, *(x.cpu().numpy() for x in ops), K)
    assert np.array_equal(c, _run_ex(rg, ctx, M, N, K, ops, v))
    if v == rg.fp8_variant(0, 1):            # rg_gemm_fp8 is this variant with compact scales
        C = torch.full((M, N), float("nan"), device="cuda")
        qa, sa, qb, sb = ops
        rg.rg_gemm_fp8(ctx, M, N, K, qa, K, sa, qb, N, sb, C, N)
        rg.rg_check(ctx)
        assert np.array_equal(C.cpu().numpy(), c)


@pytest.mark.parametrize("v", [64, 65, 67, 68, 70, 72, 73, 75])
def test_fp8_split_k_beta_and_padding(rg, ctx, v):
    M, N, K = 512, 384, 2048
    ops = _operands(rg, ctx, M, N, K, seed=6)
    host = [x.cpu().numpy() for x in ops]
    c = _run_ex(rg, ctx, M, N, K, ops, v)
    _check_fp8(c, *host, K)
    c0 = synthetic.normal_stream_f32(6, 5, M * N).reshape(M, N)
    _check_fp8(_run_ex(rg, ctx, M, N, K, ops, v, beta=1, c0=c0), *host, K, c0=c0)
    cp = _run_ex(rg, ctx, M, N, K, ops, v, pads=(M + 128, N + 256, K + 256))
    _check_fp8(cp, *host, K)
    if rg.SPLITS[(v - 64) % 4] == 1:      # zero K padding adds exact zero products: the same bits
        assert np.array_equal(cp, c)
    assert np.array_equal(c, _run_ex(rg, ctx, M, N, K, ops, v, pads=(M + 128, N + 256, K)))


@pytest.mark.parametrize("shape", [(1024, 768, 1024), (1000, 528, 640), (3968, 4096, 512)])
def test_fp8_pair_matches_one_cta_tile(rg, ctx, shape):
    """The 256x256 cta_group::2 pair computes each CTA's 128 rows x 256 columns with the same MMA
    shape per row (N = 256, K = 32 steps) and the same promotion order as the 1-CTA 128x256 tile,
    so their results agree bit for bit (ragged edges, and an odd CTA wholly past M)."""
    M, N, K = shape
    ops = _operands(rg, ctx, M, N, K, seed=9)
    c1 = _run_ex(rg, ctx, M, N, K, ops, rg.fp8_variant(0, 1))
    c2 = _run_ex(rg, ctx, M, N, K, ops, rg.fp8_variant(2, 1))
    assert not np.any(np.isnan(c2))
    assert np.array_equal(c1, c2)
    if M * N * K <= 1024 ** 3:
        _check_fp8(c2, *(x.cpu().numpy() for x in ops), K)


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("shape", [(2048, 1536, 1152), (1000, 528, 1664), (256, 256, 4096)])
def test_fp8_coupled_ring_128x128(rg, ctx, shape, split):
    """The 128x128 tile pairs its four operand stages with its four accumulator buffers (the producer
    refills a stage once the promotion warps released the buffer of the same index).  Shapes where CTAs run
    several tiles, K-block counts that are not a multiple of the ring (9, 13) and a 32-block K: within the
    FP8 bound of the float64 product of the dequantised operands, deterministic, and, at split 1, equal
    bit for bit to the 128x256 tile, whose per-element MMA steps and promotion order are the same."""
    M, N, K = shape
    ops = _operands(rg, ctx, M, N, K, seed=12)
    v = rg.fp8_variant(1, split)
    c = _run_ex(rg, ctx, M, N, K, ops, v)
    assert not np.any(np.isnan(c))
    assert np.array_equal(c, _run_ex(rg, ctx, M, N, K, ops, v))
    if split == 1:
        assert np.array_equal(c, _run_ex(rg, ctx, M, N, K, ops, rg.fp8_variant(0, 1)))
    host = [x.cpu().numpy() for x in ops]
    if M * N * K <= 1024 ** 3:
        _check_fp8(c, *host, K)
    else:
        rs = np.random.default_rng(5)
        rows, cols = rs.choice(M, 16, replace=False), rs.choice(N, 16, replace=False)
        A, B = of.dequantize(host[0], host[1]), of.dequantize(host[2], host[3])
        for got, a, b in ((c[rows, :], A[rows, :], B), (c[:, cols], A, B[:, cols])):
            ratio, exact_zero = og.error_ratio(got, a @ b, np.abs(a) @ np.abs(b))
            assert exact_zero and ratio <= FP8_BOUND_FACTOR * K * 2.0 ** -24, ratio


def test_fp8_scale_sub_views(rg, ctx):
    """A sub-problem of a quantised matrix (offsets multiples of 128) through its scale sub-views,
    with leading dimensions of the whole arrays."""
    MM, NN, KK = 768, 640, 1024
    qa, sa, qb, sb = _operands(rg, ctx, MM, NN, KK, seed=8)
    m0, n0, k0, M, N, K = 256, 128, 384, 384, 384, 512
    C = torch.full((M, N), float("nan"), device="cuda")
    lds_a, lds_b = sa.shape[1], sb.shape[1]
    qa_v = qa.view(-1)[m0 * KK + k0:]
    sa_v = sa.view(-1)[(m0 // 128) * lds_a + k0 // 128:]
    qb_v = qb.view(-1)[k0 * NN + n0:]
    sb_v = sb.view(-1)[(k0 // 128) * lds_b + n0 // 128:]
    rg.rg_gemm_fp8_ex(ctx, M, N, K, qa_v, KK, sa_v, lds_a, qb_v, NN, sb_v, lds_b, C, N, rg.fp8_variant(1, 2), 0,
                      0, 0, 0)
    rg.rg_check(ctx)
    A = of.dequantize(qa.cpu().numpy(), sa.cpu().numpy())[m0:m0 + M, k0:k0 + K]
    B = of.dequantize(qb.cpu().numpy(), sb.cpu().numpy())[k0:k0 + K, n0:n0 + N]
    ratio, ez = og.error_ratio(C.cpu().numpy(), A @ B, np.abs(A) @ np.abs(B))
    assert ez and ratio <= FP8_BOUND_FACTOR * K * 2.0 ** -24


def _fp8_plan(rg, seed):
    g = rg.make_grid((128, 128, 4))
    rs = np.random.default_rng(seed)
    s = (np.arange(4) + 1) * 128.0
    base = 50.0 + 2.0 * s[:, None, None] * s[None, :, None] * s[None, None, :] / 4e5
    T0 = np.stack([np.round(base * rs.uniform(0.6, 1.6, size=(4, 4, 4))) for _ in FP8_VARIANTS]).astype(np.int64)
    plan = rg.rg_plan_build(g, T0.reshape(len(FP8_VARIANTS), -1), FP8_VARIANTS)
    return plan


def test_fp8_plan_execution_every_cell(rg, ctx):
    """An FP8 plan (FP8 variant ids; padding, M/N/K splits with beta = 1 pieces) executed through
    rg_gemm_fp8_plan on every cell of its grid and on off-grid shapes."""
    plan = _fp8_plan(rg, 2)
    try:
        acts = set(rg.rg_plan_tables(plan)["action"].ravel().tolist())
        assert acts >= {0, 1, 2, 3}, acts
        shapes = [(128 * (a + 1), 128 * (b + 1), 128 * (c + 1)) for a in range(4) for b in range(4) for c in range(4)]
        shapes += [(200, 144, 272), (511, 400, 336)]
        for i, (M, N, K) in enumerate(shapes):
            qa, sa, qb, sb = _operands(rg, ctx, M, N, K, seed=100 + i)
            C = torch.full((M, N), float("nan"), device="cuda")
            rg.rg_gemm_fp8_plan(ctx, plan, M, N, K, qa, K, sa, sa.shape[1], qb, N, sb, sb.shape[1], C, N)
            rg.rg_check(ctx)
            _check_fp8(C.cpu().numpy(), qa.cpu().numpy(), sa.cpu().numpy(), qb.cpu().numpy(), sb.cpu().numpy(), K)
        # precisions do not mix: an FP8 plan is refused by the BF16 path and a BF16 plan by the FP8 path
        A = torch.zeros((128, 128), device="cuda", dtype=torch.bfloat16)
        Cb = torch.zeros((128, 128), device="cuda")
        with pytest.raises(rg.RGError) as e:
            rg.rg_gemm_plan(ctx, plan, 128, 128, 128, A, 128, A, 128, Cb, 128)
        assert e.value.code == rg.RG_ERR_INVALID
        gb = rg.make_grid((128, 128, 1))
        bplan = rg.rg_plan_build(gb, np.ones((1, 1), np.int64), [1])
        try:
            q = torch.zeros((128, 128), dtype=torch.uint8, device="cuda")
            s1 = torch.ones((1, 1), device="cuda")
            with pytest.raises(rg.RGError) as e:
                rg.rg_gemm_fp8_plan(ctx, bplan, 128, 128, 128, q, 128, s1, 1, q, 128, s1, 1, Cb, 128)
            assert e.value.code == rg.RG_ERR_INVALID
        finally:
            rg.rg_plan_free(bplan)
        with pytest.raises(rg.RGError):
            rg.rg_plan_build(gb, np.ones((2, 1), np.int64), [1, 64])       # BF16 and FP8 ids mixed
    finally:
        rg.rg_plan_free(plan)


def test_fp8_sweep_variants_and_plan(rg, ctx):
    """rg_sweep_fp8 over several FP8 variants (split pruning marks unhelpful splits) and over a plan;
    the returned surfaces and statistics are the oracle's from the returned times."""
    from oracle import roughness
    Mx = 512
    x = synthetic.normal_stream_f32(0, 1, Mx * Mx).reshape(Mx, Mx)
    qa, sa = quantize(rg, ctx, x)
    qb, sb = quantize(rg, ctx, x)
    C = torch.zeros(Mx * Mx, device="cuda")
    g = rg.make_grid((128, 128, 4))
    vids = [rg.fp8_variant(0, 1), rg.fp8_variant(0, 4), rg.fp8_variant(1, 1), rg.fp8_variant(1, 2)]
    t, tf, st = rg.rg_sweep_fp8_surfaces(ctx, g, vids, qa, sa, qb, sb, C)
    assert t.shape == (4, 64) and np.all(t[0] < 10 ** 8) and np.all(t[2] < 10 ** 8)
    ogrid = ((128, 128, 4),) * 3
    S = roughness.surface(t[0].reshape(4, 4, 4), ogrid)
    ref = roughness.roughness_all(S)
    assert np.array_equal(tf[0], S.ravel()) and st[0][5] == roughness.mean(S)
    assert [st[0][i] for i in range(5)] == [ref[k] for k in ("R_M", "R_N", "R_K", "R_3D", "R_N_slice")]
    plan = rg.rg_plan_build(g, np.where(t == rg.RG_T_UNMEASURED, 1 << 40, t), vids)
    try:
        tp = rg.rg_sweep_fp8(ctx, g, qa, sa, qb, sb, C, plan=plan)
        assert tp.shape == (1, 64) and np.all(tp > 0) and np.all(tp < 10 ** 8)
    finally:
        rg.rg_plan_free(plan)

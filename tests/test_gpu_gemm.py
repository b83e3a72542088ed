"""GPU parity of the BF16 NN GEMM (rg_gemm through the C ABI) against the CPU
oracle: every variant, the small-sweep shapes, ragged and padded shapes,
beta = 1, split-K, closed forms, full-size sampled rows and columns, and the
error paths."""
import numpy as np
import pytest

import synthetic
from oracle import gemm as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL_VARIANTS = list(range(55))          # 32 split-K (8 tiles), 8 stream-K, 12 cta_group::2 (3 tiles x 4 splits), 3 cta_group::2 stream-K


@pytest.fixture(scope="module")
def rg():
    from paper_2605_29752_gb300 import rg as _rg
    return _rg


@pytest.fixture(scope="module")
def ctx(rg):
    h = rg.rg_init(0)
    yield h
    rg.rg_destroy(h)


def dev_bf16(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).cuda().view(torch.bfloat16)


def run(rg, ctx, a_bits, b_bits, v, beta=0, c0=None, pads=(0, 0, 0)):
    M, K = a_bits.shape
    N = b_bits.shape[1]
    A, B = dev_bf16(a_bits), dev_bf16(b_bits)
    C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32) if c0 is None else \
        torch.from_numpy(c0.astype(np.float32)).cuda()
    rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, v, beta, *pads)
    rg.rg_check(ctx)
    return C.cpu().numpy()


def check(c, a_bits, b_bits, c0=None):
    a, b = og.bf16_bits_to_f64(a_bits), og.bf16_bits_to_f64(b_bits)
    c64 = og.gemm_f64(a, b)
    s = og.abs_sum(a, b)
    if c0 is not None:
        c64 = c64 + c0.astype(np.float32).astype(np.float64)
        s = s + np.abs(c0.astype(np.float32).astype(np.float64))
    ratio, exact_zero = og.error_ratio(c, c64, s)
    K = a.shape[1]
    assert not np.any(np.isnan(c)), "unwritten output elements"
    assert exact_zero and ratio <= og.bound(K + (1 if c0 is not None else 0)), ratio
    return ratio


@pytest.mark.parametrize("v", ALL_VARIANTS)
def test_every_variant_ragged(rg, ctx, v):
    M, N, K = 300, 200, 328           # partial tiles in M, N and K for every tile shape
    a, b = synthetic.operands_bf16(M, N, K, seed=1)
    check(run(rg, ctx, a, b, v), a, b)


SMALL = [128, 256, 384, 512]


@pytest.mark.parametrize("M", SMALL)
@pytest.mark.parametrize("N", SMALL)
@pytest.mark.parametrize("K", SMALL)
def test_small_sweep_shapes_full_matrix(rg, ctx, M, N, K):
    a, b = synthetic.operands_bf16(M, N, K, seed=0)
    check(run(rg, ctx, a, b, rg.variant(1, 1)), a, b)


@pytest.mark.parametrize("v", [rg_v for rg_v in (0, 4, 8, 12, 16, 20, 9, 22)])
def test_identity_all_ones_rank_one_exact(rg, ctx, v):
    one = np.float32(1.0).view(np.uint32) >> 16
    K = 256
    eye = np.zeros((K, K), np.uint16)
    eye[np.arange(K), np.arange(K)] = one
    _, b = synthetic.operands_bf16(K, 320, K, seed=2)
    c = run(rg, ctx, eye, b, v)
    assert np.array_equal(c, og.bf16_bits_to_f64(b).astype(np.float32))
    ones_a = np.full((192, 384), one, np.uint16)
    ones_b = np.full((384, 136), one, np.uint16)
    assert np.all(run(rg, ctx, ones_a, ones_b, v) == 384.0)
    a, b = synthetic.operands_bf16(200, 264, 96, seed=3)
    a1 = np.zeros_like(a)
    a1[:, 17] = a[:, 17]
    c = run(rg, ctx, a1, b, v)
    exact = np.outer(og.bf16_bits_to_f64(a1[:, 17]), og.bf16_bits_to_f64(b[17, :])).astype(np.float32)
    assert np.array_equal(c, exact)


@pytest.mark.parametrize("v", [1, 6, 13, 21])
def test_disjoint_k_blocks(rg, ctx, v):
    # A nonzero only in K-block 0 columns, B only in the last K block rows: C == 0 exactly
    M, N, K = 256, 256, 1024
    a, b = synthetic.operands_bf16(M, N, K, seed=4)
    a[:, 64:] = 0
    b[:-64, :] = 0
    assert np.all(run(rg, ctx, a, b, v) == 0.0)


@pytest.mark.parametrize("v", [0, 5, 10, 15, 19, 23])
def test_padding_gives_same_result(rg, ctx, v):
    M, N, K = 256, 384, 256
    a, b = synthetic.operands_bf16(M, N, K, seed=5)
    c_plain = run(rg, ctx, a, b, v)
    c_pad = run(rg, ctx, a, b, v, pads=(M + 256, N + 128, K + 384))
    check(c_pad, a, b)
    if rg.SPLITS[v % 4] == 1:
        # zero K padding adds exact zeros: bitwise the same result
        assert np.array_equal(c_plain, c_pad)
    # M/N padding alone never changes any output element's summation
    assert np.array_equal(c_plain, run(rg, ctx, a, b, v, pads=(M + 256, N + 128, K)))


@pytest.mark.parametrize("v", [1, 3, 9, 18])
def test_beta_one_accumulates(rg, ctx, v):
    M, N, K = 384, 256, 512
    a, b = synthetic.operands_bf16(M, N, K, seed=6)
    c0 = synthetic.normal_stream_f32(6, 5, M * N).reshape(M, N)
    check(run(rg, ctx, a, b, v, beta=1, c0=c0), a, b, c0=c0)


@pytest.mark.parametrize("v", [1, 2, 3, 7, 11, 15, 19, 23, 25, 26, 27, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39])
def test_split_k_deterministic(rg, ctx, v):
    M, N, K = 512, 384, 2048
    a, b = synthetic.operands_bf16(M, N, K, seed=7)
    c1 = run(rg, ctx, a, b, v)
    c2 = run(rg, ctx, a, b, v)
    check(c1, a, b)
    assert np.array_equal(c1, c2)


def test_more_splits_than_k_blocks(rg, ctx):
    M, N, K = 128, 128, 128                  # 2 K blocks, 8 splits: six splits add exact zeros
    a, b = synthetic.operands_bf16(M, N, K, seed=8)
    check(run(rg, ctx, a, b, rg.variant(1, 8)), a, b)


@pytest.mark.parametrize("shape", [(4096, 4096, 4096), (3968, 4096, 3840), (4096, 1152, 4096)])
@pytest.mark.parametrize("tile", range(8))
def test_full_size_sampled(rg, ctx, shape, tile):
    M, N, K = shape
    a_bits, b_bits = synthetic.operands_bf16(M, N, K, seed=0)
    c = run(rg, ctx, a_bits, b_bits, rg.variant(tile, 1 if tile % 2 else 2))
    a, b = og.bf16_bits_to_f64(a_bits), og.bf16_bits_to_f64(b_bits)
    rs = np.random.default_rng(tile)
    rows = rs.choice(M, 8, replace=False)
    cols = rs.choice(N, 8, replace=False)
    cr, sr, cc, sc = og.sampled_rows_cols(a, b, rows, cols)
    for got, ref, s in ((c[rows, :], cr, sr), (c[:, cols], cc, sc)):
        ratio, exact_zero = og.error_ratio(got, ref, s)
        assert exact_zero and ratio <= og.bound(K), ratio


def test_empty_and_k_zero(rg, ctx):
    C = torch.full((4, 8), 5.0, device="cuda")
    A = torch.zeros((4, 8), device="cuda", dtype=torch.bfloat16)
    rg.rg_gemm(ctx, 0, 8, 8, A, 8, A, 8, C, 8, 1)
    rg.rg_gemm(ctx, 4, 8, 0, A, 8, A, 8, C, 8, 1, 1)     # beta = 1, K = 0: C unchanged
    rg.rg_check(ctx)
    assert torch.all(C == 5.0)
    rg.rg_gemm(ctx, 4, 8, 0, A, 8, A, 8, C, 8, 1, 0)     # beta = 0, K = 0: C = 0
    rg.rg_check(ctx)
    assert torch.all(C == 0.0)


def test_alignment_and_argument_errors(rg, ctx):
    A = torch.zeros((64, 64), device="cuda", dtype=torch.bfloat16)
    C = torch.zeros((64, 64), device="cuda")
    assert rg.rg_gemm_status(ctx, 64, 64, 60, A, 60, A, 64, C, 64, 1) == rg.RG_ERR_ALIGN
    assert rg.rg_gemm_status(ctx, 64, 64, 64, A.data_ptr() + 2, 64, A, 64, C, 64, 1) == rg.RG_ERR_ALIGN
    assert rg.rg_gemm_status(ctx, 64, 64, 64, A, 64, A, 64, C, 64, 99) == rg.RG_ERR_INVALID
    assert rg.rg_gemm_status(ctx, 64, 64, 64, A, 64, A, 64, C, 64, 1, 2) == rg.RG_ERR_INVALID
    assert rg.rg_gemm_status(ctx, 64, 64, 64, A, 64, A, 64, C, 64, 1, 0, 32) == rg.RG_ERR_INVALID
    assert rg.rg_gemm_status(ctx, 64, 64, 64, A, 32, A, 64, C, 64, 1) == rg.RG_ERR_INVALID
    rg.rg_check(ctx)


@pytest.mark.parametrize("tile", range(8))
@pytest.mark.parametrize("shape", [(1664, 1664, 2048), (2176, 1920, 1152), (2560, 2048, 1024), (128, 128, 4096),
                                   (256, 512, 640)])
def test_stream_k_uneven_waves(rg, ctx, tile, shape):
    """Stream-K on shapes whose tile count is just above a wave, or far below the SM count: every tile
    spans one or several CTAs' iteration ranges; the result is within the bound and deterministic."""
    M, N, K = shape
    a, b = synthetic.operands_bf16(M, N, K, seed=12)
    v = rg.variant(tile, rg.SK)
    c1 = run(rg, ctx, a, b, v)
    check(c1, a, b)
    assert np.array_equal(c1, run(rg, ctx, a, b, v))


@pytest.mark.parametrize("v", [32, 35, 37, 38, 39])
def test_stream_k_beta_one(rg, ctx, v):
    M, N, K = 640, 384, 1536
    a, b = synthetic.operands_bf16(M, N, K, seed=13)
    c0 = synthetic.normal_stream_f32(13, 5, M * N).reshape(M, N)
    check(run(rg, ctx, a, b, v, beta=1, c0=c0), a, b, c0=c0)


@pytest.mark.parametrize("tile", [4, 5, 7])
@pytest.mark.parametrize("shape", [(384, 640, 1024), (1664, 1664, 2048), (128, 64, 256), (200, 264, 96),
                                   (4096, 1152, 4096)])
def test_two_sm(rg, ctx, tile, shape):
    """cta_group::2 pairs (one 256-row tile per 2-CTA cluster, B split by columns between
    the CTAs): ragged edges, an odd CTA wholly past M, and a full-height case; bitwise
    equal to the 1-CTA kernel of the same tile."""
    M, N, K = shape
    a, b = synthetic.operands_bf16(M, N, K, seed=16)
    c = run(rg, ctx, a, b, rg.variant(tile, rg.TWO_SM))
    if M * N * K <= 1024 * 1024 * 1024:
        check(c, a, b)
    else:
        rs = np.random.default_rng(1)
        rows, cols = rs.choice(M, 8, replace=False), rs.choice(N, 8, replace=False)
        A64, B64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
        cr, sr, cc, sc = og.sampled_rows_cols(A64, B64, rows, cols)
        for got, ref, s in ((c[rows, :], cr, sr), (c[:, cols], cc, sc)):
            ratio, exact_zero = og.error_ratio(got, ref, s)
            assert exact_zero and ratio <= og.bound(K), ratio
    # the pair computes every output element with the same MMA sequence as the 1-CTA kernel
    assert np.array_equal(c, run(rg, ctx, a, b, rg.variant(tile, 1)))


@pytest.mark.parametrize("tile", [4, 5, 7])
def test_two_sm_exact_cases_beta_and_padding(rg, ctx, tile):
    v = rg.variant(tile, rg.TWO_SM)
    one = np.float32(1.0).view(np.uint32) >> 16
    K = 256
    eye = np.zeros((K, K), np.uint16)
    eye[np.arange(K), np.arange(K)] = one
    _, b = synthetic.operands_bf16(K, 320, K, seed=2)
    assert np.array_equal(run(rg, ctx, eye, b, v), og.bf16_bits_to_f64(b).astype(np.float32))
    ones_a = np.full((392, 384), one, np.uint16)
    ones_b = np.full((384, 136), one, np.uint16)
    assert np.all(run(rg, ctx, ones_a, ones_b, v) == 384.0)
    M, N, K = 640, 384, 1536
    a, b = synthetic.operands_bf16(M, N, K, seed=15)
    c0 = synthetic.normal_stream_f32(15, 5, M * N).reshape(M, N)
    check(run(rg, ctx, a, b, v, beta=1, c0=c0), a, b, c0=c0)
    M, N, K = 256, 384, 256
    a, b = synthetic.operands_bf16(M, N, K, seed=5)
    c_plain = run(rg, ctx, a, b, v)
    check(c_plain, a, b)
    assert np.array_equal(c_plain, run(rg, ctx, a, b, v, pads=(M + 256, N + 128, K + 384)))


@pytest.mark.parametrize("tile", [4, 5, 7])
@pytest.mark.parametrize("split", [2, 4, 8])
def test_two_sm_split_k(rg, ctx, tile, split):
    """cta_group::2 with split-K: each CTA reduces its own 128 rows in the fixed split
    order, so the result is bitwise that of the 1-CTA kernel with the same split; beta = 1
    accumulates."""
    v = rg.variant(tile, (rg.TWO_SM, split))
    for (M, N, K), seed in (((512, 384, 2048), 7), ((200, 264, 1000), 8), ((1024, 1024, 4096), 9)):
        a, b = synthetic.operands_bf16(M, N, K, seed=seed)
        c = run(rg, ctx, a, b, v)
        if M * N * K <= 1024 * 1024 * 1024:
            check(c, a, b)
        assert np.array_equal(c, run(rg, ctx, a, b, rg.variant(tile, split)))
        assert np.array_equal(c, run(rg, ctx, a, b, v))
    M, N, K = 640, 384, 1536
    a, b = synthetic.operands_bf16(M, N, K, seed=13)
    c0 = synthetic.normal_stream_f32(13, 5, M * N).reshape(M, N)
    check(run(rg, ctx, a, b, v, beta=1, c0=c0), a, b, c0=c0)


@pytest.mark.parametrize("tile", [4, 5, 7])
@pytest.mark.parametrize("shape", [(4096, 1280, 4096), (4096, 2432, 1024), (2560, 2560, 2048), (3968, 3712, 512),
                                   (1000, 1000, 1000), (512, 512, 1024), (200, 264, 96)])
def test_two_sm_stream_k(rg, ctx, tile, shape):
    """cta_group::2 stream-K on shapes whose pair-tile count is just above whole waves of the 2-CTA
    clusters (the remainder tiles' K iterations shared by several clusters), far below one wave,
    and ragged: within the oracle's bound (sampled rows and columns on the large shapes) and
    deterministic from launch to launch."""
    M, N, K = shape
    a, b = synthetic.operands_bf16(M, N, K, seed=17)
    v = rg.variant(tile, rg.TWO_SM_SK)
    c = run(rg, ctx, a, b, v)
    if M * N * K <= 1024 * 1024 * 1024:
        check(c, a, b)
    else:
        rs = np.random.default_rng(3)
        rows, cols = rs.choice(M, 8, replace=False), rs.choice(N, 8, replace=False)
        A64, B64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
        cr, sr, cc, sc = og.sampled_rows_cols(A64, B64, rows, cols)
        for got, ref, s in ((c[rows, :], cr, sr), (c[:, cols], cc, sc)):
            ratio, exact_zero = og.error_ratio(got, ref, s)
            assert exact_zero and ratio <= og.bound(K), ratio
        assert not np.any(np.isnan(c))
    assert np.array_equal(c, run(rg, ctx, a, b, v))


@pytest.mark.parametrize("tile", [4, 5, 7])
def test_two_sm_stream_k_beta_and_padding(rg, ctx, tile):
    v = rg.variant(tile, rg.TWO_SM_SK)
    M, N, K = 2304, 1536, 1536
    a, b = synthetic.operands_bf16(M, N, K, seed=18)
    c0 = synthetic.normal_stream_f32(18, 5, M * N).reshape(M, N)
    rs = np.random.default_rng(4)
    rows, cols = rs.choice(M, 6, replace=False), rs.choice(N, 6, replace=False)
    A64, B64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
    cr, sr, cc, sc = og.sampled_rows_cols(A64, B64, rows, cols)
    c0d = c0.astype(np.float32).astype(np.float64)
    got = run(rg, ctx, a, b, v, beta=1, c0=c0)
    for g_, ref, s_ in ((got[rows, :], cr + c0d[rows, :], sr + np.abs(c0d[rows, :])),
                        (got[:, cols], cc + c0d[:, cols], sc + np.abs(c0d[:, cols]))):
        ratio, exact_zero = og.error_ratio(g_, ref, s_)
        assert exact_zero and ratio <= og.bound(K + 1), ratio
    # padded launch extents change the tile count and with it the stream-K split points, so only
    # the bound is asserted
    M, N, K = 1280, 1152, 2048
    a, b = synthetic.operands_bf16(M, N, K, seed=19)
    check(run(rg, ctx, a, b, v, pads=(M + 256, N + 256, K + 128)), a, b)


@pytest.mark.parametrize("tile", range(8))
def test_column_panel_tile_order(rg, ctx, tile):
    """N = 8192 with K = 4096 puts more tile columns than one 32 MiB panel of B holds, so
    tiles run in column panels: every variant family still covers every tile once
    (sampled rows and columns against the oracle; the cta_group::2 form bitwise equal to
    the 1-CTA kernel)."""
    M, N, K = 520, 8192, 4096
    a, b = synthetic.operands_bf16(M, N, K, seed=21)
    c = run(rg, ctx, a, b, rg.variant(tile, 1))
    rs = np.random.default_rng(2)
    rows, cols = rs.choice(M, 6, replace=False), rs.choice(N, 6, replace=False)
    A64, B64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
    cr, sr, cc, sc = og.sampled_rows_cols(A64, B64, rows, cols)
    for got, ref, s in ((c[rows, :], cr, sr), (c[:, cols], cc, sc)):
        ratio, exact_zero = og.error_ratio(got, ref, s)
        assert exact_zero and ratio <= og.bound(K), ratio
    others = [rg.variant(tile, rg.SK)]
    if tile in rg.PAIR_TILES:                   # the pair tiles also run as cta_group::2 pairs
        others.append(rg.variant(tile, rg.TWO_SM))
    for v in others:
        got = run(rg, ctx, a, b, v)
        if v == rg.variant(tile, rg.SK):
            check_rows = got[rows, :]
            ratio, exact_zero = og.error_ratio(check_rows, cr, sr)
            assert exact_zero and ratio <= og.bound(K), (rg.variant_name(v), ratio)
        else:
            assert np.array_equal(got, c), rg.variant_name(v)


def test_static_operands_mode(rg, ctx):
    """With A and B declared static, loads and MMAs start before the preceding grid
    completes and only the epilogue waits for it: back-to-back launches into the same
    C, a K-split plan-style chain (beta = 1 after beta = 0) and split-K launches give
    bitwise the results of the default mode."""
    M, N, K = 640, 520, 1536
    a, b = synthetic.operands_bf16(M, N, K, seed=22)
    A, B = dev_bf16(a), dev_bf16(b)
    vs = [rg.variant(1, 1), rg.variant(2, 4), rg.variant(5, rg.TWO_SM), rg.variant(0, rg.SK)]
    results = {}
    for static in (False, True):
        rg.rg_set_static_operands(ctx, static)
        try:
            for v in vs:
                C = torch.full((M, N), float("nan"), device="cuda")
                for _ in range(4):                                  # the same C rewritten back to back
                    rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, v)
                rg.rg_check(ctx)
                results[(static, v)] = C.cpu().numpy()
            # K split into two chained launches: C = A[:, :k1] B[:k1] then C += A[:, k1:] B[k1:]
            k1 = 512
            C = torch.full((M, N), float("nan"), device="cuda")
            rg.rg_gemm(ctx, M, N, k1, A, K, B, N, C, N, rg.variant(1, 1), 0)
            rg.rg_gemm(ctx, M, N, K - k1, A[:, k1:], K, B[k1:], N, C, N, rg.variant(1, 1), 1)
            rg.rg_check(ctx)
            results[(static, "chain")] = C.cpu().numpy()
        finally:
            rg.rg_set_static_operands(ctx, False)
    for v in vs:
        check(results[(True, v)], a, b)
        assert np.array_equal(results[(True, v)], results[(False, v)]), rg.variant_name(v)
    check(results[(True, "chain")], a, b)
    assert np.array_equal(results[(True, "chain")], results[(False, "chain")])

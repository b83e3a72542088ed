"""GPU parity of the grouped persistent GEMM (rg_gemm_grouped: many problems
in one launch, replayed from CUDA graphs): every problem against the oracle,
and bitwise against rg_gemm with the same tile (each output tile is computed by
the same code in the same order)."""
import numpy as np
import pytest

import synthetic
from oracle import gemm as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    from paper_2605_29752_gb300 import rg as _rg
    return _rg


@pytest.fixture(scope="module")
def ctx(rg):
    h = rg.rg_init(0)
    yield h
    rg.rg_destroy(h)


def _problem(M, N, K, seed):
    a, b = synthetic.operands_bf16(M, N, K, seed=seed)
    A = torch.from_numpy(a.view(np.int16)).cuda().view(torch.bfloat16)
    B = torch.from_numpy(b.view(np.int16)).cuda().view(torch.bfloat16)
    return a, b, A, B


SHAPES = [(128, 128, 128), (300, 200, 328), (1024, 512, 768), (256, 1024, 64), (72, 40, 1024),
          (2048, 384, 256), (128, 256, 4096), (640, 640, 640)]


@pytest.mark.parametrize("tile", range(8))
def test_grouped_mixed_shapes_match_oracle_and_rg_gemm(rg, ctx, tile):
    g = rg.rg_group_create(ctx, tile, 64)
    try:
        probs, outs, refs = [], [], []
        for i, (M, N, K) in enumerate(SHAPES):
            a, b, A, B = _problem(M, N, K, seed=20 + i)
            C = torch.full((M, N), float("nan"), device="cuda")
            Cr = torch.full((M, N), float("nan"), device="cuda")
            pads = (M + 128, N, K + 64) if i % 3 == 1 else (0, 0, 0)
            probs.append((M, N, K, A, K, B, N, C, N, 0) + pads)
            rg.rg_gemm(ctx, M, N, K, A, K, B, N, Cr, N, rg.variant(tile, 1), 0, *pads)
            outs.append((a, b, C, A, B))
            refs.append(Cr)
        rg.rg_gemm_grouped(g, probs)
        rg.rg_check(ctx)
        for (a, b, C, A, B), Cr in zip(outs, refs):
            c = C.cpu().numpy()
            ok, ratio = og.check(c, og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b))
            assert ok and not np.any(np.isnan(c)), ratio
            assert np.array_equal(c, Cr.cpu().numpy())
    finally:
        rg.rg_group_destroy(g)


def test_grouped_beta_and_many_replays(rg, ctx):
    tile = 1
    g = rg.rg_group_create(ctx, tile, 16)
    try:
        M, N, K = 384, 256, 512
        a, b, A, B = _problem(M, N, K, seed=5)
        C0 = synthetic.normal_stream_f32(5, 7, M * N).reshape(M, N)
        streams = [torch.cuda.Stream() for _ in range(3)]
        results = []
        for call in range(10):                       # more calls than the group's slots
            C = torch.from_numpy(C0).cuda()
            torch.cuda.synchronize()
            s = streams[call % 3]
            rg.rg_gemm_grouped(g, [(M, N, K, A, K, B, N, C, N, 1)], stream=s)
            results.append((C, s))
        torch.cuda.synchronize()
        rg.rg_check(ctx)
        a64, b64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
        c64 = a64 @ b64 + C0.astype(np.float64)
        s64 = np.abs(a64) @ np.abs(b64) + np.abs(C0.astype(np.float64))
        first = results[0][0].cpu().numpy()
        for C, _ in results:
            c = C.cpu().numpy()
            ratio, ez = og.error_ratio(c, c64, s64)
            assert ez and ratio <= og.bound(K + 1)
            assert np.array_equal(c, first)
    finally:
        rg.rg_group_destroy(g)


def test_grouped_limits(rg, ctx):
    """More problems than a work list holds run as several launches in turn; K == 0 problems and a
    problem whose split-K partials alone exceed the group's workspace are refused before anything
    is enqueued."""
    g = rg.rg_group_create(ctx, 0, 2, 1 << 20)
    try:
        a, b, A, B = _problem(192, 136, 200, seed=8)
        rg.rg_gemm_grouped(g, [])
        outs = [torch.full((192, 136), float("nan"), device="cuda") for _ in range(5)]
        rg.rg_gemm_grouped(g, [(192, 136, 200, A, 200, B, 136, C, 136) for C in outs])
        rg.rg_check(ctx)
        for C in outs:
            ok, ratio = og.check(C.cpu().numpy(), og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b))
            assert ok, ratio
        Z = torch.zeros((64, 64), device="cuda")
        with pytest.raises(rg.RGError):
            rg.rg_gemm_grouped(g, [(64, 64, 0, A, 64, A, 64, Z, 64)])
        big = torch.zeros((1024, 1024), device="cuda", dtype=torch.bfloat16)
        Cb = torch.full((1024, 1024), 7.0, device="cuda")
        # 128x128 split 2 on 1024^2: 64 tiles x 2 x 64 KiB = 8 MiB of partials > the 1 MiB workspace
        with pytest.raises(rg.RGError) as e:
            rg.rg_gemm_grouped(g, [(1024, 1024, 1024, big, 1024, big, 1024, Cb, 1024, 0, 0, 0, 0, rg.variant(1, 2)),
                                   (192, 136, 200, A, 200, B, 136, outs[0], 136)])
        assert e.value.code == rg.RG_ERR_SHAPE
        torch.cuda.synchronize()
        assert torch.all(Cb == 7.0)
    finally:
        rg.rg_group_destroy(g)


# (M, N, K, variant, beta, pads): split-K on several tiles, cta_group::2 with and without split,
# a stream-K choice (runs as its tile with split 1), padding and beta = 1
MIXED = [
    (512, 384, 2048, ("t", 1, 2), 0, (0, 0, 0)),
    (300, 200, 1000, ("t", 0, 4), 0, (384, 256, 1024)),
    (256, 512, 1536, ("t", 2, 8), 1, (0, 0, 0)),
    (640, 256, 512, ("t", 3, 2), 0, (0, 0, 0)),
    (520, 512, 2048, ("2sm", 5, 1), 0, (0, 0, 0)),
    (768, 640, 1024, ("2sm", 4, 2), 0, (1024, 640, 1024)),
    (384, 384, 4096, ("2sm", 5, 4), 1, (0, 0, 0)),
    (1024, 768, 512, ("sk", 2), 0, (0, 0, 0)),
    (640, 512, 768, ("2smsk", 5), 0, (0, 0, 0)),
    (200, 136, 96, ("t", 1, 1), 0, (0, 0, 0)),
]


def _vid(rg, spec):
    kind = spec[0]
    if kind == "t":
        return rg.variant(spec[1], spec[2])
    if kind == "2sm":
        return rg.variant(spec[1], (rg.TWO_SM, spec[2]))
    if kind == "sk":
        return rg.variant(spec[1], rg.SK)
    return rg.variant(spec[1], rg.TWO_SM_SK)


def _as_grouped(rg, v):
    """The variant a grouped launch runs for v: stream-K choices run as their tile, split 1."""
    name = rg.variant_name(v)
    if name.endswith("/2SM-SK"):
        return rg.variant(rg.variant_tile(v), rg.TWO_SM)
    if name.endswith("/SK"):
        return rg.variant(rg.variant_tile(v), 1)
    return v


# partials of 0.5-1 MiB each: with a 1 MiB workspace each family runs as several launches
SMALL_SPLITS = [
    (256, 256, 1024, ("t", 0, 2), 0, (0, 0, 0)),
    (256, 256, 768, ("t", 0, 2), 1, (0, 0, 0)),
    (200, 256, 1024, ("t", 0, 2), 0, (0, 0, 0)),
    (128, 384, 2048, ("t", 0, 4), 0, (0, 0, 0)),
    (256, 128, 1024, ("t", 1, 4), 0, (0, 0, 0)),
    (256, 256, 1024, ("2sm", 4, 2), 0, (0, 0, 0)),
    (512, 256, 1024, ("2sm", 4, 2), 1, (0, 0, 0)),
    (256, 256, 2048, ("2sm", 5, 2), 0, (0, 0, 0)),
    (136, 72, 512, ("t", 1, 1), 0, (0, 0, 0)),
]


@pytest.mark.parametrize("case", ["mixed_64MiB", "small_splits_1MiB"])
def test_grouped_split_k_and_two_sm_items(rg, ctx, case):
    """Problems with their own variants (split-K tiles, cta_group::2 pairs with split-K, stream-K
    choices) in one call: one launch per kernel family, several per family when the workspace
    cannot hold all their partials at once; each result within the oracle's bound and bitwise
    rg_gemm's for the same variant."""
    problems, ws = (MIXED, 64 << 20) if case == "mixed_64MiB" else (SMALL_SPLITS, 1 << 20)
    g = rg.rg_group_create(ctx, 1, 8, ws)
    try:
        probs, checks = [], []
        for i, (M, N, K, spec, beta, pads) in enumerate(problems):
            v = _vid(rg, spec)
            a, b, A, B = _problem(M, N, K, seed=40 + i)
            c0 = synthetic.normal_stream_f32(40 + i, 5, M * N).reshape(M, N) if beta else None
            C = torch.from_numpy(c0).cuda() if beta else torch.full((M, N), float("nan"), device="cuda")
            Cr = torch.from_numpy(c0).cuda() if beta else torch.full((M, N), float("nan"), device="cuda")
            rg.rg_gemm(ctx, M, N, K, A, K, B, N, Cr, N, _as_grouped(rg, v), beta, *pads)
            probs.append((M, N, K, A, K, B, N, C, N, beta) + pads + (v,))
            checks.append((a, b, c0, C, Cr, v))
        n0 = rg.rg_launch_count(ctx)
        rg.rg_gemm_grouped(g, probs)
        rg.rg_check(ctx)
        families = {("2sm" if "2SM" in rg.variant_name(_as_grouped(rg, c[5])) else "") + str(rg.variant_tile(c[5]))
                    for c in checks}
        if case == "small_splits_1MiB":
            assert rg.rg_launch_count(ctx) - n0 > len(families)      # some family ran as several launches
        else:
            assert rg.rg_launch_count(ctx) - n0 == len(families)     # one launch per family
        for a, b, c0, C, Cr, v in checks:
            got = C.cpu().numpy()
            a64, b64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
            c64 = a64 @ b64 + (c0.astype(np.float64) if c0 is not None else 0.0)
            s64 = np.abs(a64) @ np.abs(b64) + (np.abs(c0.astype(np.float64)) if c0 is not None else 0.0)
            ratio, ez = og.error_ratio(got, c64, s64)
            assert ez and ratio <= og.bound(a.shape[1] + 1), (rg.variant_name(v), ratio)
            assert np.array_equal(got, Cr.cpu().numpy()), rg.variant_name(v)
    finally:
        rg.rg_group_destroy(g)


@pytest.mark.parametrize("tile", range(8))
def test_cluster_split_equals_workspace_split(rg, ctx, tile):
    """rg_gemm runs split-K of the 128x256, 256x128 and 256x256 tiles as a cluster of S CTAs that
    reduce through distributed shared memory (the workspace kernel for the smaller tiles and where the
    partials do not fit: 256x256 with S = 8); a grouped launch runs the same split through the
    workspace and its last arriver.  Both sum the S partials in the order 0..S-1, so they agree bit
    for bit; both lie within the oracle's bound."""
    M, N, K = 520, 264, 1000
    g = rg.rg_group_create(ctx, tile, 8, 64 << 20)
    try:
        a, b, A, B = _problem(M, N, K, seed=60 + tile)
        a64, b64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
        for s in (2, 4, 8):
            v = rg.variant(tile, s)
            for beta in (0, 1):
                c0 = synthetic.normal_stream_f32(61 + tile, s, M * N).reshape(M, N)
                Cc = torch.from_numpy(c0).cuda() if beta else torch.full((M, N), float("nan"), device="cuda")
                Cw = torch.from_numpy(c0).cuda() if beta else torch.full((M, N), float("nan"), device="cuda")
                rg.rg_gemm(ctx, M, N, K, A, K, B, N, Cc, N, v, beta)
                rg.rg_gemm_grouped(g, [(M, N, K, A, K, B, N, Cw, N, beta, 0, 0, 0, v)])
                rg.rg_check(ctx)
                got = Cc.cpu().numpy()
                c64 = a64 @ b64 + (c0.astype(np.float64) if beta else 0.0)
                s64 = np.abs(a64) @ np.abs(b64) + (np.abs(c0.astype(np.float64)) if beta else 0.0)
                ratio, ez = og.error_ratio(got, c64, s64)
                assert ez and ratio <= og.bound(K + beta), (rg.variant_name(v), beta, ratio)
                assert np.array_equal(got, Cw.cpu().numpy()), (rg.variant_name(v), beta)
    finally:
        rg.rg_group_destroy(g)

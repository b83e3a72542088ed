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


@pytest.mark.parametrize("tile", range(6))
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
    g = rg.rg_group_create(ctx, 0, 2)
    try:
        A = torch.zeros((64, 64), device="cuda", dtype=torch.bfloat16)
        C = torch.zeros((64, 64), device="cuda")
        rg.rg_gemm_grouped(g, [])
        with pytest.raises(rg.RGError) as e:
            rg.rg_gemm_grouped(g, [(64, 64, 64, A, 64, A, 64, C, 64)] * 3)
        assert e.value.code == rg.RG_ERR_SHAPE
        with pytest.raises(rg.RGError):
            rg.rg_gemm_grouped(g, [(64, 64, 0, A, 64, A, 64, C, 64)])
        rg.rg_check(ctx)
    finally:
        rg.rg_group_destroy(g)

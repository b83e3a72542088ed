"""rg_gemm_noalloc: the GEMM entry point that allocates no device memory.

It serves callers that must not allocate on their call path (a framework whose
own allocator owns the device memory budget, or code that cannot take the
implicit synchronisation cudaMalloc may cause); its split-K scratch lives in a
fixed device array inside the library.  These tests call it through the C ABI:
its output must equal rg_gemm's (same kernel, same summation order, a context's
allocated workspace) bit for bit and lie within the FP64 oracle's bound, twice
in a row so that the second call starts from the scratch the first one left
behind; rg_noalloc_check must report each call's status; after the set-up call
no further call may change the device's free memory; and launches beyond the
scratch must be refused before anything is enqueued.  The file is named to be
collected last."""
import numpy as np
import pytest

import synthetic
from oracle import gemm as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LIMIT = 16 << 20          # RG_NOALLOC_PARTIAL_BYTES


@pytest.fixture(scope="module")
def rg():
    from paper_2605_29752_gb300 import rg as _rg
    return _rg


def _dev_bf16(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).cuda().view(torch.bfloat16)


def _rg_gemm(rg, M, N, K, A, B, c0, v, beta):
    ctx = rg.rg_init(0)
    try:
        ref = torch.from_numpy(c0).cuda()
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, ref, N, v, beta)
        rg.rg_check(ctx)
        return ref.cpu().numpy()
    finally:
        rg.rg_destroy(ctx)


CASES = [
    ((512, 768, 2048), 7, 0),        # 128x128, split 8
    ((512, 640, 4096), 2, 0),        # 128x64, split 4
    ((300, 200, 328), 21, 0),        # 256x256, split 2, ragged
    ((384, 512, 1024), 14, 1),       # 256x64, split 4, beta = 1
    ((2048, 1536, 1024), 8, 0),      # 128x256, split 1
    ((640, 512, 2048), 33, 0),       # 128x128, stream-K
    ((768, 1024, 2048), 44, 0),      # 256x256 cta_group::2 pair, split 1
    ((520, 512, 2048), 45, 0),       # 256x256 cta_group::2 pair, split 2, ragged M
    ((2048, 1024, 1024), 5, 0),      # 128x128 split 2 on 128 tiles: partials exactly the scratch size
    ((1024, 1024, 2048), 33, 0),     # 128x128 stream-K on 64 tiles, 2 pieces each: half the scratch
    ((768, 1000, 1024), 25, 0),      # 128x192, split 2, ragged N
]


@pytest.mark.parametrize("shape,v,beta", CASES)
def test_matches_rg_gemm_twice(rg, shape, v, beta):
    M, N, K = shape
    a, b = synthetic.operands_bf16(M, N, K, seed=11)
    A, B = _dev_bf16(a), _dev_bf16(b)
    c0 = synthetic.normal_stream_f32(11, 6, M * N).reshape(M, N) if beta else np.zeros((M, N), np.float32)
    ref = _rg_gemm(rg, M, N, K, A, B, c0, v, beta)
    a64, b64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
    c64 = og.gemm_f64(a64, b64) + c0.astype(np.float64)
    s = og.abs_sum(a64, b64) + np.abs(c0.astype(np.float64))
    for call in range(2):
        Cn = torch.from_numpy(c0).cuda()
        assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, Cn, N, v, beta) == rg.RG_OK
        assert rg.rg_noalloc_check() == rg.RG_OK, call
        got = Cn.cpu().numpy()
        assert not np.any(np.isnan(got))
        assert np.array_equal(got, ref), (call, rg.variant_name(v))     # same kernel, same summation order
        ratio, exact_zero = og.error_ratio(got, c64, s)
        assert exact_zero and ratio <= og.bound(K + beta), (call, ratio)


def test_allocates_nothing_after_set_up(rg):
    """Free device memory (cudaMemGetInfo) is the same before and after a second round of calls
    over split-K, stream-K and cta_group::2 variants: nothing on this path allocates."""
    cases = [((512, 768, 2048), 7), ((640, 512, 2048), 33), ((520, 512, 2048), 45), ((1024, 1024, 1024), 4)]
    bufs = []
    for (M, N, K), v in cases:
        a, b = synthetic.operands_bf16(M, N, K, seed=3)
        bufs.append((M, N, K, v, _dev_bf16(a), _dev_bf16(b), torch.zeros((M, N), device="cuda")))
    for M, N, K, v, A, B, C in bufs:                          # the set-up call and each kernel's first launch
        assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, C, N, v, 0) == rg.RG_OK
    assert rg.rg_noalloc_check() == rg.RG_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for M, N, K, v, A, B, C in bufs:
            assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, C, N, v, 0) == rg.RG_OK
        assert rg.rg_noalloc_check() == rg.RG_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_rejects_split_beyond_scratch(rg):
    """Launches whose partials exceed the fixed scratch are refused before anything is enqueued.  The
    scratch's ticket limit (RG_NOALLOC_MAX_TILES tiles, counted per 128-row tile) cannot be reached first:
    a launch with partials has at least 2 slots of at least 32 KiB per tile (128x64), so the 16 MiB of
    partials bound it to 256 tiles (512 counted for cta_group::2), far below 4096."""
    assert 2 * (rg.RG_NOALLOC_PARTIAL_BYTES // (2 * 128 * 64 * 4)) <= rg.RG_NOALLOC_MAX_TILES
    M = N = 4096
    K = 1024
    A = torch.zeros((M, K), device="cuda", dtype=torch.bfloat16)
    B = torch.zeros((K, N), device="cuda", dtype=torch.bfloat16)
    C = torch.full((M, N), 3.0, device="cuda")
    # 128x128 split 8 on 4096^2: 8 * 1024 tiles * 64 KiB of partials, far above the fixed scratch
    assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, C, N, 7, 0) == rg.RG_ERR_SHAPE
    # one tile over the limit: 128x128 split 2 on 2048 x 1152 (144 tiles, 18 MiB of partials)
    assert rg.rg_gemm_noalloc(2048, 1152, K, A, K, B, N, C, N, 5, 0) == rg.RG_ERR_SHAPE
    # cta_group::2 256x256 split 2 on 1280 x 2048: 40 tiles x 2 x 256 KiB = 20 MiB
    assert rg.rg_gemm_noalloc(1280, 2048, K, A, K, B, N, C, N, 45, 0) == rg.RG_ERR_SHAPE
    # stream-K 128x128 on 1792 x 1280 x 2048: 140 tiles, fewer than the SMs, so every tile is
    # shared by at least 2 CTAs: at least 2 x 140 x 64 KiB = 17.5 MiB
    A2 = torch.zeros((1792, 2048), device="cuda", dtype=torch.bfloat16)
    B2 = torch.zeros((2048, 1280), device="cuda", dtype=torch.bfloat16)
    assert rg.rg_gemm_noalloc(1792, 1280, 2048, A2, 2048, B2, 1280, C, N, 33, 0) == rg.RG_ERR_SHAPE
    torch.cuda.synchronize()
    assert torch.all(C == 3.0)                       # nothing was enqueued
    assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, C, N, 4, 0) == rg.RG_OK   # split 1: no limit
    assert rg.rg_noalloc_check() == rg.RG_OK
    assert torch.all(C == 0.0)

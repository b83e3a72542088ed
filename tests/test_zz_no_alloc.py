"""rg_gemm_noalloc: the GEMM entry point that allocates no device memory.

It serves callers that must not allocate on their call path (a framework whose
own allocator owns the device memory budget, or code that cannot take the
implicit synchronisation cudaMalloc may cause); its split-K scratch lives in a
fixed device array inside the library.  These tests call it through the C ABI
and compare it with rg_gemm (which uses a context's allocated workspace) on the
same inputs, twice in a row so that the second call starts from the scratch the
first one left behind.  The file is named to be collected last."""
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


def _dev_bf16(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).cuda().view(torch.bfloat16)


@pytest.mark.parametrize("shape,v,beta", [
    ((512, 768, 2048), 7, 0),        # 128x128, split 8
    ((512, 640, 4096), 2, 0),        # 128x64, split 4
    ((300, 200, 328), 21, 0),        # 256x256, split 2, ragged
    ((384, 512, 1024), 14, 1),       # 256x64, split 4, beta = 1
    ((2048, 1536, 1024), 8, 0),      # 128x256, split 1
    ((640, 512, 2048), 25, 0),       # 128x128, stream-K
    ((768, 1024, 2048), 40, 0),      # 256x256 cta_group::2 pair, split 1
    ((520, 512, 2048), 41, 0),       # 256x256 cta_group::2 pair, split 2, ragged M
])
def test_matches_rg_gemm_twice(rg, shape, v, beta):
    M, N, K = shape
    a, b = synthetic.operands_bf16(M, N, K, seed=11)
    A, B = _dev_bf16(a), _dev_bf16(b)
    c0 = synthetic.normal_stream_f32(11, 6, M * N).reshape(M, N) if beta else np.zeros((M, N), np.float32)
    ctx = rg.rg_init(0)
    try:
        ref = torch.from_numpy(c0).cuda()
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, ref, N, v, beta)
        rg.rg_check(ctx)
        ref = ref.cpu().numpy()
    finally:
        rg.rg_destroy(ctx)
    a64, b64 = og.bf16_bits_to_f64(a), og.bf16_bits_to_f64(b)
    s = og.abs_sum(a64, b64) + np.abs(c0.astype(np.float64))
    for call in range(2):
        Cn = torch.from_numpy(c0).cuda()
        assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, Cn, N, v, beta) == rg.RG_OK
        torch.cuda.synchronize()
        got = Cn.cpu().numpy()
        assert not np.any(np.isnan(got))
        ratio, exact_zero = og.error_ratio(got, ref.astype(np.float64), s)
        assert exact_zero and ratio <= og.bound(K + beta), (call, ratio)


def test_rejects_split_beyond_scratch(rg):
    M = N = 4096
    K = 1024
    A = torch.zeros((M, K), device="cuda", dtype=torch.bfloat16)
    B = torch.zeros((K, N), device="cuda", dtype=torch.bfloat16)
    C = torch.full((M, N), 3.0, device="cuda")
    # 128x128 split 8 on 4096^2: 8 * 1024 tiles * 64 KiB of partials, far above the fixed scratch
    assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, C, N, 7, 0) == rg.RG_ERR_SHAPE
    torch.cuda.synchronize()
    assert torch.all(C == 3.0)                       # nothing was enqueued
    assert rg.rg_gemm_noalloc(M, N, K, A, K, B, N, C, N, 4, 0) == rg.RG_OK   # split 1: no limit
    torch.cuda.synchronize()
    assert torch.all(C == 0.0)

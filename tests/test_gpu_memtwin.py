"""The memory twin of each tile (Sec. 4: the GEMM's loads, pipeline and stores
with the MMAs replaced by no-ops) on the GPU: it runs to completion on ragged
shapes, writes only inside C's logical extent, leaves the real kernel's next
result intact, and its sweep feeds the four-surface decomposition."""
import numpy as np
import pytest

import synthetic
from oracle import decompose as od
from oracle import gemm as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENTINEL = 12345.0


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


@pytest.mark.parametrize("tile", range(8))
@pytest.mark.parametrize("shape", [(300, 264, 200), (128, 64, 64), (520, 776, 1000)])
def test_memtwin_stays_inside_c(rg, ctx, tile, shape):
    M, N, K = shape
    a_bits, b_bits = synthetic.operands_bf16(M, N, K, seed=1)
    A, B = dev_bf16(a_bits), dev_bf16(b_bits)
    ldc = N + 12
    Cbuf = torch.full((M + 3, ldc), SENTINEL, device="cuda", dtype=torch.float32)
    rg.rg_gemm_memtwin(ctx, M, N, K, A, K, B, N, Cbuf, ldc, tile)
    rg.rg_check(ctx)
    c = Cbuf.cpu().numpy()
    assert np.all(c[:, N:] == SENTINEL) and np.all(c[M:, :] == SENTINEL)
    # the real kernel on the same context afterwards is unaffected
    C = torch.full((M, N), float("nan"), device="cuda")
    rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, rg.variant(tile, 1))
    rg.rg_check(ctx)
    a, b = og.bf16_bits_to_f64(a_bits), og.bf16_bits_to_f64(b_bits)
    ratio, exact_zero = og.error_ratio(C.cpu().numpy(), og.gemm_f64(a, b), og.abs_sum(a, b))
    assert exact_zero and ratio <= og.bound(K)


def test_memtwin_rejects_bad_tile(rg, ctx):
    t = torch.zeros(64 * 64, device="cuda")
    with pytest.raises(rg.RGError) as e:
        rg.rg_gemm_memtwin(ctx, 64, 64, 64, t, 64, t, 64, t, 64, rg.RG_NUM_TILES)
    assert e.value.code == rg.RG_ERR_INVALID


def test_memtwin_sweep_and_decomposition(rg, ctx):
    grid = ((256, 256, 3), (256, 256, 3), (512, 512, 2))
    g = rg.make_grid(*grid)
    a_bits, b_bits = synthetic.operands_bf16(768, 768, 1024, seed=0)
    A, B = dev_bf16(a_bits), dev_bf16(b_bits)
    C = torch.zeros(768 * 768, device="cuda")
    opts = rg.rg_sweep_opts_default()
    opts.reps = 2
    tm = rg.rg_sweep_memtwin(ctx, g, [1, 5], A, B, C, opts)
    tg = rg.rg_sweep(ctx, g, [rg.variant(1, 1), rg.variant(5, 1)], A, B, C, opts)
    assert tm.shape == (2, 18) and np.all(tm > 0) and np.all(tm < 10 ** 8)
    for i in range(2):
        comp, over, st = rg.rg_decompose(g, tg[i], tm[i], 1900.7)
        axes = [[a[0] + j * a[1] for j in range(a[2])] for a in grid]
        rc, ro, rs = od.decompose(*axes, tg[i], tm[i], 1900.7)
        assert np.array_equal(comp.reshape(rc.shape), rc) and np.array_equal(st, rs)
        assert 0.0 <= st[0] <= 1.0

"""GPU parity of plan execution (rg_gemm_plan: O(1) lookup, then the cell's
padded / split leaves, Sec. 7.1) and of the sweep (rg_sweep) against the
oracle."""
import numpy as np
import pytest

import synthetic
from oracle import dp, roughness
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


def dev_bf16(bits):
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).cuda().view(torch.bfloat16)


def _plan_with_every_action(rg, shape, seed):
    """A plan over a step-128 grid whose T0 favours splits and padding somewhere."""
    rng = np.random.default_rng(seed)
    vids = [0, 5, 10, 14, 17, 21]
    T0 = rng.integers(50, 5000, size=(len(vids),) + shape).astype(np.int64)
    g = rg.make_grid((128, 128, shape[0]), (128, 128, shape[1]), (128, 128, shape[2]))
    h = rg.rg_plan_build(g, T0.reshape(len(vids), -1), vids)
    ref = dp.plan(T0, ((128, 128, shape[0]), (128, 128, shape[1]), (128, 128, shape[2])))
    # the library's tables are the oracle's, bit for bit, on the build that executes them
    got = rg.rg_plan_tables(h)
    for key in ("T0s", "T1", "target", "T2", "action", "q"):
        assert np.array_equal(got[key], ref[key]), key
    assert np.array_equal(got["vstar"], np.asarray(vids)[ref["vstar"]])
    acts = set(int(a) for a in ref["action"].ravel())
    return h, acts, ref


def _exec(rg, ctx, plan, M, N, K, seed=0):
    a_bits, b_bits = synthetic.operands_bf16(M, N, K, seed=seed)
    A, B = dev_bf16(a_bits), dev_bf16(b_bits)
    C = torch.full((M, N), float("nan"), device="cuda")
    rg.rg_gemm_plan(ctx, plan, M, N, K, A, K, B, N, C, N)
    rg.rg_check(ctx)
    c = C.cpu().numpy()
    ok, ratio = og.check(c, og.bf16_bits_to_f64(a_bits), og.bf16_bits_to_f64(b_bits))
    assert not np.any(np.isnan(c)) and ok, (M, N, K, ratio)
    return c


def test_plan_execution_every_cell(rg, ctx):
    shape = (4, 4, 4)
    h, acts, ref = _plan_with_every_action(rg, shape, seed=0)
    try:
        assert acts >= {0, 1, 2, 3}, acts                 # keep/pad and all three split axes occur
        assert any(tuple(ref["target"][c]) != c for c in np.ndindex(*shape))   # and padding
        for a in range(4):
            for b in range(4):
                for c in range(4):
                    _exec(rg, ctx, h, 128 * (a + 1), 128 * (b + 1), 128 * (c + 1))
    finally:
        rg.rg_plan_free(h)


@pytest.mark.parametrize("shape", [(200, 136, 96), (511, 384, 264), (1, 8, 8), (384, 504, 512)])
def test_plan_execution_off_grid_shapes(rg, ctx, shape):
    h, _, _ = _plan_with_every_action(rg, (4, 4, 4), seed=5)
    try:
        _exec(rg, ctx, h, *shape)
    finally:
        rg.rg_plan_free(h)


def test_plan_execution_k_chain_beta(rg, ctx):
    # a 1 x 1 x 8 grid where K splits win: the plan becomes a chain of beta = 1 leaves
    T0 = np.array([[[100, 10000, 10000, 10000, 10000, 10000, 10000, 10000]]], dtype=np.int64)
    g = rg.make_grid((128, 128, 1), (128, 128, 1), (128, 128, 8))
    h = rg.rg_plan_build(g, T0.reshape(1, -1), [5])
    try:
        leaves, t2 = rg.rg_plan_lookup(h, 128, 128, 1024)
        assert len(leaves) == 8 and [l[1] for l in leaves] == [0] + [1] * 7 and t2 == 800
        _exec(rg, ctx, h, 128, 128, 1024)
        _exec(rg, ctx, h, 100, 72, 1000)
    finally:
        rg.rg_plan_free(h)


def test_sweep_tiny_grid_and_plan_sweep(rg, ctx):
    g = rg.make_grid((128, 128, 3))
    Mx = 384
    a_bits, b_bits = synthetic.operands_bf16(Mx, Mx, Mx)
    A = dev_bf16(synthetic.bf16_uniform_stream(0, synthetic.TAG_A, Mx * Mx))
    B = dev_bf16(synthetic.bf16_uniform_stream(0, synthetic.TAG_B, Mx * Mx))
    C = torch.zeros(Mx * Mx, device="cuda")
    vids = [rg.variant(1, 1), rg.variant(2, 2)]
    opts = rg.rg_sweep_opts_default()
    opts.prune_splits = 0
    t = rg.rg_sweep(ctx, g, vids, A, B, C, opts)
    assert t.shape == (2, 27) and np.all(t > 0) and np.all(t < 10**8)
    opts.prune_splits = 1
    tp = rg.rg_sweep(ctx, g, vids, A, B, C, opts)
    assert np.all(tp[0] < 10**8)                       # split 1 is always timed
    Ks = np.tile(np.array([128, 256, 384]), 9)
    assert np.all(tp[1][Ks < 256] == rg.RG_T_UNMEASURED)   # fewer than 2 K blocks per split
    assert np.all(tp[1][Ks >= 256] < 10**8)                # few tiles: the split variant is timed
    # the surfaces and statistics the sweep returns are the oracle's, bit for bit, from its times
    t2, tf2, st2 = rg.rg_sweep_surfaces(ctx, g, vids, A, B, C, opts)
    ogrid = ((128, 128, 3),) * 3
    for row in range(2):
        if np.any(t2[row] == rg.RG_T_UNMEASURED):
            measured = t2[row] != rg.RG_T_UNMEASURED
            assert np.all(np.isnan(st2[row])) and np.all(tf2[row][~measured] == 0.0)
            S = roughness.surface(np.where(measured, t2[row], 1).reshape(3, 3, 3), ogrid).ravel()
            assert np.array_equal(tf2[row][measured], S[measured])
            continue
        S = roughness.surface(t2[row].reshape(3, 3, 3), ogrid)
        ref = roughness.roughness_all(S)
        assert np.array_equal(tf2[row], S.ravel())
        assert [st2[row][i] for i in range(5)] == [ref[k] for k in ("R_M", "R_N", "R_K", "R_3D", "R_N_slice")]
        assert st2[row][5] == roughness.mean(S)
    plan = rg.rg_plan_build(g, t, vids)
    try:
        tp, tfp, stp = rg.rg_sweep_surfaces(ctx, g, [0], A, B, C, opts, plan=plan)
        assert tp.shape == (1, 27) and np.all(tp > 0)
        S = roughness.surface(tp[0].reshape(3, 3, 3), ogrid)
        assert np.array_equal(tfp[0], S.ravel()) and stp[0][5] == roughness.mean(S)
        # the last swept cell's C is the plan's result for 384^3 only if it ran last;
        # run it explicitly and check it
        _exec(rg, ctx, plan, 384, 384, 384)
        tf, r, mean = rg.rg_surface_stats(g, tp[0])
        assert mean > 0 and all(v >= 0 for v in r.values())
    finally:
        rg.rg_plan_free(plan)
    n0 = rg.rg_launch_count(ctx)
    rg.rg_gemm(ctx, 128, 128, 128, A, 128, B, 128, C, 128, 1)
    assert rg.rg_launch_count(ctx) == n0 + 1


def test_timeout_path_returns_error_and_context_recovers(rg, ctx):
    """With the test stall on, the MMA warp waits on a barrier nothing arrives on;
    its bounded wait (here about a millisecond) must expire, the kernel must
    record the error, let its copies land, release TMEM and return, and the next
    launch without the stall must compute the right result."""
    M = N = K = 1024
    a_bits, b_bits = synthetic.operands_bf16(M, N, K, seed=9)
    A, B = dev_bf16(a_bits), dev_bf16(b_bits)
    C = torch.zeros((M, N), device="cuda")
    rg.rg_set_timeout_cycles(ctx, 2_000_000)
    rg.rg_set_test_stall(ctx, True)
    try:
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, rg.variant(1, 2))
        status = rg.rg_check_status(ctx)
    finally:
        rg.rg_set_test_stall(ctx, False)
        rg.rg_set_timeout_cycles(ctx, 2_000_000_000)
    assert status == rg.RG_ERR_TIMEOUT
    assert rg.rg_check_status(ctx) == rg.RG_OK          # the error word was cleared
    C.fill_(float("nan"))
    rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, rg.variant(1, 2))
    rg.rg_check(ctx)
    ok, _ = og.check(C.cpu().numpy(), og.bf16_bits_to_f64(a_bits), og.bf16_bits_to_f64(b_bits))
    assert ok


@pytest.mark.parametrize("shape", [(384, 512, 256), (200, 136, 100), (511, 384, 264)])
def test_plan_host_buffers(rg, ctx, shape):
    """rg_gemm_plan_host: host operands (numpy, unaligned leading dimensions allowed) are copied
    in, the plan runs, C is copied back before the call returns; the result is the device
    path's bit for bit and within the oracle's bound."""
    M, N, K = shape
    h, _, _ = _plan_with_every_action(rg, (4, 4, 4), seed=5)
    try:
        a_bits, b_bits = synthetic.operands_bf16(M, N, K, seed=31)
        a_h = np.ascontiguousarray(a_bits.view(np.uint16))
        b_h = np.ascontiguousarray(b_bits.view(np.uint16))
        c_h = np.full((M, N), np.nan, np.float32)
        rg.rg_gemm_plan_host(ctx, h, M, N, K, a_h, K, b_h, N, c_h, N)
        ok, ratio = og.check(c_h, og.bf16_bits_to_f64(a_bits), og.bf16_bits_to_f64(b_bits))
        assert ok and not np.any(np.isnan(c_h)), ratio
        # the device path on aligned copies of the same operands
        la, lb = (K + 7) // 8 * 8, (N + 7) // 8 * 8
        a_pad = np.zeros((M, la), np.uint16)
        a_pad[:, :K] = a_h
        b_pad = np.zeros((K, lb), np.uint16)
        b_pad[:, :N] = b_h
        A, B = dev_bf16(a_pad), dev_bf16(b_pad)
        C = torch.full((M, lb), float("nan"), device="cuda")
        rg.rg_gemm_plan(ctx, h, M, N, K, A, la, B, lb, C, lb)
        rg.rg_check(ctx)
        assert np.array_equal(C.cpu().numpy()[:, :N], c_h)
    finally:
        rg.rg_plan_free(h)


def test_sharded_sweep_partitions_the_items(rg, ctx):
    """Two shards of one sweep (the same seed) time disjoint sets of (variant, cell) items that together
    cover every item the pruning keeps; pruned items are marked on both."""
    g = rg.make_grid((128, 128, 3))
    Mx = 384
    A = dev_bf16(synthetic.bf16_uniform_stream(0, synthetic.TAG_A, Mx * Mx))
    B = dev_bf16(synthetic.bf16_uniform_stream(0, synthetic.TAG_B, Mx * Mx))
    C = torch.zeros(Mx * Mx, device="cuda")
    vids = [rg.variant(1, 1), rg.variant(2, 2), rg.variant(0, 4)]
    full = rg.rg_sweep(ctx, g, vids, A, B, C)
    parts = []
    for i in range(2):
        o = rg.rg_sweep_opts_default()
        o.shard_index, o.shard_count = i, 2
        parts.append(rg.rg_sweep(ctx, g, vids, A, B, C, o))
    pruned = full == rg.RG_T_UNMEASURED
    assert np.all((parts[0] == rg.RG_T_UNMEASURED) == pruned) and np.all((parts[1] == rg.RG_T_UNMEASURED) == pruned)
    mine = [(p != rg.RG_T_OTHER_SHARD) & ~pruned for p in parts]
    assert not np.any(mine[0] & mine[1]) and np.all(mine[0] | mine[1] | pruned)
    assert abs(int(mine[0].sum()) - int(mine[1].sum())) <= 1            # balanced
    o = rg.rg_sweep_opts_default()
    o.shard_index, o.shard_count = 2, 2
    with pytest.raises(rg.RGError):
        rg.rg_sweep(ctx, g, vids, A, B, C, o)

"""GPU tests of the serving loop (rg_serve): every served request against the
oracle, results the same alone and in the mix (bitwise: each output tile is
computed by the same code in the same order), admission by the HBM budget,
and batches formed while others run."""
import numpy as np
import pytest

import synthetic
from oracle import gemm as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MX = 1024


@pytest.fixture(scope="module")
def rg():
    from paper_2605_29752_gb300 import rg as _rg
    return _rg


@pytest.fixture(scope="module")
def ctx(rg):
    h = rg.rg_init(0)
    yield h
    rg.rg_destroy(h)


@pytest.fixture(scope="module")
def streams():
    a = synthetic.bf16_uniform_stream(0, synthetic.TAG_A, MX * MX)
    b = synthetic.bf16_uniform_stream(0, synthetic.TAG_B, MX * MX)
    A = torch.from_numpy(a.view(np.int16)).cuda().view(torch.bfloat16)
    B = torch.from_numpy(b.view(np.int16)).cuda().view(torch.bfloat16)
    return a, b, A, B


def _trace(n, rate, seed, counts=(8, 8, 8)):
    cells = synthetic.uniform_cells(n, counts, seed=seed)
    t = synthetic.poisson_arrivals(rate, n, seed=seed)
    return [((int(a) + 1) * 128, (int(b) + 1) * 128, (int(c) + 1) * 128, int(ti)) for (a, b, c), ti in zip(cells, t)]


def _requests(trace, A, B, outs):
    return [(M, N, K, A, K, B, N, outs[i], N, t) for i, (M, N, K, t) in enumerate(trace)]


def test_serving_results_match_oracle_and_alone(rg, ctx, streams):
    a_bits, b_bits, A, B = streams
    trace = _trace(120, 20000.0, seed=3)
    outs = [torch.full((M, N), float("nan"), device="cuda") for M, N, K, _ in trace]
    opts = rg.rg_serve_opts_default()
    opts.max_batch = 16
    opts.max_inflight = 3
    res, st = rg.rg_serve(ctx, None, opts, _requests(trace, A, B, outs))
    rg.rg_check(ctx)
    assert st["requests"] == len(trace) and all(r["status"] == 0 for r in res)
    assert st["batches"] >= len(trace) // 16
    assert st["p99_latency_us"] >= st["p50_latency_us"] > 0
    for r, (M, N, K, t) in zip(res, trace):
        assert t <= r["admitted_ns"] <= r["launched_ns"] <= r["done_ns"]
    # overlap: some batch was launched before the previous one had completed
    by_batch = {}
    for r in res:
        by_batch.setdefault(r["batch"], r)
    order = sorted(by_batch.values(), key=lambda r: r["launched_ns"])
    assert any(order[i + 1]["launched_ns"] < order[i]["done_ns"] for i in range(len(order) - 1))
    for i, (M, N, K, _) in enumerate(trace):
        a = og.bf16_bits_to_f64(a_bits[:M * K].reshape(M, K))
        b = og.bf16_bits_to_f64(b_bits[:K * N].reshape(K, N))
        ok, ratio = og.check(outs[i].cpu().numpy(), a, b)
        assert ok, (i, ratio)
    # the same requests alone give the same bits
    for i in range(0, len(trace), 17):
        M, N, K, _ = trace[i]
        alone = torch.full((M, N), float("nan"), device="cuda")
        r1, _ = rg.rg_serve(ctx, None, opts, [(M, N, K, A, K, B, N, alone, N, 0)])
        assert r1[0]["status"] == 0
        assert torch.equal(alone, outs[i])


def test_serving_with_plan_lookup_padding(rg, ctx, streams):
    a_bits, b_bits, A, B = streams
    g = rg.make_grid((128, 128, 8))
    # a pad-only plan whose table makes every cell pad one step in N where it can
    T0 = np.zeros((8, 8, 8), np.int64)
    for i in range(8):
        for j in range(8):
            for k in range(8):
                T0[i, j, k] = 1000 + (i + 1) * (k + 1) * (10 if j % 2 == 0 else 1)
    plan = rg.rg_plan_build_ex(g, T0.reshape(1, -1), [rg.variant(1, 1)], rg.RG_PLAN_PAD_ONLY)
    try:
        trace = _trace(40, 50000.0, seed=5)
        outs = [torch.full((M, N), float("nan"), device="cuda") for M, N, K, _ in trace]
        opts = rg.rg_serve_opts_default()
        res, st = rg.rg_serve(ctx, plan, opts, _requests(trace, A, B, outs))
        rg.rg_check(ctx)
        assert all(r["status"] == 0 for r in res)
        for i, (M, N, K, _) in enumerate(trace):
            a = og.bf16_bits_to_f64(a_bits[:M * K].reshape(M, K))
            b = og.bf16_bits_to_f64(b_bits[:K * N].reshape(K, N))
            ok, ratio = og.check(outs[i].cpu().numpy(), a, b)
            assert ok, (i, ratio)
    finally:
        rg.rg_plan_free(plan)


def test_admission_budget(rg, ctx, streams):
    _, _, A, B = streams
    big = (1024, 1024, 1024)
    need = 2 * 1024 * 1024 * 2 + 4 * 1024 * 1024          # bytes of one 1024^3 request
    opts = rg.rg_serve_opts_default()
    opts.hbm_budget_bytes = need + need // 2                # one request at a time
    opts.max_batch = 8
    outs = [torch.zeros(big[:2], device="cuda") for _ in range(6)]
    reqs = [(*big, A, 1024, B, 1024, outs[i], 1024, 0) for i in range(6)]
    res, st = rg.rg_serve(ctx, None, opts, reqs)
    assert all(r["status"] == 0 for r in res)
    assert st["batches"] == 6 and st["admission_stalls"] >= 1      # budget forced one request per batch
    # a request that can never fit is rejected, the others still run
    opts.hbm_budget_bytes = need - 1
    small = torch.zeros((128, 128), device="cuda")
    res, st = rg.rg_serve(ctx, None, opts, [(*big, A, 1024, B, 1024, outs[0], 1024, 0),
                                            (128, 128, 128, A, 128, B, 128, small, 128, 10)])
    assert res[0]["status"] == rg.RG_ERR_ADMISSION and res[1]["status"] == 0
    # arena outputs (C = None) for a load test
    opts = rg.rg_serve_opts_default()
    opts.hbm_budget_bytes = 1 << 30
    trace = _trace(200, 100000.0, seed=9)
    res, st = rg.rg_serve(ctx, None, opts, [(M, N, K, A, K, B, N, None, N, t) for M, N, K, t in trace])
    rg.rg_check(ctx)
    assert st["requests"] == 200 and st["tflops"] > 0


def test_malformed_requests_are_rejected_alone(rg, ctx, streams):
    """rg_gemm's checks run at admission: a misaligned, an undersized and a negative request
    each get their own status while the well-formed requests around them are served."""
    _, _, A, B = streams
    opts = rg.rg_serve_opts_default()
    opts.hbm_budget_bytes = 1 << 30
    outs = [torch.full((256, 256), float("nan"), device="cuda") for _ in range(2)]
    bad_c = torch.zeros(256 * 256 + 4, device="cuda")
    reqs = [(256, 256, 256, A, 256, B, 256, outs[0], 256, 0),
            (256, 256, 256, A, 252, B, 256, bad_c, 256, 0),             # lda < K
            (256, 256, 256, A, 256, B, 256, bad_c[1:], 256, 0),          # C not 16-byte aligned
            (-1, 256, 256, A, 256, B, 256, bad_c, 256, 0),               # negative size
            (256, 256, 256, A, 256, B, 256, outs[1], 256, 0)]
    res, st = rg.rg_serve(ctx, None, opts, reqs)
    rg.rg_check(ctx)
    assert [r["status"] for r in res] == [0, rg.RG_ERR_INVALID, rg.RG_ERR_ALIGN, rg.RG_ERR_INVALID, 0]
    assert st["requests"] == 2
    assert not torch.isnan(outs[0]).any() and torch.equal(outs[0], outs[1])


def test_serving_routes_each_request_to_its_autotuned_tile(rg, ctx, streams):
    """A plan whose best tile differs from cell to cell (a synthetic T0 table over all six split-1
    tiles): each batch runs one grouped launch per tile present, and every result matches the
    oracle and, bitwise, rg_gemm with that cell's tile and padding."""
    a_bits, b_bits, A, B = streams
    g = rg.make_grid((128, 128, 8))
    rows = [rg.variant(t, 1) for t in range(6)]
    rs = np.random.default_rng(17)
    T0 = rs.integers(1000, 100000, size=(6, 8 * 8 * 8)).astype(np.int64)
    plan = rg.rg_plan_build_ex(g, T0, rows, rg.RG_PLAN_PAD_ONLY)
    try:
        trace = _trace(60, 50000.0, seed=6)
        outs = [torch.full((M, N), float("nan"), device="cuda") for M, N, K, _ in trace]
        opts = rg.rg_serve_opts_default()
        opts.max_batch = 16
        res, st = rg.rg_serve(ctx, plan, opts, _requests(trace, A, B, outs))
        rg.rg_check(ctx)
        assert all(r["status"] == 0 for r in res)
        tiles_used = set()
        for i, (M, N, K, _) in enumerate(trace):
            a = og.bf16_bits_to_f64(a_bits[:M * K].reshape(M, K))
            b = og.bf16_bits_to_f64(b_bits[:K * N].reshape(K, N))
            ok, ratio = og.check(outs[i].cpu().numpy(), a, b)
            assert ok, (i, ratio)
            leaves, _ = rg.rg_plan_lookup(plan, M, N, K)
            v, pm, pn, pk = leaves[0][0], leaves[0][9], leaves[0][10], leaves[0][11]
            tiles_used.add(rg.variant_tile(v))
            ref = torch.full((M, N), float("nan"), device="cuda")
            rg.rg_gemm(ctx, M, N, K, A, K, B, N, ref, N, rg.variant(rg.variant_tile(v), 1), 0,
                       max(pm, M), max(pn, N), max(pk, K))
            rg.rg_check(ctx)
            assert torch.equal(ref, outs[i]), i
        assert len(tiles_used) >= 3
    finally:
        rg.rg_plan_free(plan)

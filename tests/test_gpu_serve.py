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


def _full_plan(rg, seed, vids):
    """A plan over the 8^3 grid from a synthetic T0 table whose DP uses every action (padding,
    splits along M, N and K) and many kernel variants."""
    g = rg.make_grid((128, 128, 8))
    rs = np.random.default_rng(seed)
    s = (np.arange(8) + 1) * 128.0
    base = 50.0 + 2.0 * s[:, None, None] * s[None, :, None] * s[None, None, :] / 4e5   # a small fixed cost
    T0 = np.stack([np.round(base * rs.uniform(0.6, 1.6, size=(8, 8, 8))) for _ in vids]).astype(np.int64)
    plan = rg.rg_plan_build(g, T0.reshape(len(vids), -1), vids)
    acts = set(rg.rg_plan_tables(plan)["action"].ravel().tolist())
    assert acts >= {0, 1, 2, 3}, acts
    return plan


def _full_vids(rg):
    return [rg.variant(0, 2), rg.variant(1, 1), rg.variant(1, 4), rg.variant(2, 1), rg.variant(3, 2),
            rg.variant(4, 1), rg.variant(5, 8), rg.variant(1, rg.SK), rg.variant(4, (rg.TWO_SM, 2)),
            rg.variant(5, rg.TWO_SM), rg.variant(5, rg.TWO_SM_SK)]


def test_serving_through_the_full_plan(rg, ctx, streams):
    """Requests routed through a full plan (padding, M/N/K splits with phase-ordered beta = 1
    pieces, split-K and cta_group::2 variants): every result within the oracle's bound, the same
    bits alone as in the mix, and the same bits as rg_gemm_plan wherever no leaf is a stream-K
    choice (the grouped launch runs those as their tile with split 1)."""
    a_bits, b_bits, A, B = streams
    plan = _full_plan(rg, 0, _full_vids(rg))
    try:
        trace = _trace(90, 40000.0, seed=12)
        trace += [(200, 136, 1000, trace[-1][3] + 1000), (1000, 904, 520, trace[-1][3] + 2000)]   # off-grid
        outs = [torch.full((M, N), float("nan"), device="cuda") for M, N, K, _ in trace]
        opts = rg.rg_serve_opts_default()
        opts.max_batch = 12
        opts.max_inflight = 3
        res, st = rg.rg_serve(ctx, plan, opts, _requests(trace, A, B, outs))
        rg.rg_check(ctx)
        assert all(r["status"] == 0 for r in res) and st["requests"] == len(trace)
        multi = 0
        for i, (M, N, K, _) in enumerate(trace):
            a = og.bf16_bits_to_f64(a_bits[:M * K].reshape(M, K))
            b = og.bf16_bits_to_f64(b_bits[:K * N].reshape(K, N))
            ok, ratio = og.check(outs[i].cpu().numpy(), a, b)
            assert ok, (i, ratio)
            leaves, _ = rg.rg_plan_lookup(plan, M, N, K)
            multi += len(leaves) > 1
            if not any(rg.variant_name(l[0]).endswith("SK") for l in leaves):
                ref = torch.full((M, N), float("nan"), device="cuda")
                rg.rg_gemm_plan(ctx, plan, M, N, K, A, K, B, N, ref, N)
                rg.rg_check(ctx)
                assert torch.equal(ref, outs[i]), (i, leaves)
        assert multi >= 10
        for i in range(0, len(trace), 7):                      # alone
            M, N, K, _ = trace[i]
            alone = torch.full((M, N), float("nan"), device="cuda")
            r1, _ = rg.rg_serve(ctx, plan, opts, [(M, N, K, A, K, B, N, alone, N, 0)])
            assert r1[0]["status"] == 0
            assert torch.equal(alone, outs[i]), i
    finally:
        rg.rg_plan_free(plan)


def test_online_server_submit_poll_wait_stop(rg, ctx, streams):
    """The online entry points: requests submitted from two host threads while earlier ones run,
    polled and waited for; every result is bitwise the trace replay's for the same plan."""
    import threading
    a_bits, b_bits, A, B = streams
    plan = _full_plan(rg, 3, _full_vids(rg))
    try:
        trace = _trace(60, 1.0, seed=14)
        opts = rg.rg_serve_opts_default()
        opts.max_batch = 8
        ref = [torch.full((M, N), float("nan"), device="cuda") for M, N, K, _ in trace]
        rg.rg_serve(ctx, plan, opts, [(M, N, K, A, K, B, N, ref[i], N, 0) for i, (M, N, K, _) in enumerate(trace)])
        rg.rg_check(ctx)
        outs = [torch.full((M, N), float("nan"), device="cuda") for M, N, K, _ in trace]
        torch.cuda.synchronize()
        srv = rg.rg_serve_start(ctx, plan, opts)
        ids = {}
        try:
            def submit(part):
                for i in part:
                    M, N, K, _ = trace[i]
                    ids[i] = rg.rg_serve_submit(srv, M, N, K, A, K, B, N, outs[i], N)
            threads = [threading.Thread(target=submit, args=(range(j, len(trace), 2),)) for j in range(2)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            assert sorted(ids.values()) == list(range(len(trace)))
            done = 0
            for i in range(len(trace)):
                r = rg.rg_serve_poll(srv, ids[i])
                if r is None:
                    r = rg.rg_serve_wait(srv, ids[i])
                assert r["status"] == 0 and r["done_ns"] >= r["admitted_ns"] >= 0
                done += 1
        finally:
            st = rg.rg_serve_stop(srv)
        assert done == len(trace) and st["requests"] == len(trace)
        assert st["p99_latency_us"] >= st["p50_latency_us"] > 0
        for i in range(len(trace)):
            assert torch.equal(outs[i], ref[i]), i
        with pytest.raises(rg.RGError):
            rg.rg_serve_poll(None, 0)                           # a null server is refused
    finally:
        rg.rg_plan_free(plan)


def test_serving_mixed_bf16_and_fp8_requests(rg, ctx, streams):
    """FP8 requests (top-left blocks of one block-quantised 1024 x 1024 pair, whole scale arrays)
    interleaved with BF16 ones: each FP8 result is bitwise rg_gemm_fp8_plan's with the same FP8 plan
    and within the FP8 bound of the dequantised float64 product; the BF16 ones are unchanged by
    the mix; every request gives the same bits alone."""
    from oracle import fp8 as of
    a_bits, b_bits, A, B = streams
    plan = _full_plan(rg, 0, _full_vids(rg))
    g = rg.make_grid((128, 128, 8))
    fvids = [rg.fp8_variant(t, s) for t in range(2) for s in rg.SPLITS]
    rs = np.random.default_rng(5)
    s8 = (np.arange(8) + 1) * 128.0
    base = 50.0 + 2.0 * s8[:, None, None] * s8[None, :, None] * s8[None, None, :] / 8e5
    T0 = np.stack([np.round(base * rs.uniform(0.6, 1.6, size=(8, 8, 8))) for _ in fvids]).astype(np.int64)
    fplan = rg.rg_plan_build(g, T0.reshape(len(fvids), -1), fvids)
    try:
        xa = torch.from_numpy(synthetic.normal_stream_f32(0, 1, MX * MX)).cuda()
        xb = torch.from_numpy(synthetic.normal_stream_f32(0, 2, MX * MX)).cuda()
        qa = torch.empty(MX * MX, dtype=torch.uint8, device="cuda")
        qb = torch.empty(MX * MX, dtype=torch.uint8, device="cuda")
        nb = MX // 128
        sa = torch.empty(nb * nb, device="cuda")
        sb = torch.empty(nb * nb, device="cuda")
        rg.rg_fp8_quantize(ctx, xa, MX, MX, MX, qa, MX, sa)
        rg.rg_fp8_quantize(ctx, xb, MX, MX, MX, qb, MX, sb)
        rg.rg_check(ctx)
        Ad = of.dequantize(qa.cpu().numpy().reshape(MX, MX), sa.cpu().numpy().reshape(nb, nb))
        Bd = of.dequantize(qb.cpu().numpy().reshape(MX, MX), sb.cpu().numpy().reshape(nb, nb))
        trace = _trace(70, 40000.0, seed=21)
        reqs, outs, is8 = [], [], []
        for i, (M, N, K, t) in enumerate(trace):
            C = torch.full((M, N), float("nan"), device="cuda")
            outs.append(C)
            if i % 2:
                reqs.append((M, N, K, qa, MX, qb, MX, C, N, t, (sa, nb, sb, nb)))
            else:
                reqs.append((M, N, K, A, K, B, N, C, N, t))
            is8.append(bool(i % 2))
        opts = rg.rg_serve_opts_default()
        opts.max_batch = 10
        opts.fp8_plan = fplan
        res, st = rg.rg_serve(ctx, plan, opts, reqs)
        rg.rg_check(ctx)
        assert all(r["status"] == 0 for r in res) and st["requests"] == len(trace)
        for i, (M, N, K, _) in enumerate(trace):
            got = outs[i].cpu().numpy()
            if is8[i]:
                ref = torch.full((M, N), float("nan"), device="cuda")
                rg.rg_gemm_fp8_plan(ctx, fplan, M, N, K, qa, MX, sa, nb, qb, MX, sb, nb, ref, N)
                rg.rg_check(ctx)
                assert np.array_equal(ref.cpu().numpy(), got), i
                a, b = Ad[:M, :K], Bd[:K, :N]
                ratio, ez = og.error_ratio(got, a @ b, np.abs(a) @ np.abs(b))
                assert ez and ratio <= 4.0 * K * 2.0 ** -24, (i, ratio)
            else:
                ref = torch.full((M, N), float("nan"), device="cuda")
                rg.rg_gemm_plan(ctx, plan, M, N, K, A, K, B, N, ref, N)
                rg.rg_check(ctx)
                leaves, _ = rg.rg_plan_lookup(plan, M, N, K)
                if not any(rg.variant_name(l[0]).endswith("SK") for l in leaves):
                    assert np.array_equal(ref.cpu().numpy(), got), i
        for i in range(0, len(trace), 9):                     # alone
            alone = torch.full_like(outs[i], float("nan"))
            r = list(reqs[i])
            r[7], r[9] = alone, 0
            r1, _ = rg.rg_serve(ctx, plan, opts, [tuple(r)])
            assert r1[0]["status"] == 0 and torch.equal(alone, outs[i]), i
        # an FP8 request beyond the FP8 plan's grid fails alone
        big = torch.zeros((1152, 128), device="cuda")
        qbig = torch.zeros(1152 * 128, dtype=torch.uint8, device="cuda")    # in bounds even if it ran
        sbig = torch.ones(9, device="cuda")
        r2, _ = rg.rg_serve(ctx, plan, opts, [(1152, 128, 128, qbig, 128, qbig, 128, big, 128, 0, (sbig, 1, sbig, 1)),
                                              reqs[0][:7] + (outs[0], reqs[0][8], 0)])
        assert r2[0]["status"] == rg.RG_ERR_SHAPE and r2[1]["status"] == 0
    finally:
        rg.rg_plan_free(fplan)
        rg.rg_plan_free(plan)

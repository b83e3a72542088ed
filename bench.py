#!/usr/bin/env python
"""Benchmark: mean TFLOP/s and roughness of the BF16 NN GEMM landscape over
the 32,768-cell grid (M, N, K) in {128, ..., 4096}^3, plain fixed tile versus
the smoothed stack (autotuned best-of tiles and split factors + the DP
padding/splitting plan, O(1) lookup, fused execution), on one GB300.

Setup (not timed, "offline once per hardware/software stack"): the autotune
sweep times all 38 kernel variants (6 tiles x {split-K 1/2/4/8, stream-K}, and
the two 256-row tiles as tcgen05 cta_group::2 pairs with split-K 1/2/4/8) on
every cell, with the library's pruning, and builds the plan tables.  One timed step re-measures, for every cell, the
plain fixed 128x128 tile and the smoothed plan with the paper's protocol (one
warm-up launch, then the mean of 5 back-to-back launches between CUDA events),
then computes both surfaces' mean and roughness in the library.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "mean TFLOP/s & roughness on 32,768-shape BF16 sweep, plain vs smoothed; p50/p99"
STEP = 128
COUNT = 32
FIXED_TILE = 1          # 128 x 128, the single fixed tile of the small-sweep configuration


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--count", type=int, default=COUNT, help="grid points per axis (32 = the full grid)")
    p.add_argument("--no-extras", action="store_true", help="skip the ladder / cross-tile / e2e / CPU sections")
    p.add_argument("--out", default=None, help="also write the JSON line (and surfaces) here")
    p.add_argument("--clock-log", default=None,
                   help="CSV file for the nvidia-smi clock samples of the timed region (default: a temp file)")
    p.add_argument("--shape", type=int, nargs=3, default=None, metavar=("M", "N", "K"),
                   help="time one GEMM shape with --variant instead of the landscape (profiling aid)")
    p.add_argument("--variant", default="256x256/S1",
                   help="variant for --shape, e.g. 128x256/S1, or an FP8 variant such as 'fp8 128x256/S1'")
    p.add_argument("--reps", type=int, default=20, help="timed launches for --shape")
    p.add_argument("--phase-timers", action="store_true",
                   help="with --shape: load the phase-timer build (librg_timers.so, built with "
                        "`python -m paper_2605_29752_gb300.build --phase-timers`) and report per-CTA phase times")
    return p.parse_args()


def phase_summary(rec):
    """Medians over CTAs of each phase of one traced launch, in ns (SM-clock stamps converted with each
    CTA's own globaltimer / clock ratio); a phase's median is taken over the CTAs that reached both of
    its stamps (the odd CTA of a cta_group::2 pair issues no MMAs, only some CTAs run a fixup)."""
    rec = rec.astype(np.float64)
    f = {n: i for i, n in enumerate(("gt_entry", "gt_exit", "exit", "dep_wait", "first_stage", "last_mma_commit",
                                     "first_acc_ready", "epilogue_done", "fixup_start", "fixup_end", "units"))}
    rec = rec[rec[:, f["exit"]] > 0]
    ns_per_cycle = (rec[:, f["gt_exit"]] - rec[:, f["gt_entry"]]) / rec[:, f["exit"]]

    def span(a, b):
        sel = (rec[:, f[b]] > 0) & ((rec[:, f[a]] > 0) if a != "entry" else True)
        start = rec[sel, f[a]] if a != "entry" else 0.0
        x = (rec[sel, f[b]] - start) * ns_per_cycle[sel]
        return (float(np.median(x)), int(sel.sum())) if sel.any() else (None, 0)
    out = {"ctas": int(len(rec)), "units_per_cta": float(np.median(rec[:, f["units"]])),
           "launch_span_ns": float(rec[:, f["gt_exit"]].max() - rec[:, f["gt_entry"]].min())}
    # launch-level: when the CTAs passed the dependency wait (on the global clock) and when they exited
    rel = rec[:, f["gt_entry"]] + rec[:, f["dep_wait"]] * ns_per_cycle
    out["release_skew_ns"] = float(rel.max() - rel.min())
    out["first_release_to_last_exit_ns"] = float(rec[:, f["gt_exit"]].max() - rel.min())
    out["exit_skew_ns"] = float(rec[:, f["gt_exit"]].max() - rec[:, f["gt_exit"]].min())
    for name, a, b in (("entry_to_dep_wait", "entry", "dep_wait"), ("dep_wait_to_first_stage", "dep_wait", "first_stage"),
                       ("first_stage_to_last_mma_commit", "first_stage", "last_mma_commit"),
                       ("last_mma_commit_to_epilogue_done", "last_mma_commit", "epilogue_done"),
                       ("first_acc_ready_to_epilogue_done", "first_acc_ready", "epilogue_done"),
                       ("dep_wait_to_epilogue_done", "dep_wait", "epilogue_done"),
                       ("fixup", "fixup_start", "fixup_end"), ("cta_total", "entry", "exit")):
        v, n = span(a, b)
        out[name + "_ns"] = v
        out[name + "_ctas"] = n
    return out


def single_shape_fp8(args, rg, torch):
    """One FP8 GEMM configuration (N(0,1) operands block-quantised on the GPU): `reps` back-to-back
    launches between CUDA events."""
    M, N, K = args.shape
    names = {rg.fp8_variant_name(v): v for v in range(rg.RG_FP8_VARIANT_BASE,
                                                        rg.RG_FP8_VARIANT_BASE + rg.RG_FP8_NUM_VARIANTS)}
    v = names[args.variant]
    ctx = rg.rg_init(0)
    xa = torch.from_numpy(synthetic.normal_stream_f32(0, synthetic.TAG_A, M * K)).cuda()
    xb = torch.from_numpy(synthetic.normal_stream_f32(0, synthetic.TAG_B, K * N)).cuda()
    qa = torch.empty(M * K, dtype=torch.uint8, device="cuda")
    qb = torch.empty(K * N, dtype=torch.uint8, device="cuda")
    sa = torch.empty(-(-M // 128) * -(-K // 128), device="cuda")
    sb = torch.empty(-(-K // 128) * -(-N // 128), device="cuda")
    rg.rg_fp8_quantize(ctx, xa, M, K, K, qa, K, sa)
    rg.rg_fp8_quantize(ctx, xb, K, N, N, qb, N, sb)
    C = torch.zeros((M, N), device="cuda")

    def once():
        rg.rg_gemm_fp8_ex(ctx, M, N, K, qa, K, sa, -(-K // 128), qb, N, sb, -(-N // 128), C, N, v)
    for _ in range(3):
        once()
    rg.rg_check(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    rg.rg_check(ctx)
    rg.rg_destroy(ctx)
    us = e0.elapsed_time(e1) / args.reps * 1e3
    print(json.dumps({"shape": [M, N, K], "variant": args.variant, "us_per_launch": us,
                      "tflops": 2.0 * M * N * K / (us * 1e-6) / 1e12, "algorithmic_bytes": M * K + K * N + 4 * M * N,
                      "algorithmic_flops": 2 * M * N * K}), flush=True)
    return 0


def single_shape(args):
    """Time one GEMM configuration: `reps` back-to-back launches under the landscape's protocol (and a
    Python loop of rg_gemm calls, which also times the host), and, with --phase-timers, the last of
    five back-to-back launches of the phase-timer build."""
    if args.phase_timers:
        os.environ["RG_LIBRARY"] = os.path.join(ROOT, "paper_2605_29752_gb300", "librg_timers.so")
    import torch
    from paper_2605_29752_gb300 import rg
    M, N, K = args.shape
    if args.variant.startswith("fp8"):
        return single_shape_fp8(args, rg, torch)
    names = {rg.variant_name(v): v for v in range(rg.RG_NUM_VARIANTS)}
    v = names[args.variant]
    a, b = synthetic.operands_bf16(M, N, K, seed=0)
    A = torch.from_numpy(a.view(np.int16)).cuda().view(torch.bfloat16)
    B = torch.from_numpy(b.view(np.int16)).cuda().view(torch.bfloat16)
    C = torch.zeros((M, N), device="cuda")
    ctx = rg.rg_init(0)
    for _ in range(3):
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, v)
    rg.rg_check(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    for _ in range(args.reps):
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, v)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    rg.rg_check(ctx)
    us_host = e0.elapsed_time(e1) / args.reps * 1e3
    # The landscape's protocol: a device spin lets the host enqueue all `reps` launches first, so the
    # events time back-to-back device work (the Python loop above also times the host's launch rate).
    grid = rg.make_grid((M, 128, 1), (N, 128, 1), (K, 128, 1))
    opts = rg.rg_sweep_opts_default()
    opts.reps, opts.warmup, opts.shuffle, opts.prune_splits = args.reps, 1, 0, 0
    us = float(rg.rg_sweep(ctx, grid, [v], A, B, C, opts)[0, 0]) * 1e-3
    phases = None
    if args.phase_timers:
        rg.rg_phase_trace(ctx, True)
        opts.reps = 5               # the buffer keeps the last of the back-to-back launches
        rg.rg_sweep(ctx, grid, [v], A, B, C, opts)
        torch.cuda.synchronize()
        phases = phase_summary(rg.rg_phase_trace_read(ctx))
        rg.rg_phase_trace(ctx, False)
    rg.rg_destroy(ctx)
    tf = 2.0 * M * N * K / (us * 1e-6) / 1e12
    byts = 2 * M * K + 2 * K * N + 4 * M * N
    line = {"shape": [M, N, K], "variant": args.variant, "us_per_launch": us, "tflops": tf,
            "us_per_call_python_loop": us_host, "algorithmic_bytes": byts, "algorithmic_flops": 2 * M * N * K}
    if phases is not None:
        line["phase_times"] = phases
        line["library"] = "librg_timers.so (phase stamps compiled in; the timed launches carry them too)"
    print(json.dumps(line), flush=True)
    return 0


def cell_sizes(count):
    g = np.arange(1, count + 1) * STEP
    M, N, K = np.meshgrid(g, g, g, indexing="ij")
    return M.ravel().astype(np.int64), N.ravel().astype(np.int64), K.ravel().astype(np.int64)


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        import tempfile
        self.index = index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"rg_bench_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of a per-rank value over all ranks (the slowest replica's step time); the
    value itself without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def mean_over_ranks(value: float, dist=None, device=None) -> float:
    """The mean of a per-rank value over all ranks (replicas each measure the whole landscape)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item()) / dist.get_world_size()


def device_header(device_name, sms, grid_counts, variant_ids, version):
    """int64 header a rank sends beside its T0 shard: the merged table is valid only when every rank
    swept the same grid and variants on the same kind of GPU with the same library."""
    import hashlib

    def h63(x):
        return int.from_bytes(hashlib.sha256(str(x).encode()).digest()[:8], "little") >> 1
    return np.array([h63(device_name), int(sms), *[int(c) for c in grid_counts], len(variant_ids),
                     h63(list(variant_ids)), h63(version)], dtype=np.int64)


def merge_t0_shards(local, header, dist, device=None, unmeasured=1 << 60, other=0):
    """The exchange step of the sharded autotune sweep: all-gather every rank's header and int64 T0
    shard, check that the headers agree, and merge.  Each (variant, cell) entry is measured on exactly
    one rank (`other` elsewhere) or pruned on every rank (`unmeasured` everywhere)."""
    import torch
    world = dist.get_world_size()
    h = torch.as_tensor(np.asarray(header, dtype=np.int64), device=device)
    hs = [torch.empty_like(h) for _ in range(world)]
    dist.all_gather(hs, h)
    if any(not torch.equal(x, hs[0]) for x in hs):
        raise RuntimeError("sharded sweep: the ranks' headers differ (GPU model, SM count, grid, variants or "
                           "library); their timings cannot form one table")
    t = torch.as_tensor(np.ascontiguousarray(local, dtype=np.int64), device=device)
    ts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(ts, t)
    stack = torch.stack(ts).cpu().numpy()
    pruned = (stack == unmeasured).all(axis=0)
    measured = (stack != other) & (stack != unmeasured)
    count = measured.sum(axis=0)
    if np.any((count != 1) & ~pruned):
        raise RuntimeError("sharded sweep: some entries were measured on no rank or on several")
    return np.where(pruned, unmeasured, np.where(measured, stack, 0).sum(axis=0)).astype(np.int64)


def stats_of(rg, grid, t_ns):
    tf, r, mean = rg.rg_surface_stats(grid, t_ns)
    return tf, r, mean


def roof_times_ns(Mv, Nv, Kv, p_tflops, bw_gbs):
    """Per-cell roofline time t_roof = max(2MNK / P, (2MK + 2KN + 4MN) / BW) in ns (useful flops and
    algorithmic bytes of the BF16-in, FP32-out GEMM)."""
    Mv, Nv, Kv = (np.asarray(x, dtype=np.float64) for x in (Mv, Nv, Kv))
    t_c = 2.0 * Mv * Nv * Kv / (p_tflops * 1e3)
    t_m = (2.0 * Mv * Kv + 2.0 * Kv * Nv + 4.0 * Mv * Nv) / bw_gbs
    return np.maximum(t_c, t_m)


def summarize(tf, r, mean, t_ns=None, troof=None):
    out = {"mean_tflops": mean, "p50_tflops": float(np.percentile(tf, 50)),
           "p99_tflops": float(np.percentile(tf, 99)), "p01_tflops": float(np.percentile(tf, 1)),
           "max_tflops": float(tf.max()), "R_N_slice": r["R_N_slice"], "R_3D": r["R_3D"], "R_M": r["R_M"],
           "R_N": r["R_N"], "R_K": r["R_K"], "R_N_slice_over_mean": r["R_N_slice"] / mean if mean else None}
    if t_ns is not None and troof is not None:
        # mean over cells of t_roof / t_measured: the per-stage roofline fraction
        out["roofline_mean_frac"] = float(np.mean(troof / np.asarray(t_ns, dtype=np.float64).ravel()))
    return out


def slice_attribution(tf, count, kmax):
    """Where the N-axis roughness of the largest-K slice sits: its adjacent-N pairs split by the
    size MNK of the pair's larger cell (launch-bound < 1e9 <= mid < 1e10 <= saturated)."""
    S = np.asarray(tf, dtype=np.float64).reshape(count, count, count)[:, :, -1]
    d = np.abs(np.diff(S, axis=1))
    M = (np.arange(1, count + 1) * STEP)[:, None].astype(np.float64)
    N = (np.arange(2, count + 1) * STEP)[None, :].astype(np.float64)
    mnk = M * N * float(kmax) * np.ones_like(d)
    total = d.sum()
    out = {}
    for name, sel in (("MNK<1e9", mnk < 1e9), ("1e9<=MNK<1e10", (mnk >= 1e9) & (mnk < 1e10)),
                      ("MNK>=1e10", mnk >= 1e10)):
        out[name] = {"pair_share": float(sel.mean()), "abs_step_share": float(d[sel].sum() / total) if total else 0.0,
                     "mean_abs_step": float(d[sel].mean()) if sel.any() else 0.0,
                     "contribution_to_R_N_slice": float(d[sel].sum() / d.size)}
    return out


def noise_floor(tf_a, tf_b, count):
    """Roughness of the repeat-to-repeat difference surface (tf_a - tf_b) / sqrt(2): what measurement
    noise alone contributes to R_N on the largest-K slice and to the 3-axis R."""
    D = ((np.asarray(tf_a, np.float64) - np.asarray(tf_b, np.float64)) / np.sqrt(2.0)).reshape(count, count, count)
    rN_slice = float(np.mean(np.abs(np.diff(D[:, :, -1], axis=1))))
    r3 = float(np.mean([np.mean(np.abs(np.diff(D, axis=ax))) for ax in range(3)]))
    return {"R_N_slice": rN_slice, "R_3D": r3,
            "median_abs_rel_diff_pct": float(100 * np.median(np.abs(np.asarray(tf_a) - np.asarray(tf_b)) /
                                                           np.asarray(tf_b)))}


def sawtooth_period(series):
    """Lag (in grid steps, 1..8) with the largest autocorrelation of the step-to-step changes; among lags
    within 0.02 of the best, the smallest (a period's multiples correlate as well as the period itself)."""
    d = np.diff(np.asarray(series, dtype=np.float64))
    d = d - d.mean()
    corr = {}
    for lag in range(1, 9):
        if lag >= len(d):
            break
        corr[lag] = float(np.dot(d[:-lag], d[lag:]) / (np.linalg.norm(d[:-lag]) * np.linalg.norm(d[lag:]) + 1e-30))
    if not corr:
        return None, float("nan")
    best = max(corr.values())
    lag = min(k for k, c in corr.items() if c >= best - 0.02)
    return lag, corr[lag]


def cpu_info():
    """CPU model and the BLAS numpy uses, for the CPU-baseline record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    blas = None
    try:
        cfg = np.show_config(mode="dicts")
        b = cfg.get("Build Dependencies", {}).get("blas", {})
        blas = {k: b.get(k) for k in ("name", "version", "openblas configuration") if b.get(k)}
    except Exception:  # noqa: BLE001 - older numpy has no dict mode
        blas = None
    return {"cpu_model": model, "numpy": np.__version__, "blas": blas}


def cpu_baseline(count, seed=0, strata=256, gpu_config1=None):
    """The oracle, as it stands, on this host's cores (numpy FP64 matmul uses every core):
    (1) the 64 cells of the small sweep {128..512}^3, with the full-matrix error of the GPU's plain
    kernel on each against the oracle when gpu_config1 is given; (2) a stratified sample of the whole
    grid (cells sorted by MNK into `strata` equal strata, one seeded cell per stratum) extrapolated
    to the full sweep; (3) the textbook triple loop at 128^3 on one core; (4) the host steps."""
    from oracle import gemm as og
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    Mx = STEP * count
    a64 = og.bf16_bits_to_f64(synthetic.bf16_uniform_stream(0, synthetic.TAG_A, Mx * Mx))
    b64 = og.bf16_bits_to_f64(synthetic.bf16_uniform_stream(0, synthetic.TAG_B, Mx * Mx))

    def operands(M, N, K):
        return a64[:M * K].reshape(M, K), b64[:K * N].reshape(K, N)

    def timed(M, N, K):
        A, B = operands(M, N, K)
        t0 = time.perf_counter()
        c = og.gemm_f64(A, B)
        return time.perf_counter() - t0, c
    out = {"unit": "TFLOP/s", "cores": cores, "kind": "oracle", **cpu_info()}
    # (1) small sweep
    c1_vals, c1_flops, c1_secs, worst = [], 0.0, 0.0, 0.0
    small = [128, 256, 384, 512]
    for M in small:
        for N in small:
            for K in small:
                dt, c64 = timed(M, N, K)
                c1_vals.append(2.0 * M * N * K / dt / 1e12)
                c1_flops += 2.0 * M * N * K
                c1_secs += dt
                if gpu_config1 is not None:
                    A, B = operands(M, N, K)
                    ratio, exact = og.error_ratio(gpu_config1(M, N, K), c64, og.abs_sum(A, B))
                    worst = max(worst, ratio if exact else float("inf"))
    out["small_sweep_64_cells"] = {"mean_tflops": float(np.mean(c1_vals)), "aggregate_tflops": c1_flops / c1_secs / 1e12,
                                   "seconds": c1_secs}
    if gpu_config1 is not None:
        out["small_sweep_64_cells"]["gpu_plain_max_error_ratio"] = worst
        out["small_sweep_64_cells"]["error_bound_at_K512"] = og.bound(512)
    # (2) stratified sample of the whole grid
    Mv, Nv, Kv = cell_sizes(count)
    fl = 2.0 * Mv * Nv * Kv
    order = np.argsort(fl, kind="stable")
    groups = np.array_split(order, strata)
    rs = np.random.default_rng(seed)
    vals, secs, flops, extrap = [], 0.0, 0.0, 0.0
    for g in groups:
        i = int(g[rs.integers(len(g))])
        dt, _ = timed(int(Mv[i]), int(Nv[i]), int(Kv[i]))
        vals.append(fl[i] / dt / 1e12)
        secs += dt
        flops += fl[i]
        extrap += dt * len(g)
    out.update({"value": float(np.mean(vals)), "aggregate_tflops": flops / secs / 1e12,
                "full_sweep_extrapolated_s": extrap, "full_sweep_flops": float(fl.sum()),
                "full_sweep_extrapolated_tflops": float(fl.sum()) / extrap / 1e12,
                "sample": f"{strata} cells, one per stratum of the {count}^3 grid sorted by MNK ({len(groups[0])} "
                          f"cells per stratum, seed {seed}); oracle FP64 numpy matmul per cell on {cores} cores; "
                          f"value = mean per-cell TFLOP/s; {secs:.1f} s of CPU GEMM; the full sweep extrapolated as "
                          f"sum over strata of (sample time x stratum size)"})
    # (3) triple loop, one core
    A, B = operands(128, 128, 128)
    t0 = time.perf_counter()
    og.gemm_f64_loops(A, B)
    dt = time.perf_counter() - t0
    out["triple_loop_128cube_one_core"] = {"seconds": dt, "tflops": 2.0 * 128 ** 3 / dt / 1e12}
    out.update(host_steps_timing(count, seed))
    return out


def host_steps_timing(count, seed=0, variants=6):
    """The host steps of the path on a seeded synthetic T0 table of the whole grid: the oracle's
    pure-Python DP (best-of, T1, T2) and roughness, beside the library's native plan build and
    statistics on the same table (one thread each)."""
    from oracle import dp, roughness
    from paper_2605_29752_gb300 import rg
    rs = np.random.default_rng(seed)
    shape = (count, count, count)
    T0v = rs.integers(1000, 10 ** 7, size=(variants,) + shape).astype(np.int64)
    grid = ((STEP, STEP, count),) * 3
    t0 = time.perf_counter()
    T0s, _ = dp.best_of(T0v)
    T1, _ = dp.pad_T1(T0s, grid)
    dp.split_T2(T1, grid)
    t_oracle_dp = time.perf_counter() - t0
    t0 = time.perf_counter()
    roughness.roughness_all(roughness.surface(T0s, grid))
    t_oracle_r = time.perf_counter() - t0
    g = rg.make_grid((STEP, STEP, count))
    t0 = time.perf_counter()
    h = rg.rg_plan_build(g, T0v.reshape(variants, -1), list(range(variants)))
    t_lib_dp = time.perf_counter() - t0
    rg.rg_plan_free(h)
    t0 = time.perf_counter()
    rg.rg_surface_stats(g, T0s.reshape(-1))
    t_lib_r = time.perf_counter() - t0
    return {"host_steps": {"table": f"{variants} variants x {count}^3 cells, seeded uniform integers",
                           "oracle_dp_s": t_oracle_dp, "oracle_roughness_s": t_oracle_r,
                           "library_plan_build_s": t_lib_dp, "library_surface_stats_s": t_lib_r}}


def reference_arm(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from oracle import gemm as og
    count = args.count
    cells = synthetic.uniform_cells(64, (count, count, count), seed=1)
    # size each step to a few seconds of CPU work and at most ~2 GB of float64 operands
    per_step, t_acc, bytes_acc = [], 0.0, 0
    for a, b, c in cells:
        M, N, K = (int(a) + 1) * STEP, (int(b) + 1) * STEP, (int(c) + 1) * STEP
        if bytes_acc + 8 * (M * K + K * N) > 2 << 30:
            continue
        ab, bb = synthetic.operands_bf16(M, N, K, seed=0)
        op = (M, N, K, og.bf16_bits_to_f64(ab), og.bf16_bits_to_f64(bb))
        s0 = time.perf_counter()
        og.gemm_f64(op[3], op[4])
        t_acc += time.perf_counter() - s0
        bytes_acc += 8 * (M * K + K * N)
        per_step.append(op)
        if t_acc > 4.0:
            break

    def step():
        vals = []
        for M, N, K, A, B in per_step:
            s = time.perf_counter()
            og.gemm_f64(A, B)
            vals.append(2.0 * M * N * K / (time.perf_counter() - s) / 1e12)
        return float(np.mean(vals))

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    vals = [step() for _ in range(args.steps)]
    elapsed = time.perf_counter() - t0
    value = float(np.mean(vals))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "replicas", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"BF16 NN GEMM landscape {count}^3 cells, "
                                                        f"FP64 CPU oracle on a {len(per_step)}-cell sample"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{len(per_step)} cells drawn uniformly from the grid (seed 1), "
                                       f"FP64 numpy GEMM each, mean per-cell TFLOP/s"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.shape:
        return single_shape(args)
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2605_29752_gb300 import rg

    count = args.count
    grid = rg.make_grid((STEP, STEP, count))
    ncell = count ** 3
    Mx = STEP * count
    Mv, Nv, Kv = cell_sizes(count)
    flops = 2.0 * Mv * Nv * Kv
    dev = torch.device("cuda", local)

    def dev_bf16(bits):
        return torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)

    a_bits = synthetic.bf16_uniform_stream(0, synthetic.TAG_A, Mx * Mx)
    b_bits = synthetic.bf16_uniform_stream(0, synthetic.TAG_B, Mx * Mx)
    A, B = dev_bf16(a_bits), dev_bf16(b_bits)
    C = torch.zeros(Mx * Mx, device=dev, dtype=torch.float32)
    ctx = rg.rg_init(local)
    sms = rg.rg_sm_count(ctx)

    # ---------------- offline autotune (setup); on several GPUs each rank times a shard of the
    # (variant, cell) items and one all-gather of the int64 tables merges them
    t_setup = time.perf_counter()
    all_v = list(range(rg.RG_NUM_VARIANTS))
    if world > 1:
        o = rg.rg_sweep_opts_default()
        o.shard_index, o.shard_count = rank, world
        local_t = rg.rg_sweep(ctx, grid, all_v, A, B, C, o)
        hdr = device_header(torch.cuda.get_device_name(dev), sms, (count, count, count), all_v, rg.rg_version())
        T0v = merge_t0_shards(local_t, hdr, dist, dev, rg.RG_T_UNMEASURED, rg.RG_T_OTHER_SHARD)
    else:
        T0v = rg.rg_sweep(ctx, grid, all_v, A, B, C)
    s1_rows = [rg.variant(t, 1) for t in range(rg.RG_NUM_PAPER_TILES)]   # the paper's best-of-6
    plan_smooth = rg.rg_plan_build(grid, T0v, all_v)
    setup_s = time.perf_counter() - t_setup
    fixed_v = rg.variant(FIXED_TILE, 1)

    def one_step():
        tp = rg.rg_sweep(ctx, grid, [fixed_v], A, B, C)[0]
        ts = rg.rg_sweep(ctx, grid, [0], A, B, C, plan=plan_smooth)[0]
        return tp, ts

    for _ in range(args.warmup):
        one_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = rg.rg_launch_count(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with ClockSampler(local, args.clock_log) as clk:
        torch.cuda.nvtx.range_push("timed")
        ev0.record()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            results.append(one_step())
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    n_launch = rg.rg_launch_count(ctx) - n_launch0
    step_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, dev)

    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    p_burst = peaks.get("bf16_tflops") or 1900.0
    bw = peaks.get("hbm_gbs") or 6800.0
    peak_src = "measured" if peaks else "fallback"
    troof = roof_times_ns(Mv, Nv, Kv, p_burst, bw)

    plain = [summarize(*stats_of(rg, grid, tp), t_ns=tp, troof=troof) for tp, _ in results]
    smooth = [summarize(*stats_of(rg, grid, ts), t_ns=ts, troof=troof) for _, ts in results]
    value = mean_over_ranks(float(np.mean([s["mean_tflops"] for s in smooth])), dist, dev)
    last_p, last_s = results[-1]
    agg_flops = float(flops.sum())
    agg_smooth = agg_flops / (last_s.astype(np.float64).sum() * 1e-9) / 1e12
    agg_plain = agg_flops / (last_p.astype(np.float64).sum() * 1e-9) / 1e12
    tf_p = [stats_of(rg, grid, tp)[0] for tp, _ in results]
    tf_s = [stats_of(rg, grid, ts)[0] for _, ts in results]
    rough = {"plain_slice_attribution": slice_attribution(tf_p[-1], count, Mx),
             "smoothed_slice_attribution": slice_attribution(tf_s[-1], count, Mx)}
    if len(results) >= 2:
        rough["noise_floor_plain"] = noise_floor(tf_p[-1], tf_p[-2], count)
        rough["noise_floor_smoothed"] = noise_floor(tf_s[-1], tf_s[-2], count)
    rough["note"] = ("N-axis roughness of the K = max slice split by the size of each adjacent pair's larger "
                     "cell; noise floor = roughness of (repeat - repeat) / sqrt(2) of two timed steps")

    # dominant kernel of the smoothed pass: the variant whose single-leaf cells take the most device time
    leaf_v = np.full(ncell, -1, dtype=np.int64)
    for i in range(ncell):
        lv, _ = rg.rg_plan_lookup(plan_smooth, int(Mv[i]), int(Nv[i]), int(Kv[i]))
        if len(lv) == 1:
            leaf_v[i] = lv[0][0]
    share = {}
    for v in set(leaf_v.tolist()) - {-1}:
        share[v] = float(last_s[leaf_v == v].astype(np.float64).sum())
    dom = max(share, key=share.get)
    dsel = leaf_v == dom
    dom_ach = float(flops[dsel].sum() / (last_s[dsel].astype(np.float64).sum() * 1e-9) / 1e12)
    dom_share = share[dom] / float(last_s.astype(np.float64).sum())

    # best single cell of the autotune table
    T0s = T0v.min(axis=0)
    best_tf = flops / (T0s * 1e3)
    bi = int(np.argmax(best_tf))
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "replicas" if world > 1 else "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": f"BF16 NN GEMM landscape, (M,N,K) in {{128..{Mx} step 128}}^3 = {ncell} cells, "
                               f"U[-1,1) BF16 operands (seed 0), FP32 accumulate/output",
                   "smoothed": f"best-of-{rg.RG_NUM_VARIANTS} autotune (the paper's 6 tiles and 128x192, each x "
                               "{split-K 1/2/4/8, stream-K}; 2 cta_group::2 tiles x {split-K 1/2/4/8, stream-K}) + "
                               "DP pad/split plan, O(1) lookup",
                   "plain": "fixed 128x128 tile, split 1",
                   "timing": "per cell: 1 warm-up launch, device spin, mean of 5 back-to-back launches between "
                             "CUDA events (paper protocol, warm per cell: operands of small cells stay L2-resident "
                             "across their 5 launches, no flush); between timed steps: inputs larger than L2 (each "
                             "step reads all of A and B, 2 x 32 MiB, and writes all of C, 64 MiB: 134 MB against "
                             "the 129 MB L2, across 65,536 cell measurements)",
                   "parallelism": "single GPU" if world == 1 else
                                  f"autotune sweep sharded over {world} GPUs (one int64 T0 all-gather); the timed "
                                  f"landscape steps as {world} independent replicas"},
        "plain": {k: float(np.mean([p[k] for p in plain])) for k in plain[0]},
        "smoothed": {k: float(np.mean([s[k] for s in smooth])) for k in smooth[0]},
        "roughness_cut_pct": 100.0 * (1 - np.mean([s["R_N_slice"] for s in smooth]) /
                                      np.mean([p["R_N_slice"] for p in plain])),
        "mean_gain_pct": 100.0 * (value / np.mean([p["mean_tflops"] for p in plain]) - 1),
        "roofline": {"bound": "tensor", "achieved": dom_ach, "peak": p_burst, "unit": "TFLOP/s",
                     "frac": dom_ach / p_burst, **dominant_traffic(rg.variant_name(dom)),
                     "mean_frac": float(np.mean([q["roofline_mean_frac"] for q in smooth])),
                     "kernel": f"gemm_bf16 {rg.variant_name(dom)}",
                     "note": f"dominant kernel of the smoothed pass ({100 * dom_share:.1f}% of its device time, "
                             f"{int(dsel.sum())} single-launch cells): useful 2MNK flops / CUDA-event time of "
                             f"those cells' timed launches; peak = {peak_src} bf16 burst; the cells differ in "
                             f"size, so traffic is per launch of one captured mid-size cell (traffic_cell, "
                             f"traffic_profile), and mean_frac is the mean over all cells of t_roof / t_measured "
                             f"for the smoothed pass"},
        "roofline_all_gemms": {"achieved": agg_smooth, "frac": agg_smooth / p_burst, "unit": "TFLOP/s"},
        "roofline_mean_frac": {"plain": float(np.mean([p["roofline_mean_frac"] for p in plain])),
                               "smoothed": float(np.mean([q["roofline_mean_frac"] for q in smooth])),
                               "definition": "mean over the cells of t_roof / t_measured, t_roof = max(2MNK / P, "
                                             "(2MK + 2KN + 4MN) / BW)", "P_tflops": p_burst, "BW_gbs": bw,
                               "peaks": peak_src},
        "roughness_analysis": rough,
        "plain_aggregate_tflops": agg_plain,
        "peak_cell": {"M": int(Mv[bi]), "N": int(Nv[bi]), "K": int(Kv[bi]), "tflops": float(best_tf[bi]),
                      "variant": rg.variant_name(int(T0v[:, bi].argmin())), "frac": float(best_tf[bi]) / p_burst},
        "gpu_launches": int(n_launch),
        "sm_count": sms,
        "setup_s": setup_s,
        "clocks": clk.summary(),
    }

    if rank == 0:
        line["roofline_capture"] = roofline_capture(rg, ctx, p_burst, dev)
    if not args.no_extras and rank == 0:
        line.update(extras(args, rg, ctx, grid, T0v, plan_smooth, A, B, C, flops, Mv, Nv, Kv, dev, a_bits, b_bits,
                           s1_rows, fixed_v, p_burst, sms, troof, bw))
    rg.rg_plan_free(plan_smooth)
    rg.rg_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(line, f, indent=1)
            np.savez_compressed(os.path.splitext(args.out)[0] + "_surfaces.npz", T0v=T0v, plain=last_p,
                                smooth=last_s)
    if dist:
        dist.destroy_process_group()
    return 0


def kernel_source_hash():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2605_29752_gb300", "csrc")
    src = open(os.path.join(csrc, "rg_gemm.cu")).read()
    kern = src[:src.index("// ------------------------------------------------------------------ host side")]
    return hashlib.sha256((open(os.path.join(csrc, "ptx.cuh")).read() + kern).encode()).hexdigest()


CAPTURE_PROFILE = "gemm_bf16_256x256_2sm_8192x8192x4096"   # profiles/<name>.md and .json
CAPTURE_VARIANT = "256x256/2SM"
# ncu captures of kernels that can dominate the smoothed pass, each on a mid-size landscape cell it wins
TRAFFIC_PROFILES = {"256x256/2SM": "gemm_bf16_256x256_2sm_2048x2048x4096",
                    "128x128/S1": "gemm_bf16_128x128_2048x2048x4096",
                    "128x192/S1": "gemm_bf16_128x192_2048x1536x4096",
                    "256x192/S1": "gemm_bf16_256x192_4096x1536x4096"}


def dominant_traffic(variant_name):
    """DRAM traffic per launch of the dominant kernel on one captured mid-size landscape cell, from the ncu
    capture in profiles/ (null when the kernel differs from the captured one or the source changed since)."""
    name = TRAFFIC_PROFILES.get(variant_name)
    path = os.path.join(ROOT, "profiles", f"{name}.json")
    if name is None or not os.path.exists(path):
        return {"traffic": None, "traffic_note": "no capture of this kernel on a landscape cell"}
    prof = json.load(open(path))
    if prof["kernel_source_sha256"] != kernel_source_hash():
        return {"traffic": None, "traffic_note": "the kernel source changed since the capture"}
    t = prof["dram_bytes_read"] + prof["dram_bytes_write"]
    return {"traffic": t, "traffic_cell": prof["shape"], "traffic_over_algorithmic": t / prof["algorithmic_bytes"],
            "traffic_profile": f"profiles/{name}.md", "traffic_note": prof["l2_resident"]}


def roofline_capture(rg, ctx, p_burst, dev, reps=10):
    """The kernel and shape of profiles/<CAPTURE_PROFILE>: timed live here, DRAM traffic from that ncu
    capture (null once the kernel source differs from the captured one)."""
    import torch
    prof = json.load(open(os.path.join(ROOT, "profiles", CAPTURE_PROFILE + ".json")))
    M, N, K = prof["shape"]
    v = {rg.variant_name(x): x for x in range(rg.RG_NUM_VARIANTS)}[CAPTURE_VARIANT]
    A = torch.from_numpy(synthetic.bf16_uniform_stream(0, 1, M * K).view(np.int16)).to(dev).view(torch.bfloat16)
    B = torch.from_numpy(synthetic.bf16_uniform_stream(0, 2, K * N).view(np.int16)).to(dev).view(torch.bfloat16)
    C = torch.empty((M, N), device=dev)
    for _ in range(3):
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, v)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, C, N, v)
    e1.record()
    torch.cuda.synchronize()
    rg.rg_check(ctx)
    t = e0.elapsed_time(e1) / reps * 1e-3
    ach = 2.0 * M * N * K / t / 1e12
    same = prof["kernel_source_sha256"] == kernel_source_hash()
    traffic = prof["dram_bytes_read"] + prof["dram_bytes_write"] if same else None
    return {"bound": "tensor", "kernel": prof["kernel"], "shape": [M, N, K], "achieved": ach, "peak": p_burst,
            "unit": "TFLOP/s", "frac": ach / p_burst, "traffic": traffic,
            "algorithmic_bytes": 2 * M * K + 2 * K * N + 4 * M * N,
            "note": "10 back-to-back launches between CUDA events; inputs 384 MiB > L2; traffic = ncu "
                    f"dram__bytes_read.sum + dram__bytes_write.sum per launch (profiles/{CAPTURE_PROFILE}.md)"}


def extras(args, rg, ctx, grid, T0v, plan_smooth, A, B, C, flops, Mv, Nv, Kv, dev, a_bits, b_bits, s1_rows,
           fixed_v, p_burst, sms, troof, bw):
    import torch
    out = {}
    count = args.count
    # ---- ladder: fixed -> best-of-6 -> DP pad -> DP split+pad -> autotuner + DP (Sec. 7.5, Table 10)
    ladder = {}
    tf, r, m = rg.rg_surface_stats(grid, T0v[fixed_v])
    ladder["fixed_128x128"] = summarize(tf, r, m, T0v[fixed_v], troof)
    T6 = T0v[s1_rows]
    tf, r, m = rg.rg_surface_stats(grid, T6.min(axis=0))
    ladder["best_of_6"] = summarize(tf, r, m, T6.min(axis=0), troof)
    tf, r, m = rg.rg_surface_stats(grid, T0v.min(axis=0))
    ladder["best_of_all_variants_autotune"] = summarize(tf, r, m, T0v.min(axis=0), troof)
    for name, rows, flags in (("dp_pad_on_best_of_6", s1_rows, rg.RG_PLAN_PAD_ONLY),
                              ("dp_split_pad_on_best_of_6", s1_rows, 0),
                              ("dp_split_pad_on_fixed", [fixed_v], 0)):
        h = rg.rg_plan_build_ex(grid, T0v[rows], rows, flags)
        t = rg.rg_plan_tables(h)
        tf, r, m = rg.rg_surface_stats(grid, t["T2"])
        pred = summarize(tf, r, m, t["T2"], troof)
        meas = rg.rg_sweep(ctx, grid, [0], A, B, C, plan=h)[0]
        tf, r, m = rg.rg_surface_stats(grid, meas)
        ladder[name] = {"predicted": pred, "measured": summarize(tf, r, m, meas, troof)}
        rg.rg_plan_free(h)
    t = rg.rg_plan_tables(plan_smooth)
    tf, r, m = rg.rg_surface_stats(grid, t["T2"])
    ladder["autotune_dp_split_pad_predicted"] = summarize(tf, r, m, t["T2"], troof)
    out["ladder"] = ladder
    # ---- DP action distribution at the largest K (Sec. 7.3, Table 9)
    act = t["action"][:, :, -1].ravel()
    tgt = t["target"][:, :, -1].reshape(-1, 3)
    cells_k = np.array([(a, b, count - 1) for a in range(count) for b in range(count)])
    padded = np.any(tgt != cells_k, axis=1)
    out["dp_actions_at_kmax"] = {"as_is": float(np.mean((act == 0) & ~padded)), "pad": float(np.mean((act == 0) & padded)),
                                 "split_M": float(np.mean(act == 1)), "split_N": float(np.mean(act == 2)),
                                 "split_K": float(np.mean(act == 3))}
    vs = t["vstar"].ravel()
    out["autotune_winners"] = {rg.variant_name(v): float(np.mean(vs == v)) for v in sorted(set(vs.tolist()))}
    # ---- cross-tile N sweep at M = K = 2048 (Sec. 6.3): sawtooth period per tile
    ia = ik = 2048 // STEP - 1
    if ia < count:
        ct = {}
        for tile in range(rg.RG_NUM_PAPER_TILES):
            v = rg.variant(tile, 1)
            t_line = T0v[v].reshape(count, count, count)[ia, :, ik]
            tfl = 2.0 * 2048 * 2048 * (np.arange(1, count + 1) * STEP) / (t_line * 1e3)
            lag, corr = sawtooth_period(tfl)
            ct[rg.variant_name(v)] = {"period": "aliased at step 128 (periods below 256 cannot show; see "
                                                "fine_N_sweep)", "best_lag_steps": lag, "lag_autocorr": corr,
                                      "mean": float(tfl.mean()), "roughness": float(np.mean(np.abs(np.diff(tfl))))}
        out["cross_tile_N_at_M_K_2048"] = ct
    # ---- first-principles GB300 landscapes (Sec. 9) and KOL grades (Sec. 10) of the measured surfaces
    bw = (json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
          if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0)
    ideal = rg.rg_landscape(grid, rg.RG_LANDSCAPE_IDEAL, p_burst, sms, 0.0, [(128, 128)])
    opt = rg.rg_landscape(grid, rg.RG_LANDSCAPE_OPTIMAL, p_burst, sms, bw, rg.TILES[:rg.RG_NUM_PAPER_TILES])
    fp = {}
    for name, surf in (("ideal_128x128", ideal), ("optimal_six_tiles", opt)):
        t_eq = np.maximum(1, np.round(flops / (surf * 1e3))).astype(np.int64)   # as integer ns, for the stats call
        _, r, _ = rg.rg_surface_stats(grid, t_eq)
        fp[name] = {"mean_tflops": float(surf.mean()), "R_N_slice": r["R_N_slice"], "R_3D": r["R_3D"]}
    fp["constants"] = {"P_tflops": p_burst, "C_sms": sms, "BW_gbs": bw, "eta_channel": 1.0}
    out["first_principles"] = fp
    o = fp["optimal_six_tiles"]
    out["kol"] = {name: rg.rg_kol(ladder_mean, o["mean_tflops"], ladder_r, o["R_N_slice"])
                  for name, ladder_mean, ladder_r in (
                      ("fixed_128x128", ladder["fixed_128x128"]["mean_tflops"], ladder["fixed_128x128"]["R_N_slice"]),
                      ("best_of_6", ladder["best_of_6"]["mean_tflops"], ladder["best_of_6"]["R_N_slice"]),
                      ("dp_split_pad_on_best_of_6", ladder["dp_split_pad_on_best_of_6"]["measured"]["mean_tflops"],
                       ladder["dp_split_pad_on_best_of_6"]["measured"]["R_N_slice"]))}
    # ---- four-surface decomposition (Sec. 4) with the memory twins
    out["decomposition"] = decomposition(rg, ctx, grid, T0v, s1_rows, fixed_v, A, B, C, p_burst, count)
    # ---- fine step-32 cross-tile N sweep at M = K = 4096 with DP padding on the fine grid (Sec. 8.3-8.4)
    if count * STEP >= 4096:
        out["fine_N_sweep"] = fine_n_sweep(rg, ctx, A, B, C)
    # ---- measurement methodology (Sec. 5.3-5.4, Sec. 8.2): run-order drift, co-allocation, per-config spread
    out["methodology"] = methodology(rg, ctx, grid, T0v, fixed_v, plan_smooth, A, B, C, dev, count)
    # ---- serving (continuous batching over the grouped GEMM), at half the saturated capacity
    out["serving"] = serving(rg, ctx, plan_smooth, A, B, count)
    # ---- FP8 e4m3 block-scaled GEMM on the {512..4096 step 512}^3 subgrid: autotune, plan, re-measure
    out["fp8"], fp8_state = fp8_landscape(rg, ctx, dev, count, p_burst)
    # ---- e2e: host buffers through the public API (H2D, plan GEMM, D2H per cell)
    out["e2e"] = e2e(rg, ctx, plan_smooth, a_bits, b_bits, dev, count)
    # ---- the small sweep {128..512}^3 on the fixed tile (its own configuration)
    out["small_sweep_config"] = small_sweep(rg, ctx, A, B, C, fixed_v, p_burst, bw)

    def gpu_config1(M, N, K):
        Cc = torch.empty((M, N), device=dev)
        rg.rg_gemm(ctx, M, N, K, A, K, B, N, Cc, N, fixed_v)
        rg.rg_check(ctx)
        return Cc.cpu().numpy()
    # ---- CPU oracle baseline on this host (and the small sweep's full-matrix errors against it)
    out["cpu_baseline"] = cpu_baseline(count, gpu_config1=gpu_config1 if count >= 4 else None)
    if fp8_state is not None:     # the FP8 plan's per-shape error against the oracle (CPU-baseline leg)
        out["fp8"]["error_per_shape"] = fp8_errors(rg, ctx, fp8_state, dev)
        rg.rg_plan_free(fp8_state["plan"])
    if count >= 4:
        out["small_sweep_config"]["max_error_ratio_vs_oracle"] = \
            out["cpu_baseline"]["small_sweep_64_cells"]["gpu_plain_max_error_ratio"]
        out["small_sweep_config"]["error_bound"] = "K * 2^-24 (K <= 512: 3.05e-5)"
    return out


def small_sweep(rg, ctx, A, B, C, fixed_v, p_burst, bw):
    """The 64-cell sweep (M, N, K) in {128, 256, 384, 512}^3 with the single fixed 128x128 tile: its
    surface (from rg_sweep), roughness along each axis, mean TFLOP/s and roofline fraction."""
    g = rg.make_grid((STEP, STEP, 4))
    t, tf, st = rg.rg_sweep_surfaces(ctx, g, [fixed_v], A, B, C)
    Mv, Nv, Kv = cell_sizes(4)
    troof = roof_times_ns(Mv, Nv, Kv, p_burst, bw)
    keys = rg.SWEEP_STATS
    return {"grid": "{128, 256, 384, 512}^3 = 64 cells", "variant": rg.variant_name(fixed_v),
            **{k: float(st[0][i]) for i, k in enumerate(keys)},
            "roofline_mean_frac": float(np.mean(troof / t[0].astype(np.float64))),
            "surface_tflops": [round(float(x), 3) for x in tf[0]]}


def decomposition(rg, ctx, grid, T0v, s1_rows, fixed_v, A, B, C, p_burst, count):
    """Compute / memory / GEMM / overhead surfaces (Sec. 4): the fixed tile over the whole grid, and
    every tile's twin on the largest-K slice for the best-of-6 surface and the N profile of Fig. 6."""
    out = {}

    def summary(g, tg, tm):
        _, over, st = rg.rg_decompose(g, tg, tm, p_burst)
        _, r_mem, m_mem = rg.rg_surface_stats(g, tm)
        _, r_gemm, m_gemm = rg.rg_surface_stats(g, tg)
        return {"compute_bound_share": float(st[0]), "overhead_share_mean": float(st[1]),
                "overhead_share_pooled": float(st[2]), "memory_share_mean": float(st[3]),
                "memory_equiv_tflops_mean": m_mem, "memory_equiv_R_N_slice": r_mem["R_N_slice"],
                "memory_equiv_R_3D": r_mem["R_3D"], "gemm_R_N_slice": r_gemm["R_N_slice"],
                "gemm_R_3D": r_gemm["R_3D"]}, over

    tm_fixed = rg.rg_sweep_memtwin(ctx, grid, [rg.variant_tile(fixed_v)], A, B, C)[0]
    out["fixed_128x128_full_grid"], _ = summary(grid, T0v[fixed_v], tm_fixed)
    kmax = STEP * count
    gk = rg.make_grid((STEP, STEP, count), (STEP, STEP, count), (kmax, STEP, 1))
    tm6 = rg.rg_sweep_memtwin(ctx, gk, list(range(rg.RG_NUM_PAPER_TILES)), A, B, C)
    tg6 = np.stack([T0v[v].reshape(count, count, count)[:, :, -1].ravel() for v in s1_rows])
    win = tg6.argmin(axis=0)
    cols = np.arange(tg6.shape[1])
    best_g, best_m = tg6[win, cols], tm6[win, cols]
    out["best_of_6_K_max_slice"], _ = summary(gk, best_g, best_m)
    # Fig. 6: the time stack along N at M = K = max, fixed tile
    ti = rg.variant_tile(fixed_v)
    row = slice((count - 1) * count, count * count)
    prof = []
    for j in range(count):
        n = STEP * (j + 1)
        tg = float(T0v[fixed_v].reshape(count, count, count)[count - 1, j, -1])
        tm = float(tm6[ti][row][j])
        tc = 2.0 * kmax * n * kmax / (p_burst * 1e3)
        prof.append({"N": n, "compute_ns": tc, "memory_ns": tm, "gemm_ns": tg, "overhead_ns": tg - max(tc, tm)})
    out["N_profile_fixed_tile_M_K_max"] = prof[3::4]
    out["note"] = ("memory twin = the tile's GEMM kernel with every MMA a no-op (same TMA loads, pipeline, "
                   "TMEM read-back and stores); compute = 2MNK at the measured bf16 burst peak; "
                   "memory_equiv_* = statistics of the surface 2MNK / t_memory")
    return out


def fine_n_sweep(rg, ctx, A, B, C, n0=3000, step=32, count=35, mk=4096):
    """N = 3000..4088 step 32 at M = K = 4096 for every tile (split 1), then DP padding (T0 -> T1) on
    that fine grid per tile and on the best-of-6 envelope (Sec. 8.3-8.4, Tables 13-14)."""
    g = rg.make_grid((mk, STEP, 1), (n0, step, count), (mk, STEP, 1))
    rows = [rg.variant(t, 1) for t in range(rg.RG_NUM_PAPER_TILES)]
    T0 = rg.rg_sweep(ctx, g, rows, A, B, C)
    Ns = n0 + step * np.arange(count)
    out = {"grid": f"M = K = {mk}, N = {n0}..{Ns[-1]} step {step}"}

    def stats(t_row):
        tf, r, m = rg.rg_surface_stats(g, t_row)
        return tf, r["R_N"], m

    def entry(t_rows, vids, bn):
        t0 = t_rows.min(axis=0) if t_rows.ndim == 2 else t_rows
        tf0, r0, m0 = stats(t0)
        h = rg.rg_plan_build_ex(g, np.atleast_2d(t_rows), vids, rg.RG_PLAN_PAD_ONLY)
        t1 = rg.rg_plan_tables(h)["T1"]
        rg.rg_plan_free(h)
        tf1, r1, m1 = stats(t1)
        valleys = [int(i) for i in range(1, count - 1) if tf0[i] < tf0[i - 1] and tf0[i] < tf0[i + 1]]
        lag, corr = sawtooth_period(tf0)
        e = {"T0_roughness": r0, "T1_roughness": r1, "reduction_pct": 100.0 * (1 - r1 / r0) if r0 > 0 else 0.0,
             "T0_mean": m0, "T1_mean": m1, "T0_min": float(tf0.min()), "T1_min": float(tf1.min()),
             "period_N": None if lag is None else int(lag * step), "period_autocorr": corr,
             "valleys_N": [int(Ns[i]) for i in valleys]}
        if bn:
            mods = [int(Ns[i]) % bn for i in valleys]
            e["valley_N_mod_BN"] = mods
            e["valley_N_mod_BN_mode"] = max(set(mods), key=mods.count) if mods else None
        return e

    for t, v in enumerate(rows):
        out[rg.variant_name(v)] = entry(T0[t], [v], rg.TILES[t][1])
    out["best_of_6_envelope"] = entry(T0, rows, None)
    return out


def _ranks(x):
    r = np.empty(len(x))
    r[np.argsort(x, kind="stable")] = np.arange(len(x))
    return r


def methodology(rg, ctx, grid, T0v, fixed_v, plan, A, B, C, dev, count, runs=50):
    """Sec. 5.3-5.4: a sequential-order sweep against the randomized one (run-order drift); the memory
    twin on co-allocated prefixes against freshly allocated exact-size buffers; Sec. 8.2 / Table 12:
    the spread of 50 independent measurements of five configurations through the smoothed plan."""
    import torch
    out = {}
    o = rg.rg_sweep_opts_default()
    o.shuffle = 0
    t_seq = rg.rg_sweep(ctx, grid, [fixed_v], A, B, C, o)[0].astype(np.float64)
    t_rnd = T0v[fixed_v].astype(np.float64)
    ratio = t_seq / t_rnd
    order = np.arange(len(ratio))
    rho = float(np.corrcoef(_ranks(ratio), _ranks(order))[0, 1])
    blocks = ratio.reshape(count, -1)
    tenth = max(1, blocks.shape[1] // 10)
    out["order"] = {"median_abs_rel_diff_pct": float(100 * np.median(np.abs(ratio - 1))),
                    "mean_ratio_seq_over_random": float(ratio.mean()),
                    "spearman_ratio_vs_sequential_order": rho,
                    "first_tenth_vs_last_tenth_of_M_blocks_pct":
                        float(100 * (blocks[:, :tenth].mean() / blocks[:, -tenth:].mean() - 1))}
    # co-allocation: 64 seeded cells, memory twin of the fixed tile
    rs = np.random.default_rng(0)
    cells = rs.choice(count ** 3, 64, replace=False)
    slow = []
    for c in cells:
        a, b, k = c // (count * count), (c // count) % count, c % count
        M, N, K = STEP * (a + 1), STEP * (b + 1), STEP * (k + 1)
        g1 = rg.make_grid((M, STEP, 1), (N, STEP, 1), (K, STEP, 1))
        t_co = rg.rg_sweep_memtwin(ctx, g1, [rg.variant_tile(fixed_v)], A, B, C)[0][0]
        Ai = torch.empty(M * K, dtype=torch.bfloat16, device=dev).copy_(A[:M * K])
        Bi = torch.empty(K * N, dtype=torch.bfloat16, device=dev).copy_(B[:K * N])
        Ci = torch.empty(M * N, dtype=torch.float32, device=dev)
        t_iso = rg.rg_sweep_memtwin(ctx, g1, [rg.variant_tile(fixed_v)], Ai, Bi, Ci)[0][0]
        slow.append(t_co / t_iso)
        del Ai, Bi, Ci
    slow = np.array(slow)
    out["coallocation"] = {"cells": 64, "mean_slowdown_coallocated_over_isolated": float(slow.mean()),
                           "share_over_20pct": float(np.mean(slow > 1.2)),
                           "share_over_5pct": float(np.mean(slow > 1.05))}
    # per-configuration spread over 50 independent measurements (Table 12's five configurations)
    confs = {"aligned_rect_4096x2048x4096": (4096, 2048, 4096), "aligned_square_4096^3": (4096, 4096, 4096),
             "misaligned_N3168": (4096, 3168, 4096), "misaligned_N3096": (4096, 3096, 4096),
             "saturation_2560x1536x4096": (2560, 1536, 4096)}
    spread = {}
    for name, (M, N, K) in confs.items():
        if max(M, N, K) > STEP * count:
            continue
        g1 = rg.make_grid((M, STEP, 1), (N, STEP, 1), (K, STEP, 1))
        ts = np.array([rg.rg_sweep(ctx, g1, [0], A, B, C, plan=plan)[0][0] for _ in range(runs)], np.float64)
        tf = 2.0 * M * N * K / (ts * 1e3)
        spread[name] = {"mean_tflops": float(tf.mean()), "std": float(tf.std(ddof=1)),
                        "cv_pct": float(100 * tf.std(ddof=1) / tf.mean()),
                        "range_pct": float(100 * (tf.max() - tf.min()) / tf.mean())}
    out["per_config_spread_50_runs"] = spread
    return out


def serving(rg, ctx, plan, A, B, count, n_req=20000, n_warm=1000, tile=1):
    """Poisson stream of GEMM requests, shapes uniform over the grid cells, served by rg_serve with a
    64 GB budget through the smoothed plan (each request's leaves: autotuned variant, padding and
    splits); the rate is half the measured saturated capacity."""
    opts = rg.rg_serve_opts_default()
    opts.hbm_budget_bytes = 64 << 30
    opts.max_batch = 64
    opts.max_inflight = 2
    opts.tile = tile

    def trace(n, rate, seed):
        cells = synthetic.uniform_cells(n, (count, count, count), seed=seed)
        t = synthetic.poisson_arrivals(rate, n, seed=seed) if rate else np.zeros(n, np.int64)
        return [((int(a) + 1) * STEP, (int(b) + 1) * STEP, (int(c) + 1) * STEP, int(ti)) for (a, b, c), ti in
                zip(cells, t)]

    def run(tr):
        reqs = [(M, N, K, A, K, B, N, None, N, t) for M, N, K, t in tr]
        return rg.rg_serve(ctx, plan, opts, reqs)

    run(trace(500, None, 11))                                   # warm the graphs and clocks
    _, closed = run(trace(4000, None, 12))                      # all arrive at t = 0: saturated
    capacity = 4000 / closed["wall_s"]
    rate = 0.5 * capacity
    run(trace(n_warm, rate, 13))
    res, st = run(trace(n_req, rate, 14))
    ok = sum(1 for r in res if r["status"] == 0)
    leaves = [len(rg.rg_plan_lookup(plan, M, N, K)[0]) for M, N, K, _ in trace(n_req, rate, 14)]
    return {"requests": n_req, "served": ok, "warmup_requests": n_warm, "rate_req_per_s": rate,
            "saturated_capacity_req_per_s": capacity, "saturated_tflops": closed["tflops"],
            "p50_latency_us": st["p50_latency_us"], "p99_latency_us": st["p99_latency_us"],
            "mean_latency_us": st["mean_latency_us"], "tflops": st["tflops"], "batches": st["batches"],
            "admission_stalls": st["admission_stalls"], "hbm_budget_gb": 64,
            "routing": f"the smoothed plan ({rg.RG_NUM_VARIANTS}-variant autotune + DP pad/split): each request "
                       f"becomes its cell's leaves, phase by phase one grouped launch per kernel family "
                       f"(split-K and cta_group::2 items; stream-K choices run as their tile, split 1)",
            "multi_leaf_requests_share": float(np.mean(np.array(leaves) > 1)),
            "max_batch": opts.max_batch, "max_inflight": opts.max_inflight,
            "note": "latency = host-observed completion - arrival; outputs from a 64 GB arena"}


def fp8_landscape(rg, ctx, dev, count, p_bf16):
    """FP8 e4m3 block-scaled GEMM on the {512..4096 step 512}^3 subgrid: the autotune table over the
    twelve FP8 variants (128x256, 128x128 and the 256x256 cta_group::2 pair x split-K 1/2/4/8), the DP
    plan built from it, and the plan re-measured.  Returns the report block and the state the error
    check needs."""
    import torch
    Mx = STEP * count
    if Mx < 512:
        return None, None
    xa = torch.from_numpy(synthetic.normal_stream_f32(0, synthetic.TAG_A, Mx * Mx)).to(dev)
    xb = torch.from_numpy(synthetic.normal_stream_f32(0, synthetic.TAG_B, Mx * Mx)).to(dev)
    nb = Mx // 128
    qa = torch.empty(Mx * Mx, dtype=torch.uint8, device=dev)
    qb = torch.empty(Mx * Mx, dtype=torch.uint8, device=dev)
    sa = torch.empty(nb * nb, dtype=torch.float32, device=dev)
    sb = torch.empty(nb * nb, dtype=torch.float32, device=dev)
    rg.rg_fp8_quantize(ctx, xa, Mx, Mx, Mx, qa, Mx, sa)
    rg.rg_fp8_quantize(ctx, xb, Mx, Mx, Mx, qb, Mx, sb)
    del xa, xb
    C = torch.empty(Mx * Mx, dtype=torch.float32, device=dev)
    g = rg.make_grid((512, 512, Mx // 512))
    vids = [rg.fp8_variant(t, s) for t in range(rg.RG_FP8_NUM_TILES) for s in rg.SPLITS]
    t, tf, st = rg.rg_sweep_fp8_surfaces(ctx, g, vids, qa, sa, qb, sb, C)
    plan = rg.rg_plan_build(g, t, vids)
    tp, tfp, stp = rg.rg_sweep_fp8_surfaces(ctx, g, [0], qa, sa, qb, sb, C, plan=plan)
    cnt = Mx // 512
    sizes = (np.arange(1, cnt + 1) * 512).astype(np.int64)
    Mv, Nv, Kv = (x.ravel() for x in np.meshgrid(sizes, sizes, sizes, indexing="ij"))
    p_fp8 = 2.0 * p_bf16                  # no measured FP8 peak: the nominal 2x of the measured BF16 burst
    t_roof = 2.0 * Mv * Nv * Kv / (p_fp8 * 1e3)

    def block(row_t, row_tf, row_st):
        out = {k: float(row_st[i]) for i, k in enumerate(rg.SWEEP_STATS)}
        out.update({"p50_tflops": float(np.percentile(row_tf, 50)), "max_tflops": float(row_tf.max()),
                    "roofline_mean_frac_of_2x_bf16": float(np.mean(t_roof / row_t.astype(np.float64)))})
        return out
    tb = rg.rg_plan_tables(plan)
    fixed = vids.index(rg.fp8_variant(0, 1))
    best = t.min(axis=0)
    _, btf, bst = rg.rg_surface_stats(g, best)
    i4096 = int(np.argmax(Mv * Nv * Kv))
    out = {"grid": f"{{512..{Mx} step 512}}^3", "cells": int(t.shape[1]),
           "variants": [rg.fp8_variant_name(v) for v in vids],
           "fixed_128x256": block(t[fixed], tf[fixed], st[fixed]),
           "best_of_variants_table": {"mean_tflops": float(bst), "R_N_slice": float(btf["R_N_slice"]),
                               "R_3D": float(btf["R_3D"])},
           "plan_measured": block(tp[0], tfp[0], stp[0]),
           "winners": {rg.fp8_variant_name(v): float(np.mean(tb["vstar"].ravel() == v))
                       for v in sorted(set(tb["vstar"].ravel().tolist()))},
           "dp_actions": {a: float(np.mean(tb["action"] == i)) for i, a in enumerate(("keep", "M", "N", "K"))},
           "tflops_4096cube": {"fixed_128x256": float(tf[fixed][i4096]), "plan": float(tfp[0][i4096]),
                               "pair_256x256": float(tf[vids.index(rg.fp8_variant(rg.FP8_PAIR_TILE, 1))][i4096])},
           "peak_note": "FP8 roofline = 2 x the measured BF16 burst peak (the nominal ratio; no FP8 peak measured)",
           "scales": "per-128x128-block FP32 scales; the sweep reads compact scale arrays for each cell's "
                     "contiguous operand prefixes (timing only)"}
    state = {"plan": plan, "qa": qa, "qb": qb, "sa": sa, "sb": sb, "Mx": Mx, "cells": list(zip(Mv, Nv, Kv)), "C": C}
    return out, state


def fp8_errors(rg, ctx, state, dev, rows_per_cell=16):
    """Per-shape error of the FP8 plan against the oracle on every cell of the subgrid (CPU-baseline
    leg).  Cell (M, N, K) is the top-left M x K block of the quantised 4096^2 A and K x N block of B
    (lda = ldb = 4096, the whole scale arrays), so its 128 x 128 blocks and scales are exactly those
    of quantising that block; max |C - C64| / sum|a||b| over the whole matrix for cells up to 1024^3,
    over 16 seeded rows and 16 columns for larger ones."""
    import torch
    from oracle import fp8 as of
    from oracle import gemm as og
    Mx, plan = state["Mx"], state["plan"]
    nb = Mx // 128
    A = of.dequantize(state["qa"].cpu().numpy().reshape(Mx, Mx), state["sa"].cpu().numpy().reshape(nb, nb))
    B = of.dequantize(state["qb"].cpu().numpy().reshape(Mx, Mx), state["sb"].cpu().numpy().reshape(nb, nb))
    C = state["C"]
    rs = np.random.default_rng(0)
    ratios, worst = [], (0.0, None)
    for M, N, K in state["cells"]:
        M, N, K = int(M), int(N), int(K)
        Cv = C[:M * N].view(M, N)
        rg.rg_gemm_fp8_plan(ctx, plan, M, N, K, state["qa"], Mx, state["sa"], nb, state["qb"], Mx, state["sb"], nb,
                            Cv, N)
        rg.rg_check(ctx)
        a, b = A[:M, :K], B[:K, :N]
        if M * N * K <= 1024 ** 3:
            ratio, ez = og.error_ratio(Cv.cpu().numpy(), a @ b, np.abs(a) @ np.abs(b))
        else:
            rows = rs.choice(M, rows_per_cell, replace=False)
            cols = rs.choice(N, rows_per_cell, replace=False)
            cr, sr, cc, sc = og.sampled_rows_cols(a, b, rows, cols)
            r1, e1 = og.error_ratio(Cv[torch.as_tensor(rows, device=dev)].cpu().numpy(), cr, sr)
            r2, e2 = og.error_ratio(Cv[:, torch.as_tensor(cols, device=dev)].cpu().numpy(), cc, sc)
            ratio, ez = max(r1, r2), e1 and e2
        ratio = ratio if ez else float("inf")
        ratios.append(ratio)
        if ratio > worst[0]:
            worst = (ratio, [M, N, K])
    ratios = np.array(ratios)
    return {"cells": len(ratios), "max": float(ratios.max()), "median": float(np.median(ratios)),
            "p99": float(np.percentile(ratios, 99)), "worst_shape": worst[1],
            "bound_used_in_tests": "4 K 2^-24", "max_over_K_2^-24": float(max(
                r / (int(K) * 2.0 ** -24) for r, (_, _, K) in zip(ratios, state["cells"]))),
            "definition": "max |C - C64| / sum_k |a_ik||b_kj| against the float64 product of the dequantised "
                          "operands; whole matrix up to 1024^3, else 16 seeded rows and 16 columns"}


def e2e(rg, ctx, plan, a_bits, b_bits, dev, count, ncells=96):
    """The smoothed plan end to end through the C ABI on host buffers: rg_gemm_plan_host copies
    the cell's A and B from pinned host memory, executes the plan and copies C back to pinned
    host memory before it returns; timed on the host clock per call."""
    import torch
    cells = synthetic.uniform_cells(ncells, (count, count, count), seed=7)
    Mx = STEP * count
    ha = torch.from_numpy(a_bits.view(np.int16)).pin_memory()
    hb = torch.from_numpy(b_bits.view(np.int16)).pin_memory()
    hc = torch.empty(Mx * Mx, dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream()
    vals, h2d, d2h = [], 0, 0
    for rep in range(2):                              # the first pass grows the staging buffers and warms up
        vals = []
        h2d = d2h = 0
        for a, b, c in cells:
            M, N, K = (int(a) + 1) * STEP, (int(b) + 1) * STEP, (int(c) + 1) * STEP
            t0 = time.perf_counter()
            rg.rg_gemm_plan_host(ctx, plan, M, N, K, ha, K, hb, N, hc, N, stream=stream)
            dt = time.perf_counter() - t0
            vals.append(2.0 * M * N * K / dt / 1e12)
            h2d += 2 * M * K + 2 * K * N
            d2h += 4 * M * N
    return {"value": float(np.mean(vals)), "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "api": "rg_gemm_plan_host (C ABI, host buffers)",
            "sample": f"{ncells} cells drawn uniformly (seed 7); per cell one rg_gemm_plan_host call: pinned-host "
                      f"A, B -> device staging, plan GEMM, C -> pinned host, stream synchronised inside the call; "
                      f"host-clock time per call; mean per-cell TFLOP/s"}


if __name__ == "__main__":
    sys.exit(main())

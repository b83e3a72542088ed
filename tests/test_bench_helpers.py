"""The bench's reporting helpers on the CPU: the sawtooth period of a
cross-tile N series, the rank transform behind the run-order Spearman
correlation, the surface summary and the host-step timing record."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("period", [2, 3, 4, 5, 8])
def test_sawtooth_period_recovers_a_planted_period(period):
    n = np.arange(64)
    series = 1000.0 + 5.0 * n - 40.0 * ((n % period) == 0)   # a dip every `period` steps on a ramp
    lag, corr = bench.sawtooth_period(series)
    assert lag == period and corr > 0.5


def test_sawtooth_period_of_noise_has_no_strong_period():
    rs = np.random.default_rng(3)
    lag, corr = bench.sawtooth_period(np.cumsum(rs.normal(size=200)))   # random walk: white-noise steps
    assert abs(corr) < 0.3


def test_ranks_give_spearman():
    x = np.array([3.0, 1.0, 2.0, 10.0])
    assert list(bench._ranks(x)) == [2.0, 0.0, 1.0, 3.0]
    y = x ** 3                                   # monotone transform: rank correlation 1
    assert np.corrcoef(bench._ranks(x), bench._ranks(y))[0, 1] == pytest.approx(1.0)


def test_summarize_keys_and_percentiles():
    tf = np.arange(1.0, 101.0)
    r = {"R_N_slice": 1.0, "R_3D": 2.0, "R_M": 3.0, "R_N": 4.0, "R_K": 5.0}
    s = bench.summarize(tf, r, 50.5)
    assert s["mean_tflops"] == 50.5 and s["max_tflops"] == 100.0
    assert s["p50_tflops"] == pytest.approx(50.5) and s["R_K"] == 5.0


def test_host_steps_timing_record():
    pytest.importorskip("paper_2605_29752_gb300.rg")
    rec = bench.host_steps_timing(4, seed=1)["host_steps"]
    assert set(rec) == {"table", "oracle_dp_s", "oracle_roughness_s", "library_plan_build_s", "library_surface_stats_s"}
    assert all(rec[k] >= 0 for k in rec if k != "table")


def test_roof_times_pick_the_binding_limit():
    # P = 1000 TFLOP/s, BW = 1000 GB/s: a 4096^3 cell is compute-bound, a 128 x 128 x 4096 cell memory-bound
    t = bench.roof_times_ns([4096, 128], [4096, 128], [4096, 4096], 1000.0, 1000.0)
    assert t[0] == pytest.approx(2.0 * 4096 ** 3 / 1e6)
    assert t[1] == pytest.approx((2 * 128 * 4096 * 2 + 4 * 128 * 128) / 1000.0)


def test_summarize_reports_the_mean_roofline_fraction():
    tf = np.array([1.0, 2.0, 3.0])
    r = {"R_N_slice": 1.0, "R_3D": 1.0, "R_M": 1.0, "R_N": 1.0, "R_K": 1.0}
    s = bench.summarize(tf, r, 2.0, t_ns=np.array([10, 20, 40]), troof=np.array([5.0, 5.0, 5.0]))
    assert s["roofline_mean_frac"] == pytest.approx((0.5 + 0.25 + 0.125) / 3)
    assert s["R_N_slice_over_mean"] == 0.5


def test_slice_attribution_splits_the_slice_roughness_by_regime():
    count = 4
    tf = np.zeros((count, count, count))
    tf[:, :, -1] = np.arange(count)[None, :] * 10.0            # |dN| = 10 everywhere on the K = max slice
    out = bench.slice_attribution(tf.ravel(), count, 512)
    total = sum(v["contribution_to_R_N_slice"] for v in out.values())
    assert total == pytest.approx(10.0)                          # the slice's R_N, split without loss
    assert sum(v["pair_share"] for v in out.values()) == pytest.approx(1.0)


def test_noise_floor_of_identical_repeats_is_zero_and_scales():
    rs = np.random.default_rng(0)
    a = rs.uniform(100, 200, size=4 ** 3)
    assert bench.noise_floor(a, a, 4)["R_N_slice"] == 0.0
    b = a + np.where(np.arange(a.size) % 2 == 0, 1.0, -1.0)     # alternating +-1 difference
    nf = bench.noise_floor(a, b, 4)
    assert nf["R_3D"] >= 0.0 and nf["R_N_slice"] >= 0.0


def test_phase_summary_skips_stamps_a_cta_never_reached():
    """Phase medians of the phase-timer records: a phase counts only the CTAs that reached both of its
    stamps (the odd CTA of a cta_group::2 pair issues no MMAs; only last arrivers run a fixup)."""
    rec = np.zeros((4, 12), np.uint64)
    rec[:, 0], rec[:, 1], rec[:, 2] = 1000, 3000, 4000          # 2000 ns over 4000 cycles: 0.5 ns / cycle
    rec[:, 3], rec[:, 7], rec[:, 10] = 100, 3000, 1
    rec[:2, 4], rec[:2, 5] = 200, 1200                           # only the even CTAs issue MMAs
    rec[1, 8], rec[1, 9] = 2000, 2600                            # one fixup
    out = bench.phase_summary(rec)
    assert out["first_stage_to_last_mma_commit_ns"] == 500.0 and out["first_stage_to_last_mma_commit_ctas"] == 2
    assert out["fixup_ns"] == 300.0 and out["fixup_ctas"] == 1
    assert out["cta_total_ns"] == 2000.0 and out["launch_span_ns"] == 2000.0
    assert out["first_release_to_last_exit_ns"] == 1950.0 and out["release_skew_ns"] == 0.0

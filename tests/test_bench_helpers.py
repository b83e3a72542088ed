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

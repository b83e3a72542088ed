"""Pins for oracle.landscape against the paper's worked numbers (Sec. 3.3, 9, 10)."""
import json
import os

import pytest

from oracle import landscape

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_partial_tile_utilization():
    g = GOLD["partial_tile_utilization"]
    for n, u in g["cases"]:
        assert landscape.tile_utilization(n, g["tile"]) == u


def test_wave_efficiency_21_on_20():
    g = GOLD["wave_efficiency"]
    eta = landscape.wave_efficiency(g["w"], g["c"])
    assert eta == 21 / 40 and int(100 * eta + 0.5) == g["printed_percent"]   # 52.5 printed as 53


def test_channel_eta_one_third_at_multiples_of_768():
    g = GOLD["channel_eta_B"]
    for n in g["n_values"]:
        assert landscape.eta_channel(n, 2) == pytest.approx(g["eta"], abs=1e-15)
    assert landscape.eta_channel(1024, 2) > g["eta"]


def test_peak_and_ridge():
    g = GOLD["peak_derivation"]
    p = landscape.peak_from_units(g["units"], g["engines"], g["macs_per_clk"], g["ghz"])
    assert abs(p - g["printed_tflops"]) < 0.1
    r = GOLD["ridge"]
    assert round(r["p_tflops"] * 1e12 / (r["bw_gbs"] * 1e9)) == r["printed"]


def test_kol_table_20():
    g = GOLD["kol_table_20"]
    for row in g["rows"]:
        t = landscape.throughput_band(row["tau"])
        s = landscape.smoothness_band(row["rho"])
        assert (t, s, min(t, s)) == (row["T"], row["S"], row["L"]), row["kernel"]
    td = g["tau_dp"]
    k = landscape.kol(td["mean_a"], td["mean_o"], 5.0, 5.0 / 1.8)
    assert round(k["tau"], 3) == td["printed"] and k["L"] == 2


def test_band_edges():
    assert [landscape.throughput_band(x) for x in (0.49, 0.5, 0.749, 0.75, 0.9499, 0.95)] == [0, 1, 1, 2, 2, 3]
    assert [landscape.smoothness_band(x) for x in (3.01, 3.0, 2.0, 1.26, 1.25, 1.0)] == [0, 1, 2, 2, 3, 3]


def test_optimal_reduces_to_ideal_when_memory_is_free_and_one_tile():
    # with one tile and unbounded bandwidth the optimal is P * eta_wave, which equals the
    # ideal P * min(1, W/C) whenever W <= C (a single partial wave)
    grid = ((128, 128, 4), (128, 128, 4), (128, 128, 2))
    opt = landscape.optimal_surface(grid, 100.0, 20, [(256, 256)], 1e12)
    ide = landscape.ideal_surface(grid, 100.0, 20, (256, 256))
    assert abs(opt - ide).max() < 1e-9


def test_optimal_memory_bound_small_shape():
    # a 128^3 problem on the paper's constants is bound by memory: 2MNK / t_mem
    M = N = K = 128
    t_mem = (2 * M * K + 2 * K * N + 4 * M * N) / 451e9
    v = landscape.optimal_cell(M, N, K, 108.2, 20, [(256, 256), (128, 128), (64, 64)], 451.0)
    assert abs(v - 2 * M * N * K / t_mem / 1e12) < 1e-9


PAPER_SIX = [(128, 64), (128, 128), (128, 256), (256, 64), (256, 128), (256, 256)]


def test_optimal_hand_worked_multi_tile_cell_on_gb300_constants():
    """M = 2048, N = 1536, K = 4096 on P = 1919.8 TFLOP/s, C = 152, BW = 6789.6 GB/s, the paper's six tiles
    (Sec. 9.2), worked by hand.  Tile counts W = ceil(M/TM) ceil(N/TN) and wave efficiencies W / (ceil(W/C) C):
    128x64 -> 16 * 24 = 384, three waves of 152, eta = 384/456 = 16/19; 128x128 -> 192 and 256x64 -> 192,
    two waves, eta = 12/19; 128x256 -> 96 and 256x128 -> 96, eta = 12/19; 256x256 -> 48, eta = 6/19.
    The best tile is 128x64: t_comp = 2MNK / (P 16/19) = 15.94 us, above t_mem = (2MK + 2KN + 4MN) / BW =
    41,943,040 B / 6789.6 GB/s = 6.18 us, so the cell reaches P * 16/19.  (A min in place of the max, the
    worst tile in place of the best, or another wave formula each give a different value.)"""
    v = landscape.optimal_cell(2048, 1536, 4096, 1919.8, 152, PAPER_SIX, 6789.6)
    assert abs(v - 1919.8 * 16 / 19) < 1e-9


def test_optimal_hand_worked_memory_bound_multi_tile_cell():
    """M = 2048, N = 1536, K = 128 on the same constants: the best tile is again 128x64 (eta = 16/19), whose
    t_comp = 2MNK / (P 16/19) = 0.498 us is below t_mem = (2MK + 2KN + 4MN) / BW = 13,500,416 B / 6789.6 GB/s =
    1.988 us, so every tile is memory-bound and the cell reaches 2MNK BW / bytes = 405.00 TFLOP/s."""
    v = landscape.optimal_cell(2048, 1536, 128, 1919.8, 152, PAPER_SIX, 6789.6)
    expect = 2 * 2048 * 1536 * 128 * 6789.6e9 / 13_500_416 / 1e12
    assert abs(v - expect) < 1e-9 and abs(expect - 405.0) < 0.01

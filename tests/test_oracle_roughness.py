"""Pins for oracle.roughness (Sec. 2 definitions; Sec. 8.6 conventions)."""
import json
import math
import os
from fractions import Fraction

import numpy as np

from oracle import landscape, roughness

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_roughness_1d_by_hand():
    assert roughness.roughness_1d([1.0, 3.0, 2.0, 5.0]) == 2.0        # (2 + 1 + 3) / 3
    assert roughness.roughness_1d([4.0]) == 0.0


def test_constant_surface_is_smooth():
    S = np.full((5, 6, 7), 3.25)
    r = roughness.roughness_all(S)
    assert r == {"R_M": 0.0, "R_N": 0.0, "R_K": 0.0, "R_3D": 0.0, "R_N_slice": 0.0}


def test_linear_surface_closed_form():
    a, b, c = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    S = 1.5 * a - 0.25 * b + 2.0 * c + 10.0
    r = roughness.roughness_all(S)
    assert r["R_M"] == 1.5 and r["R_N"] == 0.25 and r["R_K"] == 2.0
    assert r["R_3D"] == (1.5 + 0.25 + 2.0) / 3 and r["R_N_slice"] == 0.25


def test_pooled_equals_mean_of_lines():
    rng = np.random.default_rng(3)
    S = rng.uniform(0, 100, size=(6, 7, 5))
    pooled = roughness.roughness_axis(S, 1)
    lines = [roughness.roughness_1d(S[i, :, k]) for i in range(6) for k in range(5)]
    assert abs(pooled - sum(lines) / len(lines)) < 1e-12


def test_sum_is_correctly_rounded():
    # terms whose naive left-to-right float sum is wrong; compare with the exact rational sum
    vals = [1e16, 1.0, 1.0, 1.0, 1.0, 3.0, 1e-3, 2.0 ** -40]
    line = [0.0]
    for i, v in enumerate(vals):                 # alternate up and down steps
        line.append(line[-1] + (v if i % 2 == 0 else -v))
    diffs = [abs(line[i + 1] - line[i]) for i in range(len(line) - 1)]
    exact = sum(Fraction(d) for d in diffs) / len(diffs)
    assert roughness.roughness_1d(line) == float(Fraction(math.fsum(diffs)) / len(diffs))
    assert math.fsum(diffs) == float(sum(Fraction(d) for d in diffs))
    assert abs(roughness.roughness_1d(line) - float(exact)) <= abs(float(exact)) * 2.0 ** -52


def test_tflops_definition():
    # 2 * 4096^3 flops in 1 ms = 137.438953472 TFLOP/s exactly
    assert roughness.tflops(4096, 4096, 4096, 1_000_000) == 137.438953472
    grid = ((128, 128, 2), (128, 128, 1), (128, 128, 1))
    S = roughness.surface(np.array([[[2000]], [[1000]]]), grid)
    assert S[0, 0, 0] == 2.0 * 128 ** 3 / 2e6 and S[1, 0, 0] == 2.0 * 256 * 128 * 128 / 1e6


def test_mean_correctly_rounded():
    assert roughness.mean(np.array([1e16, 1.0, -1e16, 1.0])) == 0.5


def test_ideal_landscape_matches_printed_values():
    g = GOLD["ideal_landscape"]
    grid = ((128, 128, 32), (128, 128, 32), (128, 128, 32))
    S = landscape.ideal_surface(grid, g["p_tflops"], g["c_units"], (g["tile"], g["tile"]))
    r = roughness.roughness_all(S)
    assert round(roughness.mean(S), 1) == g["printed_mean"]
    assert round(r["R_N_slice"], 1) == g["printed_roughness_slice"]
    assert abs(roughness.mean(S) - 97.169) < 5e-4 and abs(r["R_N_slice"] - 1.963) < 5e-4
    assert r["R_K"] == 0.0                    # the ideal does not depend on K

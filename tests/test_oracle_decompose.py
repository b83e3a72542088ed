"""Pins for oracle.decompose (Sec. 4 four-surface decomposition, Table 3
classification): a worked two-cell example done by hand, exact rational
arithmetic for the compute surface and the classification, and the special
cases the definitions reduce to."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import decompose as od


def test_compute_surface_hand_values():
    # 2 * 128^3 = 4,194,304 flops at 1 TFLOP/s = 4194.304 ns
    assert od.compute_ns(128, 128, 128, 1.0) == 4194.304
    # 2 * 4096^3 = 137,438,953,472 flops at 1900.7 TFLOP/s: the float64 result is the
    # rational value 137438953472 / 1900700 ns rounded once
    exact = Fraction(137438953472, 1900700)
    got = od.compute_ns(4096, 4096, 4096, 1900.7)
    assert abs(Fraction(got) - exact) <= exact * Fraction(1, 2 ** 51)


def test_two_cell_worked_example():
    # cell 1 (128,128,128): t_c = 4194.304 > t_mem = 3000 -> compute-bound,
    #   overhead = 10000 - 4194.304 = 5805.696
    # cell 2 (128,128,256): t_c = 8388.608 < t_mem = 9500 -> memory-bound,
    #   overhead = 9000 - 9500 = -500
    comp, over, st = od.decompose([128], [128], [128, 256], [10000, 9000], [3000, 9500], 1.0)
    assert comp.ravel().tolist() == [4194.304, 8388.608]
    assert over.ravel() == pytest.approx([5805.696, -500.0], abs=1e-9)
    assert st[0] == 0.5
    assert st[1] == pytest.approx((0.5805696 - 500 / 9000) / 2, abs=1e-15)
    assert st[2] == pytest.approx(5305.696 / 19000, abs=1e-15)
    assert st[3] == pytest.approx((0.3 + 9500 / 9000) / 2, abs=1e-15)


def test_free_memory_leaves_gemm_minus_compute():
    ms, ns, ks = [128, 256], [128, 384], [256, 512, 1024]
    rng = np.random.default_rng(1)
    tg = rng.integers(100_000, 900_000, size=(2, 2, 3))
    tm = np.ones_like(tg)                              # memory time 1 ns: below every compute time
    comp, over, st = od.decompose(ms, ns, ks, tg, tm, 10.0)
    for a, M in enumerate(ms):
        for b, N in enumerate(ns):
            for c, K in enumerate(ks):
                exact = Fraction(2 * M * N * K, 10_000)   # ns at 10 TFLOP/s
                assert abs(Fraction(comp[a, b, c]) - exact) <= exact * Fraction(1, 2 ** 51)
                assert over[a, b, c] == tg[a, b, c] - comp[a, b, c]
    assert st[0] == 1.0


def test_classification_matches_exact_rational_comparison():
    """Table 3: with an analytic memory time (algorithmic bytes over a bandwidth,
    rounded to ns) the compute-bound cells are exactly those where 2MNK / P exceeds
    it, decided here in rational arithmetic; and nearly all of them lie above the
    ridge P / BW in arithmetic intensity."""
    v = list(range(128, 2049, 128))
    P, BW = 1900.7, 6663.9                             # TFLOP/s, GB/s
    shape = (len(v),) * 3
    tm = np.zeros(shape, np.int64)
    above_ridge = 0
    for a, M in enumerate(v):
        for b, N in enumerate(v):
            for c, K in enumerate(v):
                by = 2 * M * K + 2 * K * N + 4 * M * N
                tm[a, b, c] = max(1, round(by / BW))   # bytes / (GB/s) = ns
                above_ridge += Fraction(2 * M * N * K, by) > Fraction(19007, 66639) * 1000
    tg = tm + 1000
    _, _, st = od.decompose(v, v, v, tg, tm, P)
    exact = 0
    for a, M in enumerate(v):
        for b, N in enumerate(v):
            for c, K in enumerate(v):
                exact += Fraction(2 * M * N * K) / (Fraction(19007, 10) * 1000) > tm[a, b, c]
    assert st[0] == exact / tm.size
    assert abs(exact - above_ridge) <= 0.01 * tm.size


def test_overhead_identity_and_rejections():
    rng = np.random.default_rng(5)
    tg = rng.integers(1, 10 ** 6, size=(3, 2, 2))
    tm = rng.integers(1, 10 ** 6, size=(3, 2, 2))
    comp, over, _ = od.decompose([128, 256, 384], [128, 256], [128, 4096], tg, tm, 100.0)
    assert np.array_equal(over + np.maximum(comp, tm), tg.astype(np.float64))
    with pytest.raises(ValueError):
        od.decompose([128], [128], [128], [0], [1], 1.0)

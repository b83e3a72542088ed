"""Pins for oracle.dp: exhaustive search on tiny grids, a fixpoint closure,
closed forms, invariants and special cases (Sec. 7.1)."""
import itertools
import random

import numpy as np
import pytest

from oracle import dp


def _grid(nm, nn, nk, step=128):
    return ((step, step, nm), (step, step, nn), (step, step, nk))


def _cells(shape):
    return list(itertools.product(*[range(s) for s in shape]))


def _rand_T0(rng, shape, lo=1, hi=60):
    return np.array([rng.randint(lo, hi) for _ in range(int(np.prod(shape)))], dtype=np.int64).reshape(shape)


# ---------- independent references ----------

def _pad_closed_form(T0s):
    """T1[c] = min over every cell c' >= c componentwise of T0*[c'] (brute force)."""
    out = np.zeros_like(T0s)
    for c in _cells(T0s.shape):
        out[c] = min(T0s[d] for d in _cells(T0s.shape) if all(d[x] >= c[x] for x in range(3)))
    return out


def _split_options(cell):
    a, b, c = cell
    p = (a + 1, b + 1, c + 1)
    for axis in range(3):
        for q in range(1, p[axis]):
            first = list(cell)
            second = list(cell)
            first[axis] = p[axis] - q - 1
            second[axis] = q - 1
            yield tuple(first), tuple(second)


def _all_tree_costs(cell, leaf_cost):
    """Every binary split tree of ``cell`` written out, each leaf padded optimally: yields costs."""
    yield leaf_cost[cell]
    for p1, p2 in _split_options(cell):
        for x in _all_tree_costs(p1, leaf_cost):
            for y in _all_tree_costs(p2, leaf_cost):
                yield x + y


def _closure(T0s):
    """Relax padding (any dominating cell) and splitting (any cut) until nothing changes."""
    T = {c: int(T0s[c]) for c in _cells(T0s.shape)}
    while True:
        old = dict(T)
        for c in T:
            for d in T:
                if all(d[x] >= c[x] for x in range(3)):
                    T[c] = min(T[c], T[d])
        for c in T:
            for p1, p2 in _split_options(c):
                T[c] = min(T[c], T[p1] + T[p2])
        if T == old:
            return T


# ---------- tests ----------

def test_best_of_min_and_lowest_id_on_ties():
    T0v = np.array([[[[5, 7]]], [[[5, 3]]], [[[4, 3]]]], dtype=np.int64)   # V=3, cells (1,1,2)
    best, arg = dp.best_of(T0v)
    assert best.tolist() == [[[4, 3]]]
    assert arg.tolist() == [[[2, 1]]]


@pytest.mark.parametrize("seed", range(40))
def test_T1_equals_dominance_closed_form(seed):
    rng = random.Random(seed)
    shape = (rng.randint(1, 4), rng.randint(1, 4), rng.randint(1, 4))
    T0s = _rand_T0(rng, shape)
    T1, tgt = dp.pad_T1(T0s, _grid(*shape))
    assert np.array_equal(T1, _pad_closed_form(T0s))
    for c in _cells(shape):
        t = tuple(int(x) for x in tgt[c])
        assert all(t[x] >= c[x] for x in range(3))
        assert T0s[t] == T1[c]


@pytest.mark.parametrize("shape", [(1, 1, 2), (2, 1, 1), (2, 2, 1), (2, 2, 2), (3, 2, 1), (1, 3, 2)])
@pytest.mark.parametrize("seed", range(6))
def test_T2_equals_exhaustive_tree_search(shape, seed):
    rng = random.Random(1000 + seed)
    T0s = _rand_T0(rng, shape)
    T1, _ = dp.pad_T1(T0s, _grid(*shape))
    T2, _, _ = dp.split_T2(T1, _grid(*shape))
    leaf_cost = {c: int(x) for c, x in zip(_cells(shape), _pad_closed_form(T0s).ravel())}
    for c in _cells(shape):
        assert T2[c] == min(_all_tree_costs(c, leaf_cost)), c


@pytest.mark.parametrize("seed", range(60))
def test_T2_equals_fixpoint_closure(seed):
    rng = random.Random(seed)
    n = rng.choice((2, 3, 4))
    shape = (n, rng.randint(1, n), rng.randint(1, n))
    T0s = _rand_T0(rng, shape)
    T1, _ = dp.pad_T1(T0s, _grid(*shape))
    T2, _, _ = dp.split_T2(T1, _grid(*shape))
    cl = _closure(T0s)
    assert all(T2[c] == cl[c] for c in _cells(shape))


@pytest.mark.parametrize("seed", range(20))
def test_invariants(seed):
    rng = random.Random(seed)
    shape = (rng.randint(2, 6), rng.randint(2, 6), rng.randint(2, 6))
    T0s = _rand_T0(rng, shape, 1, 1000)
    T1, _ = dp.pad_T1(T0s, _grid(*shape))
    T2, _, _ = dp.split_T2(T1, _grid(*shape))
    assert np.all(T2 <= T1) and np.all(T1 <= T0s)
    for ax in range(3):
        assert np.all(np.diff(T1, axis=ax) >= 0)          # padding only helps smaller cells
    for c in _cells(shape):                                 # subadditive along every axis
        for p1, p2 in _split_options(c):
            assert T2[c] <= T2[p1] + T2[p2]


def _check_leaves(pl, grid, shape):
    step = grid[0][1]
    for c in _cells(shape):
        lv = pl["leaves"][c]
        M, N, K = ((c[i] + 1) * step for i in range(3))
        # cost additivity: the leaves' T1 times add up to T2
        cost = 0
        for (v, beta, phase, m0, n0, k0, m, n, k, pm, pn, pk) in lv:
            cell = (m // step - 1, n // step - 1, k // step - 1)
            tgt = (pm // step - 1, pn // step - 1, pk // step - 1)
            assert pl["T1"][cell] == pl["T0s"][tgt] and v == pl["vstar"][tgt]
            assert pm >= m and pn >= n and pk >= k
            cost += int(pl["T1"][cell])
        assert cost == pl["T2"][c]
        # the boxes tile M x N x K exactly once; per output element the K pieces
        # run in increasing phase, the first with beta 0, the rest with beta 1
        cover = np.zeros((M // step, N // step, K // step), dtype=np.int64)
        per_out = {}
        for (v, beta, phase, m0, n0, k0, m, n, k, pm, pn, pk) in lv:
            cover[m0 // step:(m0 + m) // step, n0 // step:(n0 + n) // step, k0 // step:(k0 + k) // step] += 1
            for i in range(m0 // step, (m0 + m) // step):
                for j in range(n0 // step, (n0 + n) // step):
                    per_out.setdefault((i, j), []).append((k0, phase, beta))
        assert np.all(cover == 1)
        for pieces in per_out.values():
            pieces.sort()
            assert pieces[0][0] == 0 and pieces[0][2] == 0
            assert all(p[2] == 1 for p in pieces[1:])
            assert all(pieces[i][1] < pieces[i + 1][1] for i in range(len(pieces) - 1))


@pytest.mark.parametrize("seed", range(15))
def test_leaves_cover_and_add_up(seed):
    rng = random.Random(seed)
    shape = (rng.randint(1, 5), rng.randint(1, 5), rng.randint(1, 5))
    V = rng.randint(1, 4)
    T0v = np.stack([_rand_T0(rng, shape, 5, 80) for _ in range(V)])
    grid = _grid(*shape)
    pl = dp.plan(T0v, grid)
    _check_leaves(pl, grid, shape)


def test_superadditive_increasing_keeps_everything():
    shape = (4, 4, 4)
    grid = _grid(*shape)
    T0 = np.zeros(shape, dtype=np.int64)
    for a, b, c in _cells(shape):
        T0[a, b, c] = 1000 + (a + 1) * (b + 1) * (c + 1)
    pl = dp.plan(T0[None], grid)
    assert np.array_equal(pl["T1"], T0) and np.array_equal(pl["T2"], T0)
    assert np.all(pl["action"] == dp.KEEP)
    for c in _cells(shape):
        assert tuple(pl["target"][c]) == c


def test_additive_time_ties_keep_as_is():
    shape = (3, 3, 3)
    T0 = np.zeros(shape, dtype=np.int64)
    for a, b, c in _cells(shape):
        T0[a, b, c] = (a + 1) * (b + 1) * (c + 1)           # every split ties exactly
    pl = dp.plan(T0[None], _grid(*shape))
    assert np.all(pl["action"] == dp.KEEP) and np.array_equal(pl["T2"], T0)


def test_constant_time_no_split_no_pad():
    shape = (3, 2, 3)
    T0 = np.full(shape, 77, dtype=np.int64)
    pl = dp.plan(T0[None], _grid(*shape))
    assert np.all(pl["action"] == dp.KEEP) and np.all(pl["T2"] == 77)
    for c in _cells(shape):
        assert tuple(pl["target"][c]) == c                  # as-is wins the volume tie-break


def test_one_bad_cell_pads_to_cheapest_dominating_neighbour():
    shape = (3, 3, 3)
    T0 = np.zeros(shape, dtype=np.int64)
    for a, b, c in _cells(shape):
        T0[a, b, c] = 100 * (a + 1) * (b + 1) * (c + 1) + 50
    T0[1, 1, 1] = 10 ** 9
    T0[1, 2, 1] = 700                                         # cheaper than the bad cell's others
    pl = dp.plan(T0[None], _grid(*shape))
    assert tuple(pl["target"][1, 1, 1]) == (1, 2, 1) and pl["T1"][1, 1, 1] == 700


def test_split_k_chain_beta_and_phase():
    # only the K axis is long; make K-splits strictly better than the whole
    shape = (1, 1, 4)
    T0 = np.array([[[10, 100, 100, 1000]]], dtype=np.int64)
    pl = dp.plan(T0[None], _grid(*shape))
    lv = pl["leaves"][(0, 0, 3)]
    assert pl["T2"][0, 0, 3] == 40 and len(lv) == 4
    assert [l[5] for l in lv] == [0, 128, 256, 384]           # k0 in order
    assert [l[1] for l in lv] == [0, 1, 1, 1]                 # beta
    assert [l[2] for l in lv] == [0, 1, 2, 3]                 # phase


@pytest.mark.slow
def test_full_grid_runs_and_is_consistent():
    rng = np.random.default_rng(0)
    shape = (32, 32, 32)
    grid = _grid(*shape)
    M = (np.arange(32) + 1)[:, None, None] * 128.0
    N = (np.arange(32) + 1)[None, :, None] * 128.0
    K = (np.arange(32) + 1)[None, None, :] * 128.0
    base = 3000 + 2 * M * N * K / 1.2e6
    T0v = np.stack([np.round(base * rng.uniform(0.8, 1.6, size=shape)).astype(np.int64) for _ in range(3)])
    pl = dp.plan(T0v, grid)
    assert np.all(pl["T2"] <= pl["T1"]) and np.all(pl["T1"] <= pl["T0s"])
    assert np.any(pl["action"] != dp.KEEP)

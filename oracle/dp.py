"""O-DP: dynamic best-of-tiles selection and the padding-and-splitting dynamic
programme T0 -> T1 -> T2 (Sec. 6.4 "Dynamic Best-of-Six Tile Selection";
Sec. 7.1 "The T0 -> T1 -> T2 Algorithm", Eq. for T1 and the T2 recurrence;
split semantics of Sec. 7.1, Figs. 14-16).

Test infrastructure only (see the package docstring).

Grid.  An axis is (start, step, count); cell index a in [0, count) stands for
the size start + a*step.  The paper's grid is start = step = 128, count = 32
on all three axes.  Splitting needs start == step so that sizes are whole
multiples of the step: a cell with 1-based size p = a + 1 (in steps) splits
into pieces of p - q and q steps, q = 1 .. p - 1.

Readings taken where the paper is silent (each is a total order, so every
correct implementation produces the same tables):
  * Times are integers (nanoseconds); min and + are exact.
  * Best-of selection: T0*[c] = min over variants v of T0[v][c]; ties go to
    the lowest variant id (variants are numbered tile-major, then split
    factor).
  * "M + 1" in the T1 formula is one grid step; cells outside the grid do
    not exist (no padding beyond the last grid value).
  * T1 pad target: among all cells c' >= c (componentwise) the minimiser of
    (T0*[c'], M'N'K', M', N', K') lexicographically; "as-is" (c' = c) wins
    every tie because it has the smallest volume.
  * T2 action: the minimiser of (value, rank, q) where rank 0 = keep the T1
    choice (pad or as-is), 1 = split M, 2 = split N, 3 = split K (the order
    of the terms in the paper's recurrence), q = size of the second piece in
    steps, smallest first.  A split replaces the T1 choice only when strictly
    faster.
  * Split pieces: piece 1 = the first p - q steps of the axis, piece 2 = the
    last q steps.  For a K split, piece 2 accumulates into C (beta = 1) and
    runs after piece 1 (Sec. 7.1: the two GEMMs run one after the other and
    the second adds into C); piece 1 inherits the parent's beta.
  * Cost model: a split's time is the sum of its pieces' times (the paper's
    sequential execution).
"""
from __future__ import annotations

import itertools

import numpy as np

KEEP, SPLIT_M, SPLIT_N, SPLIT_K = 0, 1, 2, 3


def axis_values(axis):
    start, step, count = axis
    return [start + i * step for i in range(count)]


def best_of(T0v: np.ndarray):
    """T0*[c] = min_v T0[v][c] and its argmin (lowest v on ties).  T0v has shape (V, nm, nn, nk)."""
    T0v = np.asarray(T0v, dtype=np.int64)
    V = T0v.shape[0]
    best = T0v[0].copy()
    arg = np.zeros(best.shape, dtype=np.int64)
    for v in range(1, V):
        better = T0v[v] < best          # strict: an equal later variant never wins
        best[better] = T0v[v][better]
        arg[better] = v
    return best, arg


def pad_T1(T0s: np.ndarray, grid):
    """T1 by the paper's sweep from the last cell back to the first:
    T1[m][n][k] = min over (i, j, l) in {0,1}^3 of T1[m+i][n+j][k+l], starting
    from T1 = T0*.  Returns (T1, target) with target[c] = the padded cell (a', b', c')."""
    T0s = np.asarray(T0s, dtype=np.int64)
    nm, nn, nk = T0s.shape
    Mv, Nv, Kv = (axis_values(ax) for ax in grid)

    def key_of(cell):
        a, b, c = cell
        return (int(T0s[a, b, c]), Mv[a] * Nv[b] * Kv[c], Mv[a], Nv[b], Kv[c])

    best_key = {}
    target = {}
    for a in reversed(range(nm)):
        for b in reversed(range(nn)):
            for c in reversed(range(nk)):
                cur_key = key_of((a, b, c))
                cur_tgt = (a, b, c)
                for i, j, l in itertools.product((0, 1), repeat=3):
                    if (i, j, l) == (0, 0, 0):
                        continue
                    nb = (a + i, b + j, c + l)
                    if nb[0] >= nm or nb[1] >= nn or nb[2] >= nk:
                        continue
                    if best_key[nb] < cur_key:
                        cur_key = best_key[nb]
                        cur_tgt = target[nb]
                best_key[(a, b, c)] = cur_key
                target[(a, b, c)] = cur_tgt
    T1 = np.zeros_like(T0s)
    tgt = np.zeros(T0s.shape + (3,), dtype=np.int64)
    for cell, k in best_key.items():
        T1[cell] = k[0]
        tgt[cell] = target[cell]
    return T1, tgt


def split_T2(T1: np.ndarray, grid):
    """T2 by the paper's sweep from the first cell to the last, starting from T2 = T1:
    T2[M][N][K] = min(T2[M][N][K], min_i T2[M-i][N][K] + T2[i][N][K],
                      min_j T2[M][N-j][K] + T2[M][j][K], min_k T2[M][N][K-k] + T2[M][N][k]).
    Returns (T2, action, q)."""
    for ax in grid:
        if ax[0] != ax[1]:
            raise ValueError("splitting needs grid start == step on every axis")
    T1 = np.asarray(T1, dtype=np.int64)
    nm, nn, nk = T1.shape
    T2 = [[[int(T1[a, b, c]) for c in range(nk)] for b in range(nn)] for a in range(nm)]
    action = np.zeros(T1.shape, dtype=np.int64)
    qarg = np.zeros(T1.shape, dtype=np.int64)
    for a in range(nm):
        for b in range(nn):
            for c in range(nk):
                best = T2[a][b][c]
                act, qq = KEEP, 0
                p = a + 1
                for q in range(1, p):                 # split M: pieces p-q and q
                    v = T2[p - q - 1][b][c] + T2[q - 1][b][c]
                    if v < best:
                        best, act, qq = v, SPLIT_M, q
                p = b + 1
                for q in range(1, p):                 # split N
                    v = T2[a][p - q - 1][c] + T2[a][q - 1][c]
                    if v < best:
                        best, act, qq = v, SPLIT_N, q
                p = c + 1
                for q in range(1, p):                 # split K
                    v = T2[a][b][p - q - 1] + T2[a][b][q - 1]
                    if v < best:
                        best, act, qq = v, SPLIT_K, q
                T2[a][b][c] = best
                action[a, b, c] = act
                qarg[a, b, c] = qq
    return np.array(T2, dtype=np.int64), action, qarg


def leaves(cell, grid, action, qarg, target, vstar):
    """Expand one cell's plan into its leaf sub-GEMMs, in execution order.

    A leaf is a tuple (variant, beta, phase, m0, n0, k0, m, n, k, pm, pn, pk):
    the box [m0, m0+m) x [n0, n0+n) x [k0, k0+k) of the original problem, run
    as if it were the padded problem pm x pn x pk with the variant measured
    fastest there.  ``phase`` orders dependent leaves: a leaf may start once
    every leaf of a lower phase has finished (all phase-0 leaves are
    independent of each other)."""
    step = (grid[0][1], grid[1][1], grid[2][1])
    Mv, Nv, Kv = (axis_values(ax) for ax in grid)

    def rec(a, b, c, m0, n0, k0, beta):
        act = int(action[a, b, c])
        q = int(qarg[a, b, c])
        if act == KEEP:
            ta, tb, tc = (int(x) for x in target[a, b, c])
            v = int(vstar[ta, tb, tc])
            return [(v, beta, 0, m0, n0, k0, Mv[a], Nv[b], Kv[c], Mv[ta], Nv[tb], Kv[tc])], 1
        if act == SPLIT_M:
            p = a + 1
            l1, d1 = rec(p - q - 1, b, c, m0, n0, k0, beta)
            l2, d2 = rec(q - 1, b, c, m0 + (p - q) * step[0], n0, k0, beta)
            return l1 + l2, max(d1, d2)
        if act == SPLIT_N:
            p = b + 1
            l1, d1 = rec(a, p - q - 1, c, m0, n0, k0, beta)
            l2, d2 = rec(a, q - 1, c, m0, n0 + (p - q) * step[1], k0, beta)
            return l1 + l2, max(d1, d2)
        p = c + 1                                     # SPLIT_K
        l1, d1 = rec(a, b, p - q - 1, m0, n0, k0, beta)
        l2, d2 = rec(a, b, q - 1, m0, n0, k0 + (p - q) * step[2], 1)
        l2 = [lf[:2] + (lf[2] + d1,) + lf[3:] for lf in l2]
        return l1 + l2, d1 + d2

    out, _ = rec(*cell, 0, 0, 0, 0)
    return out


def plan(T0v: np.ndarray, grid):
    """The whole offline phase: best-of, T1, T2 and every cell's leaf list."""
    T0s, vstar = best_of(T0v)
    T1, target = pad_T1(T0s, grid)
    T2, action, qarg = split_T2(T1, grid)
    nm, nn, nk = T0s.shape
    all_leaves = {}
    for cell in itertools.product(range(nm), range(nn), range(nk)):
        all_leaves[cell] = leaves(cell, grid, action, qarg, target, vstar)
    return {"T0s": T0s, "vstar": vstar, "T1": T1, "target": target, "T2": T2,
            "action": action, "q": qarg, "leaves": all_leaves}

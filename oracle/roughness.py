"""O-Roughness: the throughput surface and its roughness (Sec. 2,
definitions: achieved TFLOPs = 2MNK / (t 1e12); Roughness({T_1..T_n}) =
1/(n-1) sum_i |T_{i+1} - T_i|; Sec. 8.6 / Table 17 for the slice and 3D
conventions).

Test infrastructure only (see the package docstring).

Readings:
  * Times are integer nanoseconds; the surface value of a cell is
    (2.0 * M * N * K) / (t_ns * 1e3) in IEEE double, in exactly this
    operation order (the product 2MNK is exact for sizes up to 2**17).
  * Roughness along an axis pools every adjacent pair of every line parallel
    to that axis: sum |delta| / (number of pairs).  All lines along one axis
    have the same length, so this equals the mean of the per-line values.
  * Headline value: the N axis on the slice at the largest K (the paper's
    K = 4096 slice), pooled over M.
  * 3D aggregate: (R_M + R_N + R_K) / 3 over the whole grid.
  * Sums are correctly rounded (math.fsum), so any summation order gives the
    same double.
"""
from __future__ import annotations

import math

import numpy as np


def tflops(M: int, N: int, K: int, t_ns: int) -> float:
    return (2.0 * M * N * K) / (float(t_ns) * 1e3)


def surface(t_ns: np.ndarray, grid) -> np.ndarray:
    """TFLOP/s per cell from integer nanoseconds, shape (nm, nn, nk)."""
    t_ns = np.asarray(t_ns, dtype=np.int64)
    (ms, mstep, nm), (ns, nstep, nn), (ks, kstep, nk) = grid
    out = np.empty((nm, nn, nk), dtype=np.float64)
    for a in range(nm):
        M = ms + a * mstep
        for b in range(nn):
            N = ns + b * nstep
            for c in range(nk):
                K = ks + c * kstep
                out[a, b, c] = tflops(M, N, K, int(t_ns[a, b, c]))
    return out


def roughness_1d(values) -> float:
    """1/(n-1) * sum_{i=1}^{n-1} |T_{i+1} - T_i| for one line of values."""
    v = [float(x) for x in values]
    if len(v) < 2:
        return 0.0
    return math.fsum(abs(v[i + 1] - v[i]) for i in range(len(v) - 1)) / (len(v) - 1)


def roughness_axis(S: np.ndarray, axis: int) -> float:
    """Pooled mean |delta| over all adjacent pairs along ``axis`` of a 3D surface."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[axis]
    if n < 2:
        return 0.0
    terms = []
    for idx in np.ndindex(*[S.shape[d] for d in range(3) if d != axis]):
        line = []
        for i in range(n):
            full = list(idx)
            full.insert(axis, i)
            line.append(float(S[tuple(full)]))
        terms.extend(abs(line[i + 1] - line[i]) for i in range(n - 1))
    return math.fsum(terms) / len(terms)


def roughness_all(S: np.ndarray) -> dict:
    """R_M, R_N, R_K, R_3D and the N-axis roughness on the largest-K slice."""
    S = np.asarray(S, dtype=np.float64)
    rM = roughness_axis(S, 0)
    rN = roughness_axis(S, 1)
    rK = roughness_axis(S, 2)
    r3 = (rM + rN + rK) / 3.0
    sl = S[:, :, S.shape[2] - 1]
    rs = roughness_axis(sl[:, :, None], 1)
    return {"R_M": rM, "R_N": rN, "R_K": rK, "R_3D": r3, "R_N_slice": rs}


def mean(S: np.ndarray) -> float:
    """Arithmetic mean TFLOP/s over the cells (correctly rounded sum, one division)."""
    v = [float(x) for x in np.asarray(S, dtype=np.float64).ravel()]
    return math.fsum(v) / len(v) if v else 0.0

"""Four-surface decomposition of a measured landscape (Sec. 4, "Decomposition:
Where Does Texture Come From?"; Figs. 5-6; the bottleneck classification of
Table 3).

Test infrastructure only (see the package docstring).

Over one grid of cells (M, N, K):
  compute surface   t_compute = 2 M N K / P      (useful flops at peak; tile- and
                                                  kernel-independent, Sec. 4)
  memory surface    t_memory  = the measured memory twin (given)
  GEMM surface      t_GEMM    = the measured GEMM (given)
  overhead surface  t_overhead = t_GEMM - max(t_compute, t_memory)
A cell is compute-bound when even a zero-waste, perfectly pipelined kernel
would be limited by compute: t_compute > t_memory (Table 3).

Times are in ns, P in TFLOP/s, so t_compute = 2MNK / (P 1e3) ns.  Summary:
  [0] share of compute-bound cells,
  [1] mean over cells of t_overhead / t_GEMM (the overhead share of Fig. 6),
  [2] sum t_overhead / sum t_GEMM,
  [3] mean over cells of t_memory / t_GEMM.
Sums are correctly rounded (math.fsum).
"""
from __future__ import annotations

import math

import numpy as np


def compute_ns(M: int, N: int, K: int, p_tflops: float) -> float:
    """2MNK useful flops at p_tflops TFLOP/s, in ns."""
    flops = 2.0 * float(M) * float(N) * float(K)
    return flops / (p_tflops * 1e3)


def decompose(ms, ns, ks, t_gemm_ns, t_mem_ns, p_tflops: float):
    """Compute and overhead surfaces ([len(ms)][len(ns)][len(ks)] float64) and the
    four summary values, from integer ns surfaces of the same shape."""
    tg = np.asarray(t_gemm_ns).reshape(len(ms), len(ns), len(ks))
    tm = np.asarray(t_mem_ns).reshape(len(ms), len(ns), len(ks))
    if np.any(tg <= 0) or np.any(tm <= 0):
        raise ValueError("times must be positive")
    comp = np.zeros(tg.shape)
    over = np.zeros(tg.shape)
    bound = 0
    share_o, share_m, sum_o, sum_g = [], [], [], []
    for a, M in enumerate(ms):
        for b, N in enumerate(ns):
            for c, K in enumerate(ks):
                t_c = compute_ns(M, N, K, p_tflops)
                t_g = float(tg[a, b, c])
                t_m = float(tm[a, b, c])
                t_o = t_g - max(t_c, t_m)
                comp[a, b, c] = t_c
                over[a, b, c] = t_o
                bound += t_c > t_m
                share_o.append(t_o / t_g)
                share_m.append(t_m / t_g)
                sum_o.append(t_o)
                sum_g.append(t_g)
    cells = tg.size
    stats = np.array([bound / cells, math.fsum(share_o) / cells, math.fsum(sum_o) / math.fsum(sum_g),
                      math.fsum(share_m) / cells])
    return comp, over, stats

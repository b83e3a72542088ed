"""First-principles landscapes and the Kernel Optimality Level grading
(Sec. 3.3 partial-tile waste at tile boundaries; Sec. 9.1 "The ideal ceiling and its ramp";
Sec. 9.2 "The optimal: deriving ruggedness in closed form"; Sec. 10.2-10.3,
Table 19).

Test infrastructure only (see the package docstring).

ideal_surface (Sec. 9.1): P * min(1, W / C) with W = ceil(M/TM) ceil(N/TN) for
the default tile and C compute units; independent of K.

optimal_surface (Sec. 9.2): per cell, the best over the tile set of
max(t_compute, t_memory) with t_compute = 2MNK / (P eta_wave),
eta_wave = W / (ceil(W / C) C), and t_memory = 2MK/(BW eta_A) + 2KN/(BW eta_B)
+ 4MN/(BW eta_D).  The channel efficiencies eta follow the paper's GDDR6
interleave model when ``channels`` is given, else 1 (HBM: no disclosed hash).
Pins: its parts (eta_wave, the channel eta, the memory and compute terms), the
one-tile free-memory reduction to the ideal, and hand-worked cells on GB300
constants (a compute-bound multi-tile cell and a memory-bound one), which fix
the best-over-tiles of max(t_compute, t_memory) composition.  Against the
paper's own numbers it stays unpinned: its printed optimal statistics (Table
18) are not reproduced by its stated constants under any reading found.

kol (Sec. 10.2-10.3, Table 19): tau = mean A / mean O, rho = R(A) / R(O);
throughput bands T0 < 0.50 <= T1 < 0.75 <= T2 < 0.95 <= T3; smoothness bands
S3 for rho <= 1.25, S2 for 1.25 < rho <= 2, S1 for 2 < rho <= 3, S0 above 3;
level L = min(T, S).
"""
from __future__ import annotations

import math

import numpy as np


def tile_utilization(n: int, t: int) -> float:
    """Useful fraction of the last partial tile row: n / (t ceil(n / t)) (Sec. 3.3 alignment cliffs)."""
    return n / (t * math.ceil(n / t))


def wave_efficiency(w: int, c: int) -> float:
    """eta_wave = W / (ceil(W / C) C)."""
    return w / (math.ceil(w / c) * c)


def eta_channel(L: int, e: int, channels: int = 6, interleave: int = 256) -> float:
    """Per-tensor channel utilisation of the GDDR6 interleave model:
    a row covers w = min(channels, e) channels, consecutive rows start s =
    (L e / interleave) mod channels blocks apart, reaching channels / gcd(s,
    channels) distinct start channels; eta = min(channels, w * that) / channels."""
    w = min(channels, e)
    s = (L * e // interleave) % channels
    g = math.gcd(s, channels)
    return min(channels, w * channels / g) / channels


def peak_from_units(units: int, engines: int, macs_per_clk: int, ghz: float) -> float:
    """Datasheet peak in TFLOP/s: units x engines x MAC/clk x 2 flop/MAC x clock."""
    return units * engines * macs_per_clk * 2 * ghz / 1e3


def ideal_surface(grid, p_tflops: float, c_units: int, tile=(256, 256)) -> np.ndarray:
    (ms, mstep, nm), (ns, nstep, nn), (ks, kstep, nk) = grid
    out = np.empty((nm, nn, nk))
    for a in range(nm):
        M = ms + a * mstep
        for b in range(nn):
            N = ns + b * nstep
            W = math.ceil(M / tile[0]) * math.ceil(N / tile[1])
            out[a, b, :] = p_tflops * min(1.0, W / c_units)
    return out


def optimal_cell(M, N, K, p_tflops, c_units, tiles, bw_gbs, channels=None, interleave=256):
    fl = 2.0 * M * N * K
    if channels:
        eA, eB, eD = (eta_channel(K, 2, channels, interleave), eta_channel(N, 2, channels, interleave),
                      eta_channel(N, 4, channels, interleave))
    else:
        eA = eB = eD = 1.0
    bw = bw_gbs * 1e9
    t_mem = 2.0 * M * K / (bw * eA) + 2.0 * K * N / (bw * eB) + 4.0 * M * N / (bw * eD)
    best = math.inf
    for tm, tn in tiles:
        W = math.ceil(M / tm) * math.ceil(N / tn)
        t_comp = fl / (p_tflops * 1e12 * wave_efficiency(W, c_units))
        best = min(best, max(t_comp, t_mem))
    return fl / best / 1e12


def optimal_surface(grid, p_tflops, c_units, tiles, bw_gbs, channels=None, interleave=256):
    (ms, mstep, nm), (ns, nstep, nn), (ks, kstep, nk) = grid
    out = np.empty((nm, nn, nk))
    for a in range(nm):
        for b in range(nn):
            for c in range(nk):
                out[a, b, c] = optimal_cell(ms + a * mstep, ns + b * nstep, ks + c * kstep,
                                            p_tflops, c_units, tiles, bw_gbs, channels, interleave)
    return out


def throughput_band(tau: float) -> int:
    if tau < 0.50:
        return 0
    if tau < 0.75:
        return 1
    if tau < 0.95:
        return 2
    return 3


def smoothness_band(rho: float) -> int:
    if rho > 3.0:
        return 0
    if rho > 2.0:
        return 1
    if rho > 1.25:
        return 2
    return 3


def kol(mean_a: float, mean_o: float, r_a: float, r_o: float) -> dict:
    tau = mean_a / mean_o
    rho = r_a / r_o
    t = throughput_band(tau)
    s = smoothness_band(rho)
    return {"tau": tau, "rho": rho, "T": t, "S": s, "L": min(t, s)}

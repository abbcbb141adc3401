"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle callers.

This module holds no arithmetic of the method: only random numbers (numpy
PCG64 streams from explicit seeds) and workload shapes (sector tables with the
degeneracy distributions described for the benchmark bonds).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BOND = 20260604


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def complex_normal(gen: np.random.Generator, shape) -> np.ndarray:
    """i.i.d. N(0,1) real and imaginary parts, complex128."""
    return gen.standard_normal(shape) + 1j * gen.standard_normal(shape)


def gaussian_sector_table(D0: float, k: int, qmax: int = 12, tsmax: int = 12, parity: bool = True):
    """Multiplets (Q, 2S, d) with d = round(D0 exp(-Q^2/18 - S^2/4.5)), Q in [-qmax, qmax],
    2S in [0, tsmax], optionally only Q + 2S = k (mod 2); zero-degeneracy entries dropped."""
    out = []
    for Q in range(-qmax, qmax + 1):
        for ts in range(0, tsmax + 1):
            if parity and (Q + ts - k) % 2:
                continue
            S = ts / 2
            d = int(math.floor(D0 * math.exp(-Q * Q / 18.0 - S * S / 4.5) + 0.5))
            if d > 0:
                out.append((Q, ts, d))
    return out


def chi_of(table) -> int:
    """U(1)-equivalent bond dimension sum d (2S+1)."""
    return sum(d * (ts + 1) for (_, ts, d) in table)


def chi_su2_of(table) -> int:
    return sum(d for (_, _, d) in table)


def gaussian_table_for_chi(chi_target: int, k: int, parity: bool = True, **kw):
    """Smallest D0 (bisection) whose table reaches chi >= chi_target; returns (D0, table)."""
    lo, hi = 0.0, 1.0
    while chi_of(gaussian_sector_table(hi, k, parity=parity, **kw)) < chi_target:
        hi *= 2
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if chi_of(gaussian_sector_table(mid, k, parity=parity, **kw)) >= chi_target:
            hi = mid
        else:
            lo = mid
    return hi, gaussian_sector_table(hi, k, parity=parity, **kw)


def to_u1u1(table):
    """Expand SU(2) multiplets (Q, 2S, d) into U(1)xU(1) sectors (Q, 2S^z, d_total)."""
    acc = {}
    for (Q, ts, d) in table:
        for tz in range(-ts, ts + 1, 2):
            acc[(Q, tz)] = acc.get((Q, tz), 0) + d
    return [(Q, tz, d) for (Q, tz), d in sorted(acc.items())]


def random_blocks(seed: int, shapes):
    """One complex normal block per entry of shapes (in order) from one PCG64 stream."""
    g = rng(seed)
    return [complex_normal(g, s) for s in shapes]

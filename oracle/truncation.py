"""Truncation of a two-site SVD over symmetry sectors (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py``; never by the product package.

Restates the truncation of Sec. S2.4 (the kept set is fixed by the "truncated
weight", the summed squares of the discarded singular values, relative to the
whole) for a bond whose singular values come in symmetry sectors, with the
multiplet structure of Sec. S2.1 (Eq. symdecomp): under U(1)xSU(2) one reduced
singular value stands for a whole multiplet of 2S+1 states that share one
singular value s, and a symmetric truncation keeps or drops the multiplet as a
unit.  Under U(1)xU(1) every state is its own multiplet (2S+1 = 1).

Readings where the paper is silent (each one a line of the product's header):

* the reduced value r of a multiplet is normalised so that r^2 is the weight of
  the whole multiplet, r^2 = (2S+1) s^2;
* multiplets are ranked by the singular value s of their states (equivalently
  by the per-state weight s^2 = r^2 / (2S+1)), largest first; equal values go
  to the lower sector index, then to the lower index inside the sector;
* the discarded-weight rule drops the longest tail of the ranking whose weight
  is at most eps times the total weight; the bond-dimension cap keeps the
  longest head of the ranking that holds at most chi_max states; the kept head
  is the shorter of the two, and never empty;
* optionally (``degeneracy`` > 0) the cut may not fall between two ranked
  multiplets whose per-state weights are equal to within that relative
  tolerance: degenerate multiplets are kept or dropped together.  Both rules
  then move to the nearest allowed cut (the tail rule to a longer head, the cap
  to a shorter one); if no allowed head fits under the cap, the first allowed
  head is kept.

Everything is plain Python over small lists; no step is blocked or fused.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Selection:
    kept: list            # kept values per sector (a prefix of each sector)
    K: int                # multiplets kept
    states: int           # states kept, sum of (2S+1) over the kept multiplets
    total: float          # total weight
    discarded: float      # weight of the dropped multiplets
    cap_set_K: bool       # the chi cap (not the tail rule) fixed K


def ranked_multiplets(sectors):
    """sectors: list of (mult, values) with mult = 2S+1 and values the sector's reduced
    values r in descending order.  Returns [(per-state weight, sector, index, r, mult)]
    in rank order: per-state weight r*r/mult descending, then sector, then index."""
    items = []
    for k, (mult, values) in enumerate(sectors):
        for i, r in enumerate(values):
            r = float(r)
            lam = r * r / float(mult) if r == r and r >= 0.0 else -1.0
            items.append((lam, k, i, r, int(mult)))
    # Python's sort is stable; sort by (-lam, sector, index) explicitly
    items.sort(key=lambda t: (-t[0], t[1], t[2]))
    return items


def select_multiplets(sectors, eps: float, chi_max: int, degeneracy: float = 0.0) -> Selection:
    """The kept multiplets of one bond (rule in the module docstring)."""
    items = ranked_multiplets(sectors)
    n = len(items)
    if n == 0:
        raise ValueError("no singular values")
    weight = [(t[3] * t[3] if t[0] >= 0.0 else 0.0) for t in items]
    mult = [t[4] for t in items]
    total = sum(weight)

    def cut_allowed(K):
        # a head of K multiplets; K = n (keep everything) is always allowed
        if K == n:
            return True
        lam_prev, lam_next = items[K - 1][0], items[K][0]
        return not (degeneracy > 0.0 and lam_prev - lam_next <= degeneracy * lam_prev)

    allowed = [K for K in range(1, n + 1) if cut_allowed(K)]
    # tail[K] = weight of the ranked multiplets K, K+1, ..., summed from the smallest up
    tail = [0.0] * (n + 1)
    for K in range(n - 1, -1, -1):
        tail[K] = tail[K + 1] + weight[K]
    # head[K] = states in the first K ranked multiplets
    head = [0] * (n + 1)
    for K in range(1, n + 1):
        head[K] = head[K - 1] + mult[K - 1]
    # tail rule: the shortest allowed head whose dropped tail weighs <= eps * total
    K_eps = None
    for K in allowed:
        if tail[K] <= eps * total:
            K_eps = K
            break
    # cap: the longest allowed head with at most chi_max states, else the first allowed head
    K_chi = None
    for K in allowed:
        if head[K] <= chi_max:
            K_chi = K
    if K_chi is None:
        K_chi = allowed[0]
    K = min(K_eps, K_chi)
    kept = [0] * len(sectors)
    for t in items[:K]:
        kept[t[1]] += 1
    return Selection(kept=kept, K=K, states=head[K], total=total, discarded=tail[K], cap_set_K=K_chi < K_eps)


def dense_keep_count(s: np.ndarray, chi_max: int, eps: float, degeneracy: float) -> int:
    """Number of leading values of one dense (unblocked) spectrum that the rule keeps,
    with every state its own multiplet and degenerate states cut together."""
    sel = select_multiplets([(1, list(s))], eps, chi_max, degeneracy)
    return sel.K

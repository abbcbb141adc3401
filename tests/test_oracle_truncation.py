"""Pins of the oracle's sector-aware truncation rule (Sec. S2.4 with the multiplets of
Sec. S2.1), ``oracle.truncation.select_multiplets``.

Every hand case uses values whose squares, per-state weights and sums are exact in
binary floating point (dyadic s; multiplicities 1, 4, 9 so that r = sqrt(2S+1) s is
s, 2s or 3s), so the expected answers below are worked out by hand and no decision
depends on rounding.  Each case names the plausible mistake it catches.
"""
import itertools

import numpy as np
import pytest

from oracle import mps
from oracle.truncation import dense_keep_count, select_multiplets


def sel(sectors, eps, chi, deg=0.0):
    return select_multiplets(sectors, eps, chi, deg)


def test_cap_at_a_multiplet_boundary():
    # singlet s=1/2 (weight 1/4), quartet s=1/4 (r=1/2, weight 4/16=1/4), singlet s=1/8
    secs = [(1, [0.5, 0.125]), (4, [0.5])]
    # ranking: singlet 1/2 (1 state), quartet (4 states), singlet 1/8 (1 state)
    assert sel(secs, 0.0, 5).kept == [1, 1]      # 1 + 4 = 5 states fit exactly
    assert sel(secs, 0.0, 4).kept == [1, 0]      # off by one: the quartet would need 5
    assert sel(secs, 0.0, 6).kept == [2, 1]
    # the prefix rule does not skip the quartet to take the later singlet
    s = sel(secs, 0.0, 3)
    assert s.kept == [1, 0] and s.states == 1 and s.cap_set_K


def test_cap_below_the_first_multiplet_keeps_it_whole():
    s = sel([(4, [0.5]), (1, [0.25])], 0.0, 2)
    assert s.kept == [1, 0] and s.states == 4


def test_ranking_uses_the_per_state_value_not_the_multiplet_weight():
    # singlet s=3/8 (weight 9/64) against a quartet of s=1/4 (r=1/2, weight 16/64):
    # per state the singlet is larger, as a multiplet the quartet is heavier
    s = sel([(4, [0.5]), (1, [0.375])], 0.0, 1)
    assert s.kept == [0, 1]
    s = sel([(4, [0.5]), (1, [0.375])], 0.0, 5)
    assert s.kept == [1, 1]


def test_multiplet_weight_counts_2S_plus_1():
    # singlet s=1/2 (1/4), quartet s=1/4 (4 x 1/16 = 1/4), singlet s=1/8 (1/64)
    secs = [(1, [0.5, 0.125]), (4, [0.5])]
    total = 0.25 + 0.25 + 1.0 / 64
    s = sel(secs, 0.5, 100)
    # eps * total = 0.2578..: the last singlet (1/64) goes, the quartet (+1/4) does not
    assert s.kept == [1, 1] and s.total == total and s.discarded == 1.0 / 64
    # a rule that weighted the quartet as 1/16 (one state) would drop it as well
    assert s.K == 2 and not s.cap_set_K


def test_exact_ties_break_by_sector_then_index():
    # per-state weight 1/4 for all three: singlet r=1/2, quartet r=1, nonet r=3/2
    q, one, non = (4, [1.0]), (1, [0.5]), (9, [1.5])
    assert sel([q, one, non], 0.0, 5).kept == [1, 1, 0]
    assert sel([one, q, non], 0.0, 5).kept == [1, 1, 0]
    assert sel([non, one, q], 0.0, 9).kept == [1, 0, 0]
    assert sel([non, one, q], 0.0, 10).kept == [1, 1, 0]
    # inside one sector equal values go by index
    assert sel([(1, [0.5, 0.5, 0.5])], 0.0, 2).kept == [2]


def test_eps_and_cap_bind_on_the_same_value():
    # weights 1/4, 1/4, 1/16, 1/16, 1/64 (singlets); total 41/64
    secs = [(1, [0.5, 0.25, 0.125]), (1, [0.5, 0.25])]
    tot = 41.0 / 64
    # tail rule: dropping {1/16, 1/64} = 5/64 <= eps*tot needs eps >= 5/41; keep 3
    s = sel(secs, 5.0 / 41 * (1 + 1e-12), 3)
    assert s.K == 3 and not s.cap_set_K
    assert s.kept == [2, 1]
    # cap 3 alone gives the same K; eps alone too
    assert sel(secs, 0.0, 3).K == 3 and sel(secs, 0.0, 3).cap_set_K
    assert sel(secs, 5.0 / 41 * (1 + 1e-12), 100).K == 3
    assert tot == sel(secs, 0.0, 100).total


def test_all_weight_in_one_sector():
    secs = [(1, [0.0, 0.0]), (3, [0.75, 0.5]), (1, [0.0])]
    s = sel(secs, 0.0, 100)
    # eps = 0 still drops exact zeros (tail weight 0 <= 0)
    assert s.kept == [0, 2, 0] and s.discarded == 0.0
    s = sel(secs, 0.5, 100)
    assert s.kept == [0, 1, 0]
    # nothing but zeros: one multiplet is kept
    assert sel([(1, [0.0, 0.0])], 0.0, 10).K == 1


def test_nan_and_negative_values_rank_last_with_no_weight():
    s = sel([(1, [float("nan"), 0.5]), (1, [-1.0])], 0.0, 10)
    assert s.kept == [1, 0] and s.total == 0.25


def test_degenerate_multiplets_are_cut_together():
    # values s = 1/2, 1/4, 1/4(1 + 2^-40), 1/8: the middle two are degenerate at 1e-9
    v = [0.5, 0.25 * (1 + 2.0 ** -40), 0.25, 0.125]
    secs = [(1, [v[0], v[2]]), (1, [v[1], v[3]])]
    assert sel(secs, 0.0, 2).K == 2                     # plain: the cap splits the pair
    assert sel(secs, 0.0, 2, 1e-9).K == 1               # degeneracy-aware: the pair goes together
    assert sel(secs, 0.0, 3, 1e-9).K == 3
    # tail rule moves to a longer head: dropping one of the pair would fit, not both
    tot = 0.25 + 2 * 0.0625 + 1.0 / 64 + 2.0 ** -40 * 0.125
    eps = (1.0 / 64 + 0.0625) / tot
    assert sel(secs, eps, 100).K == 2
    assert sel(secs, eps, 100, 1e-9).K == 3
    # the first allowed head is kept when nothing fits under the cap
    s = sel([(1, [0.5, 0.5 * (1 - 2.0 ** -45)])], 0.0, 1, 1e-9)
    assert s.K == 2 and s.states == 2


def test_multiplets_equal_their_expanded_states():
    """The SU(2) rule on reduced values keeps exactly the states that the same rule keeps
    on the full-basis spectrum (each multiplet expanded into its 2S+1 states, states of one
    multiplet cut together), for every cap and threshold."""
    rng = np.random.default_rng(5)
    for trial in range(40):
        secs, full = [], []
        for k in range(rng.integers(1, 5)):
            m = int(rng.choice([1, 4, 9]))
            sv = np.sort(rng.integers(1, 64, size=rng.integers(1, 4)))[::-1] / 64.0
            secs.append((m, list(sv * np.sqrt(m))))    # r = s sqrt(m) is exact for m in 1, 4, 9
            full += [(x, k) for x in sv for _ in range(m)]
        s_full = np.array(sorted([x for x, _ in full], reverse=True))
        for chi in (1, 3, 5, 8, 13, 100):
            for eps in (0.0, 1e-3, 1e-2, 0.1, 0.3):
                got = sel(secs, eps, chi, 1e-12)
                want = dense_keep_count(s_full, chi, eps, 1e-12)
                assert got.states == want, (trial, chi, eps)


def test_dense_rule_reduces_to_the_plain_dense_count():
    rng = np.random.default_rng(7)
    for _ in range(50):
        s = np.sort(rng.random(rng.integers(1, 12)))[::-1]
        for chi in (1, 2, 5, 20):
            for eps in (0.0, 1e-3, 0.05, 0.5):
                assert dense_keep_count(s, chi, eps, 0.0) == mps.truncation_count(s, chi, eps)


def test_monotone_in_eps_and_chi_and_scale_free():
    rng = np.random.default_rng(9)
    for _ in range(30):
        secs = [(int(m), list(np.sort(rng.random(rng.integers(1, 6)))[::-1]))
                for m in rng.choice([1, 2, 3, 4, 5], size=rng.integers(1, 5))]
        prev = None
        for chi in range(1, 30):
            st = sel(secs, 1e-3, chi).states
            assert prev is None or st >= prev
            prev = st
        prev = None
        for eps in (0.0, 1e-4, 1e-3, 1e-2, 0.1, 0.5):
            K = sel(secs, eps, 10 ** 6).K
            assert prev is None or K <= prev
            prev = K
        scaled = [(m, [4.0 * x for x in v]) for m, v in secs]
        for chi in (1, 4, 9):
            assert sel(secs, 1e-2, chi).kept == sel(scaled, 1e-2, chi).kept


@pytest.mark.parametrize("perm", list(itertools.permutations(range(3))))
def test_result_follows_the_sectors_not_their_order_without_ties(perm):
    secs = [(1, [0.9, 0.3]), (3, [0.7, 0.2]), (5, [0.55])]
    base = sel(secs, 1e-2, 9)
    p = [secs[i] for i in perm]
    got = sel(p, 1e-2, 9)
    assert [got.kept[perm.index(i)] for i in range(3)] == base.kept

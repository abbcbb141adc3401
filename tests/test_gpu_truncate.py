"""GPU parity of the truncation's multiplet selection (Sec. S2.4 with the multiplets of
Sec. S2.1): the engine's selection kernel, called through tdvp_truncate, against the
oracle's restatement ``oracle.truncation.select_multiplets``.

Selection is integer work (how many values of each sector are kept), so the bar is
exact equality of the kept counts, of K, of the states kept and of the flag that
says which rule set K.  Both sides rank on the same per-state weight r*r/(2S+1) in
FP64.  Hand cases use dyadic values (every sum exact); seeded random spectra skip
cases whose decision lies within 1e-12 (relative) of a rule's boundary, where the
two sides' different summation orders could legitimately differ.
"""
import numpy as np
import pytest

from oracle.truncation import select_multiplets

pytestmark = pytest.mark.gpu


def gpu(sectors, eps, chi, deg=0.0):
    from paper_2606_04771_b300._lib import truncate

    kept, st = truncate([v for _, v in sectors], [m for m, _ in sectors], eps, chi, deg)
    return list(int(k) for k in kept), st


def same(sectors, eps, chi, deg=0.0):
    want = select_multiplets(sectors, eps, chi, deg)
    got, st = gpu(sectors, eps, chi, deg)
    assert got == want.kept, (got, want.kept)
    assert int(st[3]) == want.K and int(st[4]) == want.states
    assert bool(st[5]) == want.cap_set_K
    assert abs(st[0] - want.total) <= 1e-14 * max(want.total, 1e-300)
    assert abs(st[1] - want.discarded) <= 1e-13 * max(want.total, 1e-300)
    return want


HAND = [
    # (sectors, eps, chi, degeneracy): the oracle pins' hand cases, each exact in binary
    ([(1, [0.5, 0.125]), (4, [0.5])], 0.0, 5, 0.0),
    ([(1, [0.5, 0.125]), (4, [0.5])], 0.0, 4, 0.0),
    ([(1, [0.5, 0.125]), (4, [0.5])], 0.0, 3, 0.0),
    ([(1, [0.5, 0.125]), (4, [0.5])], 0.5, 100, 0.0),
    ([(4, [0.5]), (1, [0.25])], 0.0, 2, 0.0),
    ([(4, [0.5]), (1, [0.375])], 0.0, 1, 0.0),
    ([(4, [0.5]), (1, [0.375])], 0.0, 5, 0.0),
    ([(4, [1.0]), (1, [0.5]), (9, [1.5])], 0.0, 5, 0.0),
    ([(1, [0.5]), (4, [1.0]), (9, [1.5])], 0.0, 5, 0.0),
    ([(9, [1.5]), (1, [0.5]), (4, [1.0])], 0.0, 9, 0.0),
    ([(9, [1.5]), (1, [0.5]), (4, [1.0])], 0.0, 10, 0.0),
    ([(1, [0.5, 0.5, 0.5])], 0.0, 2, 0.0),
    ([(1, [0.5, 0.25, 0.125]), (1, [0.5, 0.25])], 0.0, 3, 0.0),
    ([(1, [0.0, 0.0]), (3, [0.75, 0.5]), (1, [0.0])], 0.0, 100, 0.0),
    ([(1, [0.0, 0.0]), (3, [0.75, 0.5]), (1, [0.0])], 0.5, 100, 0.0),
    ([(1, [0.0, 0.0])], 0.0, 10, 0.0),
    ([(1, [0.5, 0.25]), (1, [0.25 * (1 + 2.0 ** -40), 0.125])], 0.0, 2, 0.0),
    ([(1, [0.5, 0.25]), (1, [0.25 * (1 + 2.0 ** -40), 0.125])], 0.0, 2, 1e-9),
    ([(1, [0.5, 0.25]), (1, [0.25 * (1 + 2.0 ** -40), 0.125])], 0.0, 3, 1e-9),
    ([(1, [0.5, 0.5 * (1 - 2.0 ** -45)])], 0.0, 1, 1e-9),
]


@pytest.mark.parametrize("case", range(len(HAND)))
def test_hand_cases_match_the_oracle(case):
    secs, eps, chi, deg = HAND[case]
    same(secs, eps, chi, deg)


def test_ties_both_rules_binding_together():
    secs = [(1, [0.5, 0.25, 0.125]), (1, [0.5, 0.25])]
    w = same(secs, 5.0 / 41 * (1 + 1e-12), 3)
    assert w.K == 3 and not w.cap_set_K


def _margin_ok(sectors, eps, chi, deg):
    """The decision is not within 1e-12 (relative) of a boundary of the tail rule."""
    from oracle.truncation import ranked_multiplets

    items = ranked_multiplets(sectors)
    w = [t[3] * t[3] for t in items]
    tot = sum(w)
    for K in range(1, len(w) + 1):
        tail = sum(w[K:])
        if abs(tail - eps * tot) <= 1e-12 * tot:
            return False
    return True


def _config2_sectors(rng, nsec, scale_chi):
    """Sector spectra shaped like the chi = 4096 bond of the benchmark: multiplets
    (Q, 2S), mult = 2S + 1 with 2S in 0..12, sector sizes ~ exp(-Q^2/18 - S^2/4.5),
    singular values decaying like a late-time TDVP spectrum (log-uniform over 12
    decades)."""
    secs = []
    for _ in range(nsec):
        q = int(rng.integers(-12, 13))
        two_s = int(rng.integers(0, 13))
        d = max(1, int(round(scale_chi * np.exp(-q * q / 18.0 - (two_s / 2) ** 2 / 4.5))))
        sv = np.sort(10.0 ** rng.uniform(-6, 0, size=d))[::-1] * np.sqrt(two_s + 1)
        secs.append((two_s + 1, list(sv)))
    return secs


@pytest.mark.parametrize("seed", range(12))
def test_random_sector_spectra_with_both_rules_binding(seed):
    rng = np.random.default_rng(1000 + seed)
    secs = _config2_sectors(rng, int(rng.integers(20, 90)), float(rng.uniform(5, 40)))
    tot_states = sum(m * len(v) for m, v in secs)
    bound_cap = bound_eps = 0
    for eps in (1e-12, 1e-9, 1e-6, 1e-4):
        for frac in (0.05, 0.3, 0.7):
            chi = max(1, int(frac * tot_states))
            for deg in (0.0, 1e-8):
                if not _margin_ok(secs, eps, chi, deg):
                    continue
                w = same(secs, eps, chi, deg)
                bound_cap += w.cap_set_K
                bound_eps += not w.cap_set_K and w.K < sum(len(v) for _, v in secs)
    assert bound_cap > 0 and bound_eps > 0   # both rules did bind somewhere


def test_many_values_span_several_ranking_tiles():
    # more values than one shared-memory tile of the ranking (2048) and than one pass of
    # the CTA (1024 threads x 8): 9000 values over 40 sectors, with exact duplicates
    rng = np.random.default_rng(77)
    secs = []
    for k in range(40):
        m = int(rng.choice([1, 2, 3, 4, 5]))
        base = np.sort(rng.integers(1, 4000, size=225))[::-1] / 4096.0
        secs.append((m, list(base * np.sqrt(m))))
    for eps, chi in ((1e-3, 4000), (1e-2, 100000), (0.0, 777)):
        if _margin_ok(secs, eps, chi, 0.0):
            same(secs, eps, chi, 0.0)


def test_rejects_bad_arguments():
    from paper_2606_04771_b300._lib import TdvpError, truncate

    with pytest.raises(TdvpError):
        truncate([[0.5]], [1], -1.0, 4)
    with pytest.raises(TdvpError):
        truncate([[0.5]], [0], 0.0, 4)
    with pytest.raises(TdvpError):
        truncate([[0.5]], [1], 0.0, 0)
    with pytest.raises(TdvpError):
        truncate([[]], [1], 0.0, 4)

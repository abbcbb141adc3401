"""Exact SU(2) Clebsch-Gordan coefficients (test infrastructure).

The U(1)xSU(2) reduced tensors of Eq. (symdecomp) (Sec. S2.1) hold one
element per multiplet; turning them back into m-resolved components needs the
Clebsch-Gordan coefficients <j1 m1; j2 m2 | J M> in the Condon-Shortley phase
convention.  They are evaluated here from Racah's closed form in exact rational
arithmetic (``fractions.Fraction``); only the final square root is floating
point.  All angular momenta are passed doubled (tj = 2j, tm = 2m) so that
half-integers stay integers.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache


def _f(n2: int) -> int:
    """(n2/2)! for an even doubled argument n2."""
    assert n2 % 2 == 0 and n2 >= 0
    return math.factorial(n2 // 2)


@lru_cache(maxsize=None)
def cg(tj1: int, tm1: int, tj2: int, tm2: int, tJ: int, tM: int) -> float:
    """<j1 m1; j2 m2 | J M> with every argument doubled."""
    if tm1 + tm2 != tM:
        return 0.0
    if not (abs(tj1 - tj2) <= tJ <= tj1 + tj2) or (tj1 + tj2 + tJ) % 2:
        return 0.0
    for tj, tm in ((tj1, tm1), (tj2, tm2), (tJ, tM)):
        if abs(tm) > tj or (tj + tm) % 2:
            return 0.0
    pref = Fraction((tJ + 1) * _f(tJ + tj1 - tj2) * _f(tJ - tj1 + tj2) * _f(tj1 + tj2 - tJ),
                    _f(tj1 + tj2 + tJ + 2))
    pref *= (_f(tJ + tM) * _f(tJ - tM) * _f(tj1 - tm1) * _f(tj1 + tm1)
             * _f(tj2 - tm2) * _f(tj2 + tm2))
    total = Fraction(0)
    k = 0
    while True:
        args = (tj1 + tj2 - tJ - 2 * k, tj1 - tm1 - 2 * k, tj2 + tm2 - 2 * k,
                tJ - tj2 + tm1 + 2 * k, tJ - tj1 - tm2 + 2 * k)
        if args[0] < 0 or args[1] < 0 or args[2] < 0:
            break
        if args[3] >= 0 and args[4] >= 0:
            den = math.factorial(k)
            for a in args:
                den *= _f(a)
            total += Fraction((-1) ** k, den)
        k += 1
    if total == 0:
        return 0.0
    sign = 1.0 if total > 0 else -1.0
    return sign * math.sqrt(pref * total * total)


def cg_array(tj1: int, tj2: int, tJ: int):
    """C[m1, m2, M] = <j1 m1; j2 m2 | J M>, m indices ordered from +j down to -j."""
    import numpy as np

    C = np.zeros((tj1 + 1, tj2 + 1, tJ + 1))
    for a in range(tj1 + 1):
        for b in range(tj2 + 1):
            for c in range(tJ + 1):
                C[a, b, c] = cg(tj1, tj1 - 2 * a, tj2, tj2 - 2 * b, tJ, tJ - 2 * c)
    return C

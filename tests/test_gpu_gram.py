"""The FP64 finish of the split-precision SVD split by Gram iteration.

After the FP32 Jacobi preconditioner the columns of G = W V32 are orthogonal to
the FP32 level.  The engine then forms C = conj(G^H G) with one GEMM per sector,
rotates every column pair at once by the complex Jacobi rotation of its 2x2
Gram block (first order in the off-diagonals, so one step squares them) and
applies the rotation with a second GEMM; it stops, like the FP64 Jacobi it
replaces, after a step whose rotations were all below 1e-6 relative or 1e-10 in
weight.  When near-degenerate columns of weight would need a large rotation, or
the iteration does not settle in four steps, the split finishes with the
sequential FP64 Jacobi from where the iteration left G.

Checked here:
* bond updates from the Neel state in BF16x4 against the oracle's dense TDVP
  (the same sequence as the FP64 bond test): entropies and centre observables
  within 3e-7, a few times the BF16x4 matvec's relative error;
* on a chi = 2048 synthetic bond and on a short quench, the Gram finish against
  the Jacobi finish (TDVP_SPLIT_FINISH=jacobi): the same kept dimensions, the first
  update's entropy within 1e-12, and later values within 3e-7 (the BF16x4 matvec
  turns tiny input differences into differences of up to that size);
* with TDVP_GRAM_TMAX=0 every pair of weight is declined, G stays unchanged and
  the fallback Jacobi gives the Jacobi finish's result bit for bit.
"""
import os

import numpy as np
import pytest

from oracle import mps

pytestmark = pytest.mark.gpu


def _with_env(env, fn):
    old = {k: os.environ.get(k) for k in env}
    for k, v in env.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = str(v)
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("sym", ["su2", "u1u1"])
def test_split_precision_bond_updates_match_oracle(sym):
    from paper_2606_04771_b300 import Chain

    L, J, U, dt = 6, 1.0, 4.0, 0.08
    ref = mps.DenseTDVP(L, J, U)
    ch = Chain(L, J, U, symmetry=sym, precision="bf16x4")
    seq = [(0, 0), (1, 0), (2, 0), (3, 0), (3, 1), (2, 1), (1, 1)]
    for bond, direction in seq:
        s = ch.bond_update(bond, direction, dt, 256, 1e-12)
        if direction == 0:
            ref.bond_lr(bond, dt / 2, 256, 1e-12, True)
        else:
            ref.bond_rl(bond, dt / 2, 256, 1e-12, True)
        p = ref.last_s ** 2
        s_ref = float(-np.sum(p[p > 1e-300] * np.log(p[p > 1e-300])))
        assert abs(s - s_ref) < 3e-7, (bond, direction, s, s_ref)
    site, o = ch.measure_center()
    r = mps.observables_full(mps.full_state(ref.mps), L)
    for key in ("n", "sz", "docc"):
        assert abs(o[key] - r[key][site]) < 3e-7, key
    assert ch.stats()["gram_steps"] > 0
    ch.close()


def _bond(env):
    from paper_2606_04771_b300 import Chain

    def run():
        ch = Chain(16, 1.0, 4.0, symmetry="su2", random_chi=2048, seed=7, center=7, precision="bf16x4")
        s1 = ch.bond_update(7, 0, 0.05, 2048, 1e-9)
        s2 = ch.bond_update(7, 1, 0.05, 2048, 1e-9)
        o = ch.measure_center()[1]
        chis, _ = ch.bond_dims()
        st = ch.stats()
        ch.close()
        return (s1, s2, o, chis), st

    return _with_env(env, run)


def test_gram_finish_equals_jacobi_finish_on_large_bond():
    a, sa = _bond({"TDVP_SPLIT_FINISH": None, "TDVP_GRAM_TMAX": None})
    b, sb = _bond({"TDVP_SPLIT_FINISH": "jacobi"})
    assert sa["gram_steps"] >= 4 and sa["gram_fallbacks"] == 0 and sa["jacobi64_flops"] == 0
    assert sb["gram_steps"] == 0 and sb["jacobi64_flops"] > 0
    assert np.array_equal(a[3], b[3])  # the same kept bond dimensions
    # the first update starts from the same state: both finishes give the singular
    # values to the FP64 level.  The second starts from states that differ at the
    # level of the BF16x4 updates of the Gram steps (~1e-12), which the BF16x4 matvec
    # turns into differences of up to ~1e-7 (a digit that rounds the other way moves
    # an entry by 2^-30 of its row's scale): the bar is that of the BF16x4 mode's
    # own accuracy, not of the SVD.
    assert abs(a[0] - b[0]) < 1e-12
    assert abs(a[1] - b[1]) < 3e-7
    for key in ("n", "sz", "docc"):
        assert abs(a[2][key] - b[2][key]) < 3e-7, key


def test_gram_finish_quench_matches_jacobi_finish():
    from paper_2606_04771_b300 import Chain

    def run():
        ch = Chain(10, 1.0, 4.0, symmetry="su2", precision="bf16x4")
        for _ in range(8):
            ch.step(0.05, 48, 1e-10)
        o, st = ch.measure(), ch.stats()
        ch.close()
        return o, st

    a, sa = _with_env({"TDVP_SPLIT_FINISH": None, "TDVP_GRAM_TMAX": None}, run)
    b, sb = _with_env({"TDVP_SPLIT_FINISH": "jacobi"}, run)
    assert sa["gram_steps"] > 0
    for key in ("n_up", "n_dn", "docc", "s_ent"):
        assert np.abs(a[key] - b[key]).max() < 3e-7, key
    assert abs(a["energy"] - b["energy"]) < 3e-7  # E ~ 1e-7 here: the BF16x4 drift of a conserved zero


def test_declined_gram_steps_fall_back_to_the_jacobi_bit_for_bit():
    a, sa = _bond({"TDVP_SPLIT_FINISH": None, "TDVP_GRAM_TMAX": 0})
    b, sb = _bond({"TDVP_SPLIT_FINISH": "jacobi"})
    assert sa["gram_fallbacks"] == 2 and sa["jacobi64_flops"] > 0
    assert a[0] == b[0] and a[1] == b[1]
    assert a[2] == b[2]
    assert np.array_equal(a[3], b[3])
    assert sa["sweeps64"] == sb["sweeps64"]

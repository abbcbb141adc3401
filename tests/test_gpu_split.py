"""Parity of the tensor-core (split-precision) block GEMMs.

BF16X4 (scaled 8-bit digits, exact per-order FP32 accumulation) must reproduce
the oracle's FP64 H_eff.psi to 2e-7 relative to the output norm on every case and
the full TDVP observables within the 1e-6 bar; 3XTF32 (FP32 accumulation) is the
faster, looser mode and must stay within 3e-5 on the matvec.  Both use the same
task lists as the FP64 path; differences come only from the split arithmetic.
"""
import numpy as np
import pytest

from gpu_helpers import fill_bond_problem, oracle_heff
from oracle import mps

pytestmark = pytest.mark.gpu

CASES = {
    "su2_small": (True, [(3, 1, 2), (4, 0, 1), (4, 2, 2), (5, 1, 1), (2, 0, 1)],
                  [(5, 1, 2), (6, 0, 2), (6, 2, 1), (4, 0, 1), (5, 3, 1)]),
    "su2_tiles": (True, [(3, 1, 70), (4, 0, 65), (4, 2, 3), (2, 2, 1)],
                  [(5, 1, 66), (6, 0, 1), (4, 0, 67), (5, 3, 2)]),
    "u1_tiles": (False, [(3, 1, 70), (4, 0, 130), (3, -1, 5)], [(5, 1, 66), (6, 0, 1), (5, -1, 129)]),
    "one_block": (True, [(4, 0, 1)], [(6, 0, 1)]),
    # 119 theta blocks of d = 12..75 (328 output tiles of 64 x 64 in the last stage,
    # more in the first): more tiles than SMs, so each persistent CTA takes several
    # tiles (both TMEM accumulator sets, the operand ring wrapping, the epilogue of
    # one tile beside the MMAs of the next)
    "su2_many_tiles": (True, [(1, 1, 66), (2, 0, 70), (2, 2, 20), (3, 1, 72), (3, 3, 12), (4, 0, 75), (4, 2, 30),
                              (5, 1, 68), (6, 0, 66), (6, 2, 16), (7, 1, 65)],
                       [(3, 1, 66), (4, 0, 70), (4, 2, 20), (5, 1, 72), (5, 3, 12), (6, 0, 75), (6, 2, 30),
                        (7, 1, 68), (8, 0, 66), (8, 2, 16), (9, 1, 65)]),
}
TOL = {"bf16x4": 2e-7, "3xtf32": 3e-5}


@pytest.mark.parametrize("prec", ["bf16x4", "bf16x4-blocks", "3xtf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_split_heff_matches_oracle(name, prec, monkeypatch):
    """bf16x4: the packed plan (long GEMMs per input / output sector); bf16x4-blocks:
    the per-block task lists (TDVP_HEFF_PACKED=0); both to the BF16x4 bar."""
    from paper_2606_04771_b300 import BondProblem

    if prec == "bf16x4-blocks":
        monkeypatch.setenv("TDVP_HEFF_PACKED", "0")
        prec = "bf16x4"
    su2, left, right = CASES[name]
    bp = BondProblem(left, right, symmetry="su2" if su2 else "u1u1", precision=prec)
    lb, rb, keys, theta, th, Ld, Rd, (dims, _) = fill_bond_problem(bp, left, right, su2, seed=4321)
    if name == "su2_many_tiles":
        tiles = sum(-(-int(r) // 64) * -(-int(c) // 64) for r, c in dims)
        assert tiles > 2 * 148, tiles
    got = bp.heff_apply(theta)
    ref = oracle_heff(lb, rb, keys, th, Ld, Rd, 1.0, 4.0)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < TOL[prec], err
    bp.close()


def test_split_env_conjugate_operands():
    """The environment updates use conjugate-transposed operands (op = C); a chain
    evolved with BF16X4 must match the FP64 oracle through several sweeps."""
    from paper_2606_04771_b300 import Chain

    L, J, U, dt = 8, 1.0, 4.0, 0.05
    ref = mps.DenseTDVP(L, J, U)
    ch = Chain(L, J, U, symmetry="su2", precision="bf16x4")
    for k in range(12):
        ref.step(dt, 256, 1e-12)
        ch.step(dt, 256, 1e-12)
    o, r = ch.measure(), ref.observables()
    for key in ("n_up", "n_dn", "docc", "s_ent"):
        assert np.abs(o[key] - r[key]).max() < 1e-6, key
    assert abs(o["energy"] - r["energy"]) < 1e-6
    ch.close()

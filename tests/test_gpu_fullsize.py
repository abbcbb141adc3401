"""Full-size parity of H_eff.psi at the benchmark bond (chi = 4096 U(1)-equivalent).

The U(1)xSU(2) benchmark table expanded to U(1)xU(1) sectors (145 sectors,
d_max = 198, 5.3 M complex elements) runs through the engine in the bench's
launch configuration, in each precision: FP64, and the tensor-core split modes
BF16x4 and 3xTF32, whose persistent kernels here take thousands of output tiles
(many per CTA).  The oracle recomputes a seeded sample of output blocks one by
one by brute force (oracle.blockwise) and every sampled block must agree element
by element: FP64 to 1e-12 of the block's scale; the split modes to their matvec
bars, 2e-7 (BF16x4) and 3e-5 (3xTF32) of the output's scale (their error is set
by the row and column scales of whole operand groups, not by one block).
"""
import numpy as np
import pytest

import synth
from oracle import blockwise, heff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fullsize_case():
    """The bond tables, seeded blocks and the oracle's sampled output blocks (computed once)."""
    D0, tab = synth.gaussian_table_for_chi(4096, 30)
    u1 = synth.to_u1u1(tab)
    left = [(Q + 30, tz, d) for (Q, tz, d) in u1]
    right = [(Q + 32, tz, d) for (Q, tz, d) in u1]
    lb, rb = heff.Bond(left, False), heff.Bond(right, False)
    th_keys = heff.theta_blocks(lb, rb)
    lk, rk = heff.left_env_blocks(lb, lb), heff.right_env_blocks(rb, rb)
    dims = [(lb.sectors[k[0]][2], rb.sectors[k[4]][2]) for k in th_keys]
    ld = [(lb.sectors[k[0]][2], lb.sectors[k[2]][2]) for k in lk]
    rd = [(rb.sectors[k[0]][2], rb.sectors[k[2]][2]) for k in rk]
    th = synth.random_blocks(31, dims)
    Lb = synth.random_blocks(32, ld)
    Rb = synth.random_blocks(33, rd)
    sample = synth.rng(34).choice(len(th_keys), size=24, replace=False)
    ref, _ = blockwise.heff2_u1_blocks(lb, rb, th_keys, th, lk, Lb, rk, Rb, heff.shiba_mpo_tensor(1.0, 4.0),
                                       [th_keys[i] for i in sample])
    return left, right, th_keys, dims, ld, rd, th, Lb, Rb, sample, ref


@pytest.mark.parametrize("prec", ["fp64", "bf16x4", "3xtf32"])
def test_fullsize_u1_heff_sampled_blocks_each_precision(prec, fullsize_case):
    from paper_2606_04771_b300 import BondProblem

    left, right, th_keys, dims0, ld0, rd0, th, Lb, Rb, sample, ref = fullsize_case
    bp = BondProblem(left, right, symmetry="u1u1", precision=prec)
    keys, dims, offs, n = bp.blocks(0)
    assert [tuple(int(x) for x in d) for d in dims] == dims0
    _, ld, _, _ = bp.blocks(1)
    _, rd, _, _ = bp.blocks(2)
    assert [tuple(int(x) for x in d) for d in ld] == ld0 and [tuple(int(x) for x in d) for d in rd] == rd0
    flat = lambda bl: np.concatenate([b.reshape(-1) for b in bl])
    bp.set_env(1, flat(Lb))
    bp.set_env(2, flat(Rb))
    got = bp.heff_apply(flat(th))
    out_scale = max(np.abs(ref[th_keys[i]]).max() for i in sample)
    tol = {"bf16x4": 2e-7, "3xtf32": 3e-5}.get(prec)
    for i in sample:
        r, c = dims[i]
        blk = got[offs[i]:offs[i] + r * c].reshape(r, c)
        want = ref[th_keys[i]]
        if prec == "fp64":
            scale = max(np.abs(want).max(), 1e-300)
            assert np.abs(blk - want).max() < 1e-12 * scale, (th_keys[i], np.abs(blk - want).max() / scale)
        else:
            assert np.abs(blk - want).max() < tol * out_scale, (prec, th_keys[i],
                                                                 np.abs(blk - want).max() / out_scale)
    bp.close()

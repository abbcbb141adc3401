"""Full-size parity of H_eff.psi at the benchmark bond (chi = 4096 U(1)-equivalent).

The U(1)xSU(2) benchmark table expanded to U(1)xU(1) sectors (145 sectors,
d_max = 198, 5.3 M complex elements) runs through the engine's FP64 path in the
bench's launch configuration; the oracle recomputes a seeded sample of output
blocks one by one by brute force (oracle.blockwise) and every sampled block
must agree element by element (1e-12 relative to the block norm).
"""
import numpy as np
import pytest

import synth
from oracle import blockwise, heff

pytestmark = pytest.mark.gpu


def test_fullsize_u1_heff_sampled_blocks():
    from paper_2606_04771_b300 import BondProblem

    D0, tab = synth.gaussian_table_for_chi(4096, 30)
    u1 = synth.to_u1u1(tab)
    left = [(Q + 30, tz, d) for (Q, tz, d) in u1]
    right = [(Q + 32, tz, d) for (Q, tz, d) in u1]
    bp = BondProblem(left, right, symmetry="u1u1", precision="fp64")
    lb, rb = heff.Bond(left, False), heff.Bond(right, False)
    keys, dims, offs, n = bp.blocks(0)
    th_keys = heff.theta_blocks(lb, rb)
    assert len(th_keys) == len(keys)
    lk, rk = heff.left_env_blocks(lb, lb), heff.right_env_blocks(rb, rb)
    _, ld, _, _ = bp.blocks(1)
    _, rd, _, _ = bp.blocks(2)
    th = synth.random_blocks(31, [tuple(d) for d in dims])
    Lb = synth.random_blocks(32, [tuple(d) for d in ld])
    Rb = synth.random_blocks(33, [tuple(d) for d in rd])
    flat = lambda bl: np.concatenate([b.reshape(-1) for b in bl])
    bp.set_env(1, flat(Lb))
    bp.set_env(2, flat(Rb))
    got = bp.heff_apply(flat(th))
    sample = synth.rng(34).choice(len(th_keys), size=24, replace=False)
    ref, _ = blockwise.heff2_u1_blocks(lb, rb, th_keys, th, lk, Lb, rk, Rb, heff.shiba_mpo_tensor(1.0, 4.0),
                                       [th_keys[i] for i in sample])
    for i in sample:
        r, c = dims[i]
        blk = got[offs[i]:offs[i] + r * c].reshape(r, c)
        want = ref[th_keys[i]]
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(blk - want).max() < 1e-12 * scale, (th_keys[i], np.abs(blk - want).max() / scale)
    bp.close()

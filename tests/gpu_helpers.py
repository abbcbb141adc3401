"""Shared helpers of the GPU parity tests: build the same seeded bond problem for the
engine (through the C ABI) and for the oracle (dense m-resolved expansion)."""
import numpy as np

import synth
from oracle import heff


def fill_bond_problem(bp, left, right, su2, seed):
    """Random L, R, theta in the engine's block order; returns the oracle-side dicts."""
    lb = heff.Bond(left, su2)
    rb = heff.Bond(right, su2)
    keys, dims, offs, n = bp.blocks(0)
    ref_keys = heff.theta_blocks(lb, rb)
    got = [(int(k[0]), int(k[1]), (int(lb.sectors[k[0]][0] + heff._site(su2)[k[1]][0][0]), int(k[2])),
            int(k[3]), int(k[4])) for k in keys]
    assert got == ref_keys, "theta block enumeration differs from the oracle's"
    lkeys, ldims, loffs, ln = bp.blocks(1)
    rkeys, rdims, roffs, rn = bp.blocks(2)
    assert [tuple(int(x) for x in k[:3]) for k in lkeys] == heff.left_env_blocks(lb, lb)
    assert [tuple(int(x) for x in k[:3]) for k in rkeys] == heff.right_env_blocks(rb, rb)
    th_blocks = synth.random_blocks(seed, [tuple(d) for d in dims])
    L_blocks = synth.random_blocks(seed + 1, [tuple(d) for d in ldims])
    R_blocks = synth.random_blocks(seed + 2, [tuple(d) for d in rdims])
    flat = lambda bl: np.concatenate([b.reshape(-1) for b in bl]).astype(np.complex128)
    theta = flat(th_blocks)
    bp.set_env(1, flat(L_blocks))
    bp.set_env(2, flat(R_blocks))
    th = {k: b for k, b in zip(ref_keys, th_blocks)}
    Ld = {heff.left_env_blocks(lb, lb)[i]: b for i, b in enumerate(L_blocks)}
    Rd = {heff.right_env_blocks(rb, rb)[i]: b for i, b in enumerate(R_blocks)}
    return lb, rb, ref_keys, theta, th, Ld, Rd, (dims, offs)


def oracle_heff(lb, rb, keys, th, Ld, Rd, J, U):
    W = heff.shiba_mpo_tensor(J, U)
    Lenv = heff.expand_left_env(Ld, lb, lb)
    Renv = heff.expand_right_env(Rd, rb, rb)
    out = heff.heff2_dense(Lenv, W, W, Renv, heff.expand_theta(th, lb, None, rb))
    red = heff.reduce_theta(out, lb, rb, keys)
    return np.concatenate([red[k].reshape(-1) for k in keys])

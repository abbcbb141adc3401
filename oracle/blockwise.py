"""O4 at benchmark scale: U(1)xU(1) block-sparse effective Hamiltonian (test infrastructure).

The dense einsum of ``heff`` cannot hold a chi ~ 4096 two-site tensor, so at the
benchmark sizes the oracle evaluates the same definition (Sec. S2.3),

  theta'[a',s1',s2',b'] = sum L[a',w,a] W[w,w1,s1',s1] W[w1,w2,s2',s2] R[b,w2,b'] theta[a,s1,s2,b],

one output block at a time, with every bond index split into U(1)xU(1)
sectors (n, 2S^z): for an output block (a', s1', s2', b') it loops over the left
environment blocks (a', w, a), the right environment blocks (b, w2, b') and the
site states (s1, s2), and accumulates coef * L @ theta @ R where coef is the
MPO product summed over the inner channel w1.  Plain matmuls, no reordering
beyond the definition.  Channels are the six components of the
particle-hole-frame MPO of ``heff.shiba_mpo_tensor``.
"""
from __future__ import annotations

import numpy as np

from . import heff


def index_blocks(keys):
    return {k: i for i, k in enumerate(keys)}


def heff2_u1_blocks(left, right, th_keys, th_blocks, l_keys, l_blocks, r_keys, r_blocks, W, out_keys):
    """left/right: heff.Bond (U(1)xU(1)); *_keys as enumerated by heff.theta_blocks /
    left_env_blocks / right_env_blocks, *_blocks the matching arrays.  Returns
    ({out_key: block}, flops) with flops = 8 per complex multiply-add performed."""
    site = heff.SITE_MULTIPLETS_U1
    th = {k: b for k, b in zip(th_keys, th_blocks)}
    lby = {}
    for k, b in zip(l_keys, l_blocks):
        lby.setdefault(k[0], []).append((k[1], k[2], b))
    rby = {}
    for k, b in zip(r_keys, r_blocks):
        rby.setdefault(k[2], []).append((k[0], k[1], b))
    out, flops = {}, 0
    for key in out_keys:
        ap, s1p, cp, s2p, bp = key
        acc = np.zeros((left.sectors[ap][2], right.sectors[bp][2]), dtype=complex)
        y1, y2 = site[s1p][1][0], site[s2p][1][0]
        for (w, a, Lb) in lby.get(ap, []):
            for (b, w2, Rb) in rby.get(bp, []):
                for s1 in range(len(site)):
                    x1 = site[s1][1][0]
                    c = (left.sectors[a][0] + site[s1][0][0], left.sectors[a][1] + site[s1][0][1])
                    for s2 in range(len(site)):
                        x2 = site[s2][1][0]
                        coef = float(np.dot(W[w, :, y1, x1], W[:, w2, y2, x2]))
                        if coef == 0.0:
                            continue
                        blk = th.get((a, s1, c, s2, b))
                        if blk is None:
                            continue
                        acc += coef * ((Lb @ blk) @ Rb)
                        flops += 8 * (Lb.shape[0] * Lb.shape[1] * blk.shape[1] + Lb.shape[0] * blk.shape[1] * Rb.shape[1])
        out[key] = acc
    return out, flops

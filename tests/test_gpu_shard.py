"""The sharded H_eff product on one GPU: every rank's share (``tdvp_heff_apply_owned``
with the greedy partition of the output groups) computed in turn and assembled must
equal the whole product bit for bit (the same tasks and tiles run, only split over
launches), for 2 and 3 ranks, in FP64 and in the packed BF16x4 plan.  The exchange
itself is the CPU test ``test_shard_host``; no run of this build has two GPUs."""
import numpy as np
import pytest

from gpu_helpers import fill_bond_problem

pytestmark = pytest.mark.gpu

LEFT = [(1, 1, 66), (2, 0, 70), (2, 2, 20), (3, 1, 72), (4, 0, 75), (5, 1, 68)]
RIGHT = [(3, 1, 66), (4, 0, 70), (4, 2, 20), (5, 1, 72), (6, 0, 75), (7, 1, 68)]


@pytest.mark.parametrize("prec", ["fp64", "bf16x4"])
@pytest.mark.parametrize("world", [2, 3])
def test_owned_shares_assemble_the_whole_product(prec, world):
    import torch

    from paper_2606_04771_b300 import BondProblem
    from paper_2606_04771_b300.shard import partition

    bp = BondProblem(LEFT, RIGHT, symmetry="su2", precision=prec)
    _, _, _, theta, *_ = fill_bond_problem(bp, LEFT, RIGHT, True, seed=77)
    flops, block_group = bp.heff_groups()
    assert (block_group >= 0).all() and len(flops) == block_group.max() + 1
    owner, load = partition(flops.astype(float), world)
    assert load.max() <= flops.sum() / world + flops.max()  # the greedy bound: mean + largest group
    _, dims, offs, n = bp.blocks(0)
    psi = torch.from_numpy(theta).cuda()
    whole = bp.heff_apply(psi).cpu().numpy()
    got = np.full_like(whole, np.nan)
    for r in range(world):
        out = torch.full_like(psi, float("nan"))
        bp.heff_apply_owned(owner, r, psi, out)
        o = out.cpu().numpy()
        for b, (rr, cc) in enumerate(dims):
            if owner[block_group[b]] == r:
                got[offs[b]:offs[b] + rr * cc] = o[offs[b]:offs[b] + rr * cc]
            else:  # blocks of other ranks are not written
                assert np.isnan(o[offs[b]:offs[b] + rr * cc]).all()
    assert np.array_equal(got, whole)
    bp.close()

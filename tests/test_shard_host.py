"""The multi-GPU H_eff product on CPU (unmeasured on multi-GPU hardware: every run of
this build has one GPU).

The greedy partition (``tdvp_partition``, host-only) is pinned on hand cases and
against a brute-force optimum bound.  Then two gloo ranks run the sharded product's
orchestration exactly as ``paper_2606_04771_b300.shard`` does on GPUs -- output groups
(the theta blocks of one right sector, the engine's packed last stage), their flops,
the partition, each rank computing only the blocks it owns, one all-gather, and the
assembly -- with the CPU oracle standing in for the device kernels, and must
reproduce the single-rank product bit for bit.
"""
import itertools
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_hand_cases():
    from paper_2606_04771_b300.shard import partition

    owner, load = partition([5, 3, 3, 2, 2, 1], 2)
    # largest first, each to the lighter rank: 5 -> 0 (5), 3 -> 1 (3), 3 -> 1 (6),
    # 2 -> 0 (7), 2 -> 1 (8), 1 -> 0 (8)
    assert load.tolist() == [8.0, 8.0]
    assert owner.tolist() == [0, 1, 1, 0, 1, 0]
    owner, load = partition([1.0] * 7, 3)
    assert sorted(load.tolist()) == [2.0, 2.0, 3.0] and owner.tolist() == [0, 1, 2, 0, 1, 2, 0]
    owner, load = partition([4.0], 3)
    assert owner.tolist() == [0] and load.tolist() == [4.0, 0.0, 0.0]
    owner, load = partition([], 2)
    assert len(owner) == 0 and load.tolist() == [0.0, 0.0]


def test_partition_within_the_lpt_bound_of_the_optimum():
    """Graham's bound: the greedy makespan is at most 4/3 - 1/(3m) of the optimum
    (brute force over all assignments of up to 8 units)."""
    from paper_2606_04771_b300.shard import partition

    rng = np.random.default_rng(3)
    for _ in range(30):
        n, m = int(rng.integers(1, 9)), int(rng.integers(2, 4))
        c = rng.integers(1, 20, size=n).astype(float)
        owner, load = partition(c, m)
        assert np.allclose([c[owner == r].sum() for r in range(m)], load)
        best = min(max(sum(c[i] for i in range(n) if a[i] == r) for r in range(m))
                   for a in itertools.product(range(m), repeat=n))
        assert load.max() <= (4.0 / 3.0 - 1.0 / (3 * m)) * best + 1e-12


def _problem():
    import synth
    from oracle import heff

    left = [(3, 1, 7), (4, 0, 9), (3, -1, 5), (5, 0, 4)]
    right = [(5, 1, 6), (6, 0, 8), (5, -1, 7), (7, 0, 3)]
    lb, rb = heff.Bond(left, False), heff.Bond(right, False)
    th_keys = heff.theta_blocks(lb, rb)
    lk, rk = heff.left_env_blocks(lb, lb), heff.right_env_blocks(rb, rb)
    dims = [(lb.sectors[k[0]][2], rb.sectors[k[4]][2]) for k in th_keys]
    th = synth.random_blocks(41, dims)
    Lb = synth.random_blocks(42, [(lb.sectors[k[0]][2], lb.sectors[k[2]][2]) for k in lk])
    Rb = synth.random_blocks(43, [(rb.sectors[k[0]][2], rb.sectors[k[2]][2]) for k in rk])
    return lb, rb, th_keys, dims, th, lk, Lb, rk, Rb


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import blockwise, heff
    from paper_2606_04771_b300.shard import dist_all_gather, gather_blocks, partition

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    lb, rb, keys, dims, th, lk, Lb, rk, Rb = _problem()
    W = heff.shiba_mpo_tensor(1.0, 4.0)
    sizes = [r * c for r, c in dims]
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int).tolist()
    # output groups: the blocks of one right sector; their flops from the oracle's count
    sectors = sorted({k[4] for k in keys})
    block_group = [sectors.index(k[4]) for k in keys]
    flops = np.zeros(len(sectors))
    for b, k in enumerate(keys):
        _, f = blockwise.heff2_u1_blocks(lb, rb, keys, th, lk, Lb, rk, Rb, W, [k])
        flops[block_group[b]] += f
    group_owner, _ = partition(flops, ws)
    block_rank = [int(group_owner[g]) for g in block_group]
    local = torch.zeros(sum(sizes), dtype=torch.complex128)
    mine = [k for b, k in enumerate(keys) if block_rank[b] == rank]
    got, _ = blockwise.heff2_u1_blocks(lb, rb, keys, th, lk, Lb, rk, Rb, W, mine)
    for b, k in enumerate(keys):
        if block_rank[b] == rank:
            local[offsets[b]:offsets[b] + sizes[b]] = torch.from_numpy(got[k].reshape(-1))
    full = gather_blocks(local, block_rank, offsets, sizes, rank, ws, dist_all_gather())
    q.put((rank, full.numpy(), sorted(set(block_rank))))
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_product():
    import torch.multiprocessing as mp

    from oracle import blockwise, heff

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted((q.get(timeout=300) for _ in ps), key=lambda x: x[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    lb, rb, keys, dims, th, lk, Lb, rk, Rb = _problem()
    ref, _ = blockwise.heff2_u1_blocks(lb, rb, keys, th, lk, Lb, rk, Rb, heff.shiba_mpo_tensor(1.0, 4.0), keys)
    want = np.concatenate([ref[k].reshape(-1) for k in keys])
    assert out[0][2] == [0, 1]  # both ranks own work
    for rank, full, _ in out:
        assert np.array_equal(full, want), rank

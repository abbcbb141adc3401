"""One effective-Hamiltonian product shared by several GPUs (Sec. S2.3, "GPU
acceleration": the block products are spread over the GPUs with greedy load
balancing, here one process per GPU).

The last GEMM stage of H_eff.psi writes every output block from one task (an
output group).  The groups are shared out by the library's greedy partition of
their flops (``tdvp_partition``); each rank runs the first stages in full and its
own groups (``tdvp_heff_apply_owned``), then the ranks exchange their output
blocks with one all-gather, so that every rank holds the whole product for its
replicated Lanczos recurrence.  Argument marshalling and the exchange only: the
arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import check, lib


def partition(costs, nranks):
    """(owner, load): the rank of each unit and the summed cost per rank."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    owner = np.zeros(len(c), dtype=np.int32)
    load = np.zeros(nranks, dtype=np.float64)
    check(lib().tdvp_partition(len(c), c.ctypes.data if len(c) else None, int(nranks),
                               owner.ctypes.data if len(c) else None, load.ctypes.data))
    return owner, load


def gather_blocks(local, block_rank, offsets, sizes, rank, world, all_gather):
    """Assemble the whole output from each rank's own blocks.

    local: this rank's output vector (1-D complex), valid on its own blocks;
    block_rank[b]: the rank that owns block b; offsets / sizes: the blocks' first
    element and element count; all_gather(tensor) -> list of the ranks' tensors (equal
    shapes).  Each rank packs its blocks in block order into a buffer padded to the
    longest rank's length, the buffers are exchanged, and every rank unpacks all."""
    import torch

    block_rank = np.asarray(block_rank)
    mine = [b for b in range(len(sizes)) if block_rank[b] == rank]
    per_rank = [int(sum(sizes[b] for b in range(len(sizes)) if block_rank[b] == r)) for r in range(world)]
    width = max(per_rank) if per_rank else 0
    buf = torch.zeros(width, dtype=local.dtype, device=local.device)
    pos = 0
    for b in mine:
        buf[pos:pos + sizes[b]] = local[offsets[b]:offsets[b] + sizes[b]]
        pos += sizes[b]
    parts = all_gather(torch.view_as_real(buf))
    out = torch.empty_like(local)
    for r in range(world):
        got = torch.view_as_complex(parts[r])
        pos = 0
        for b in range(len(sizes)):
            if block_rank[b] == r:
                out[offsets[b]:offsets[b] + sizes[b]] = got[pos:pos + sizes[b]]
                pos += sizes[b]
    return out


def dist_all_gather(group=None):
    """all_gather over a torch.distributed group (NCCL for device tensors, gloo for host)."""
    import torch
    import torch.distributed as dist

    def ag(t):
        t = t.contiguous()
        parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, t, group=group)
        return parts

    return ag


class ShardedHeff:
    """H_eff.psi of a bond problem shared over the ranks of a process group."""

    def __init__(self, bp, rank, world, all_gather):
        self.bp, self.rank, self.world, self.all_gather = bp, rank, world, all_gather
        flops, self.block_group = bp.heff_groups()
        self.group_owner, self.load = partition(flops.astype(np.float64), world)
        _, dims, offs, self.n = bp.blocks(0)
        self.offsets = [int(o) for o in offs]
        self.sizes = [int(r) * int(c) for r, c in dims]
        self.block_rank = np.array([self.group_owner[g] for g in self.block_group], dtype=np.int32)

    def apply(self, psi):
        """The whole H_eff psi on every rank (psi and the result: device tensors)."""
        out = psi.new_zeros(psi.shape)
        self.bp.heff_apply_owned(self.group_owner, self.rank, psi, out)
        return gather_blocks(out, self.block_rank, self.offsets, self.sizes, self.rank, self.world, self.all_gather)

"""The offline stage split across GPUs by patches.

The local solves of Algorithm alg:summary are independent from patch to patch
(the offline loop over m), so the patches are the unit of work to share out.
One process per GPU (torchrun): the patches are dealt to the ranks by the
longest-processing-time rule on their local-solve work (columns times interior
unknowns of the buffered patch); each rank solves its share
(msp_sample_patch_list); then every snapshot block is broadcast from the rank
that computed it, so that every rank holds the whole snapshot set and runs the
extraction and the online stage as a replica.  The broadcast is the only data
exchanged, once per offline stage.  Serving needs no split: each GPU serves its
own requests from a replica of the bases.

The functions take plain callables for reading and writing a patch's block, so
the same code runs on device tensors over NCCL and on host tensors over gloo.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch


def patch_costs(infos: Sequence) -> list:
    """Local-solve work of each patch: its columns times the interior unknowns of
    its buffered patch (infos: objects with X0, X1, Y0, Y1, cols)."""
    return [float(p.cols) * max(p.X1 - p.X0 - 1, 0) * max(p.Y1 - p.Y0 - 1, 0) for p in infos]


def lpt_partition(costs: Sequence[float], world: int) -> list:
    """Longest processing time first: patches in decreasing cost (ties by index)
    go to the rank with the least work so far (ties to the lowest rank).  Every
    rank computes the same partition from the same costs.  Returns per rank the
    sorted list of its patches."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for m in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(m)
        load[r] += costs[m]
    return [sorted(p) for p in parts]


def owners(parts: Sequence[Sequence[int]], n: int) -> list:
    """Rank that computes each of the n patches."""
    own = [-1] * n
    for r, p in enumerate(parts):
        for m in p:
            own[m] = r
    if min(own, default=0) < 0:
        raise ValueError("the partition does not cover every patch")
    return own


def exchange_blocks(n: int, owner: Sequence[int], rank: int, shape_of: Callable[[int], tuple],
                    get_block: Callable[[int], torch.Tensor], set_block: Callable[[int, torch.Tensor], None],
                    device, group=None):
    """Broadcast every patch's block from its owner, in patch order; each rank
    writes the blocks it did not compute.  Blocks are FP64 tensors."""
    import torch.distributed as dist
    for m in range(n):
        if owner[m] == rank:
            buf = get_block(m).to(device=device, dtype=torch.float64).contiguous()
        else:
            buf = torch.empty(shape_of(m), dtype=torch.float64, device=device)
        dist.broadcast(buf, src=owner[m], group=group)
        if owner[m] != rank:
            set_block(m, buf)


def sharded_sample(med, seed: int, precision: str, tol: float, max_iter: int, rank: int, world: int, group=None):
    """The offline local solves of a medium (paper_1807_08848_gb300.Medium) split
    across the ranks of the default process group, then the snapshot blocks
    exchanged: on return every rank's medium holds every patch's snapshots.
    Returns (partition, this rank's solve statistics)."""
    infos = [med.patch(m) for m in range(med.n_patches)]
    parts = lpt_partition(patch_costs(infos), world)
    st = med.sample_patches(parts[rank], seed, precision, tol=tol, max_iter=max_iter)
    if world > 1:
        own = owners(parts, med.n_patches)
        exchange_blocks(med.n_patches, own, rank, lambda m: (infos[m].n_k, infos[m].cols), med.snapshots,
                        med.set_snapshots, "cuda", group)
    return parts, st

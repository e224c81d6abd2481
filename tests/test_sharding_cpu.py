"""The offline stage split across ranks by patches, on CPU: the partition rule
and the exchange of snapshot blocks between two gloo ranks.  The ranks run the
oracle as their local solver, so the test needs no GPU: after the exchange every
rank must hold every patch's block exactly as a single process computes it, and
the bases built from them must match too."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import elliptic as E
from paper_1807_08848_gb300 import sharding


class _Info:
    def __init__(self, P, cols):
        self.X0, self.X1, self.Y0, self.Y1 = P.X0, P.X1, P.Y0, P.Y1
        self.cols = cols


def _infos(N, ps):
    pts = E.patch_boxes(N, ps)
    out = []
    for P in pts:
        ring = E.ring_nodes(P.X0, P.X1, P.Y0, P.Y1)
        n_b = int(np.sum((ring[:, 0] == 0) | (ring[:, 0] == N) | (ring[:, 1] == 0) | (ring[:, 1] == N)))
        out.append(_Info(P, P.S + n_b))
    return out


def test_lpt_partition_covers_and_balances():
    for N, ps in ((2048, synth.workload_batched()["patches"]), (1024, synth.workload_uneven()["patches"])):
        costs = sharding.patch_costs(_infos(N, ps))
        for world in (1, 2, 3, 8):
            parts = sharding.lpt_partition(costs, world)
            flat = sorted(m for p in parts for m in p)
            assert flat == list(range(len(costs)))
            own = sharding.owners(parts, len(costs))
            assert all(m in parts[own[m]] for m in range(len(costs)))
            loads = [sum(costs[m] for m in p) for p in parts]
            # the LPT bound: no rank exceeds the mean by more than the largest single patch
            assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
            assert sharding.lpt_partition(costs, world) == parts        # every rank computes the same split
    with pytest.raises(ValueError):
        sharding.owners([[0, 1], [3]], 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workload_small()
    N = 128
    aE, aN = E.face_coefficients(w["medium"])
    pts = E.patch_boxes(N, w["patches"])
    infos = _infos(N, w["patches"])
    parts = sharding.lpt_partition(sharding.patch_costs(infos), world)
    own = sharding.owners(parts, len(pts))
    blocks = {m: torch.tensor(E.snapshots(aE, aN, pts[m], w["seed"], N)) for m in parts[rank]}
    sharding.exchange_blocks(len(pts), own, rank, lambda m: (pts[m].n_k, infos[m].cols), lambda m: blocks[m],
                             lambda m, t: blocks.__setitem__(m, t.clone()), "cpu")
    out[rank] = ({m: blocks[m].numpy() for m in range(len(pts))}, [len(p) for p in parts])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_exchange_every_block():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    w = synth.workload_small()
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    for r in range(world):
        blocks, sizes = out[r]
        assert sum(sizes) == 16 and min(sizes) >= 1
        for m in range(16):
            np.testing.assert_array_equal(blocks[m], off.R[m])
            q, s = E.basis(blocks[m], w["tau"])
            assert q.shape[1] == off.Q[m].shape[1]
            np.testing.assert_array_equal(s, off.sigma[m])

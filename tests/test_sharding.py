"""Sharding of nodes across ranks, exercised with world_size-2 gloo ranks on
CPU (no GPU): each rank's batches are disjoint from the other's in every
step, one sweep of steps covers every node once, and gathering the per-rank
results reproduces the single-rank vector."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1907_02604_gb300.sharding import batch_slice, gather_density


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_nodes, bs, q):
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_batches = n_nodes // bs
    steps = n_batches // world
    mine = []
    for step in range(steps):
        sl = batch_slice(n_nodes, bs, world, rank, step)
        mine.extend(range(sl.start, sl.stop))
    t = torch.tensor(mine, dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([len(mine)]))
    gathered = [torch.zeros(int(s.item()), dtype=torch.int64) for s in sizes]
    dist.all_gather(gathered, t)
    # the max-over-ranks timing reduction used by the benchmark
    el = torch.tensor([float(rank + 1)])
    dist.all_reduce(el, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((np.concatenate([g.numpy() for g in gathered]).tolist(), float(el.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_nodes_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n_nodes, bs, world = 64, 8, 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_nodes, bs, q)) for r in range(world)]
    for p in procs:
        p.start()
    nodes, el = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(nodes) == list(range(n_nodes))
    assert el == 2.0


def test_batch_slice_properties():
    for world in (1, 2, 4, 8):
        seen = []
        for step in range(4096 // 256 // world):
            for rank in range(world):
                sl = batch_slice(4096, 256, world, rank, step)
                seen.extend(range(sl.start, sl.stop))
        assert sorted(seen) == list(range(4096))
    with pytest.raises(ValueError):
        batch_slice(10, 0, 1, 0, 0)


def test_gather_density():
    rho = np.arange(10.0)
    slices = [slice(0, 5), slice(5, 10)]
    out = gather_density([rho[s] for s in slices], slices, 10)
    np.testing.assert_array_equal(out, rho)

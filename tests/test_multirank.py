"""Sample sharding across ranks (the multi-GPU path) on CPU gloo ranks.

Each rank computes its block of the level's samples with the oracle, the level
sums are all-reduced, and the result equals the single-process sums over the
union of the blocks (counter-based normals make the partition irrelevant)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads
from oracle import covariance as ocv
from oracle import embedding as oem
from oracle import mlmc as omlmc


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup():
    e = oem.setup_embedding(ocv.MATERN, 0.5, 0.3, 1.0, 8, oem.PAD_DOUBLING)
    mf, mc = omlmc.default_masks(e, smoothing=False, finest=True)
    return e, mf, mc


def _rank_main(rank, world, port, N, steps, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    e, mf, mc = _setup()
    acc = torch.zeros(5, dtype=torch.float64)
    for step in range(steps):
        first = workloads.shard_first_sample(step, rank, world, N)
        sums, _ = omlmc.level_estimate(e, mf, mc, 0, 1, first, N, qoi_index=0)
        t = torch.tensor(sums, dtype=torch.float64)
        dist.all_reduce(t)
        acc += t
    if rank == 0:
        out_q.put(acc.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_level_sums_equal_single_process():
    world, N, steps = 2, 3, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, N, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    e, mf, mc = _setup()
    sums, _ = omlmc.level_estimate(e, mf, mc, 0, 1, 0, world * N * steps, qoi_index=0)
    assert got[0] == world * N * steps
    assert np.allclose(got[1:], np.array(sums[1:]), rtol=1e-13, atol=1e-15)


def test_shard_ranges_tile_without_overlap():
    seen = set()
    for step in range(5):
        for rank in range(4):
            f = workloads.shard_first_sample(step, rank, 4, 7)
            r = set(range(f, f + 7))
            assert not (r & seen)
            seen |= r
    assert seen == set(range(5 * 4 * 7))

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


# ---- the benchmark's own sharding step (bench.sharded_step_sums) on gloo ranks
_LEVELS = [(0, 4, 3), (1, 8, 2)]     # (level, n, N): a two-level hierarchy


def _oracle_level_runner():
    embs = {}
    for (l, n, _) in _LEVELS:
        e = oem.setup_embedding(ocv.MATERN, 0.5, 0.3, 1.0, n, oem.PAD_DOUBLING)
        embs[l] = (e, *omlmc.default_masks(e, smoothing=False, finest=l == 1))

    def run_levels(tasks):
        out = []
        for (l, first, N) in tasks:
            e, mf, mc = embs[l]
            out.append(omlmc.level_estimate(e, mf, mc, 5, l, first, N, qoi_index=0)[0])
        return out
    return run_levels


def _bench_rank_main(rank, world, port, steps, out_q):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    run_levels = _oracle_level_runner()
    acc = torch.zeros(len(_LEVELS), 5, dtype=torch.float64)
    for step in range(steps):
        acc += bench.sharded_step_sums(run_levels, _LEVELS, step, rank, world)
    slowest = bench.max_over_ranks(float(rank + 1), world)
    if rank == 0:
        out_q.put((acc.numpy(), slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_sharded_step_equals_single_rank_steps():
    """Two gloo ranks through bench.sharded_step_sums: step s of the sharded
    run holds the samples of single-rank steps 2s and 2s+1, so its all-reduced
    level sums equal theirs bit for bit; max_over_ranks returns the largest
    rank's value."""
    import bench
    world, steps = 2, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank_main, args=(r, world, port, steps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    run_levels = _oracle_level_runner()
    want = torch.zeros(len(_LEVELS), 5, dtype=torch.float64)
    for s in range(steps):
        want += (bench.sharded_step_sums(run_levels, _LEVELS, 2 * s, 0, 1) +
                 bench.sharded_step_sums(run_levels, _LEVELS, 2 * s + 1, 0, 1))
    assert np.array_equal(got, want.numpy())
    assert got[0, 0] == world * steps * 3 and got[1, 0] == world * steps * 2
    assert slowest == 2.0

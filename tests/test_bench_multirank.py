"""The N > 1 bench path: replicas, barrier, max-over-ranks timing (CPU, gloo, 2 ranks).

Each rank runs an independent replica (a film pair does not shard); the job's
time is the slowest rank's and its rate counts the units of every rank.  Two
gloo processes on 127.0.0.1 exercise exactly the aggregation bench.py uses.
"""

import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, local = bench.dist_info()
    assert (r, w, local) == (rank, world, rank)
    my_seconds = 1.0 + rank          # rank 1 is the slow one
    dist.barrier()
    t = bench.max_over_ranks(my_seconds, world, "cpu")
    rate = bench.whole_job_rate(1000, 10, t, world)
    out[rank] = (t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_timing_and_whole_job_rate():
    world = 2
    port = _free_port()
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, rate = res[0]
    assert t == pytest.approx(2.0)
    assert rate == pytest.approx(1000 * 10 * 2 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 4, 2.0, 1) == 20.0


def _batch_worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads

    specs = workloads.batch_pairs(256, seed=0)
    mine, lanes = bench.batch_shard(specs, world, rank, 16)
    got = [None] * world
    dist.all_gather_object(got, (mine, lanes))
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_batch_shard_covers_every_pair_once():
    """Under torchrun the 256-pair batch is spread over the ranks (no data-path
    collective): every pair on exactly one rank, the ranks' loads within one
    pair's cost of each other, every lane index in range."""
    from paper_1801_04181_gb300.build import build

    build()
    world = 2
    port = _free_port()
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_batch_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    shards = res[0]
    import bench
    import workloads

    specs = workloads.batch_pairs(256, seed=0)
    allp = sorted(i for mine, _ in shards for i in mine)
    assert allp == list(range(256))
    loads = [sum(bench.batch_cost(specs[i]) for i in mine) for mine, _ in shards]
    assert abs(loads[0] - loads[1]) <= max(bench.batch_cost(fp) for fp in specs)
    for mine, lanes in shards:
        assert len(lanes) == len(mine) and all(0 <= l < 16 for l in lanes)

"""The bench's multi-rank logic (one replica per GPU, no data-path collective)
on two CPU processes with the gloo backend: group set-up, barrier, the
max-over-ranks step time, per-rank noise seeds and the whole-job rate."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    import torch.distributed as dist
    bench.init_group(world, rank, "gloo")
    bench.barrier(world)
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, device="cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(0, rank))
    q.put((rank, ms, seeds, bench.job_rate(world, 256, ms)))
    dist.destroy_process_group()


def test_two_rank_replicas_on_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, seeds, rate in out:
        assert ms == 150.0                      # the slowest rank's time on every rank
        assert len(set(seeds)) == world         # independent noise per replica
        assert rate == pytest.approx(2 * 256 / 0.15)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.rank_seed(7, 0) == 7
    assert bench.job_rate(1, 256, 250.0) == pytest.approx(1024.0)

"""The bench's multi-rank logic (one replica per GPU, no data-path collective)
on two CPU processes with the gloo backend: group set-up, barrier, the
max-over-ranks step time, the per-rank sample ranges and the whole-job rate."""
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
    ranges = [None] * world
    dist.all_gather_object(ranges, bench.rank_samples(rank, 256))
    q.put((rank, ms, ranges, bench.job_rate(world, 256, ms)))
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
    for rank, ms, ranges, rate in out:
        assert ms == 150.0                      # the slowest rank's time on every rank
        # the ranks' sample ranges are disjoint and together cover 0 .. world*256 - 1
        covered = sorted(s for first, n in ranges for s in range(first, first + n))
        assert covered == list(range(world * 256))
        assert rate == pytest.approx(2 * 256 / 0.15)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.rank_samples(0, 256) == (0, 256) and bench.rank_samples(3, 64) == (192, 64)
    assert bench.job_rate(1, 256, 250.0) == pytest.approx(1024.0)


def test_reference_arm_json_contract():
    # the reference arm times the oracle on the host cores and prints one JSON line
    # with the contract's keys; it needs no GPU
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=root, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "samples/s" and line["higher_is_better"] is True
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 0 and line["value"] > 0
    assert line["ms_per_step"] > 0 and line["config"]["workload"] == "sphere_p2_j6_mixed_s256"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 runs the reference arm; the others exit 0 without work
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and res.stdout.strip() == "", (res.stdout, res.stderr[-1000:])

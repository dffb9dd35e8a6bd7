"""The multi-process path of the benchmark on CPU (gloo, world size 2): every
rank takes its own frames (replicas only: no collective touches the data),
the job's time is the slowest rank's, and the whole-job rate counts all
ranks' frames.  The reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        sys.path.insert(0, ROOT)
        import bench
        F = 8
        first = bench.first_frame(rank, F)
        seconds = bench.max_over_ranks(0.5 + rank, world, "cpu")   # rank 1 is the slow one
        out.put((rank, list(range(first, first + F)), seconds, bench.job_rate(world, F, seconds)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_disjoint_frames_and_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    frames = [set(r[1]) for r in res]
    assert not (frames[0] & frames[1]) and len(frames[0] | frames[1]) == 16
    assert all(r[2] == 1.5 for r in res)                 # both ranks see the max
    assert all(r[3] == pytest.approx(2 * 8 / 1.5) for r in res)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_bench_helpers_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.first_frame(3, 64) == 192
    assert bench.job_rate(4, 64, 0.5) == 512.0
    line = json.dumps({"x": bench.job_rate(1, 64, 0.032)})
    assert json.loads(line)["x"] == pytest.approx(2000.0)

"""The N > 1 path of bench.py on CPU: two gloo ranks run the host logic that
the GPU ranks run (barrier, maximum time over ranks, whole-job value), and
the reference arm under torchrun prints its one line from rank 0 only."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        bench.barrier(world)
        ms = [7.5, 9.25][rank]  # the second rank is the slowest
        slowest = bench.max_over_ranks(ms, world, torch.device("cpu"))
        value = bench.whole_job_mlups(world, 1000, 20, slowest)
        bench.barrier(world)
        out.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_whole_job_value():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, slowest, value in got:
        assert slowest == 9.25
        # two replicas of 1000 nodes, 20 steps in 9.25 ms
        assert value == pytest.approx(2 * 1000 * 20 / 9.25e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.0, 1, None) == 3.0
    bench.barrier(1)
    assert bench.whole_job_mlups(1, 4096 * 4096, 2000, 1376.0) == pytest.approx(24385.4, rel=1e-4)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """torchrun with two ranks on the host: rank 0 times the oracle (a small
    window, about a second) and prints the JSON line; rank 1 exits 0 silently."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"), "--impl",
           "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--reference-seconds", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

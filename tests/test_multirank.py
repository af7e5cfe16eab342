"""The N > 1 path of bench.py on CPU: world_size 2 over gloo.

Each rank is a replica that moves its own copy of the workload, so the only
exchanges are the barriers around the timed region and the max over ranks of
the elapsed time; the whole-job value sums bytes over ranks. Under torchrun the
reference arm runs on rank 0 alone and the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = [12.5, 40.0][rank]          # the ranks' own timed regions
        job_ms = bench.max_over_ranks(ms, dist, "cpu")
        dist.barrier()
        out[rank] = (job_ms, bench.job_value(world, 10**9, 4, job_ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_bytes():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1]
    job_ms, value = out[0]
    assert job_ms == 40.0
    assert value == pytest.approx(2 * 4 * 1e9 / 0.040 / 1e9)


def test_single_process_has_no_exchange():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 2 * 10**9, 10, 1000.0) == pytest.approx(20.0)


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0

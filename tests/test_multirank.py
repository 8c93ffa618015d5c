"""The host side of `bench.py --gpus N` (replicas: one process per GPU, no
data-path collective), run as world_size-2 gloo ranks on the CPU: the job's
time is the slowest rank's, its throughput all ranks' units over that time,
and the reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    ms_local = [12.5, 30.0][rank]  # rank 1 is the slow replica
    ms = bench.rank_max(ms_local, ws, torch.device("cpu"))  # joins a gloo group
    rate = bench.job_rate(1000, ms, ws)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate, "backend": dist.get_backend()}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_every_rank(tmp_path):
    ws = 2
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    for g in got:
        assert g["backend"] == "gloo"
        assert g["ms"] == 30.0
        assert g["rate"] == pytest.approx(2 * 1000 / 30e-3)


def test_one_rank_needs_no_process_group():
    assert bench.rank_max(7.0, 1, torch.device("cpu")) == 7.0
    assert bench.job_rate(500, 10.0, 1) == pytest.approx(5e4)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""

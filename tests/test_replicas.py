"""Replica aggregation across processes (gloo, world size 2, CPU) and the bench's
CPU reference arm."""
import json
import os
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_00737_gb300 import replicas as RP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 200.0][rank]           # rank 1 is the slower replica
    value, ms = RP.job_throughput(1024 * 10, local_ms, world)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_throughput_is_all_queries_over_the_slowest_rank():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, 29517, out), nprocs=2, join=True,
                       start_method="spawn")
    for rank in range(2):
        value, ms = out[rank]
        assert ms == 200.0
        assert abs(value - 2 * 10240 / 0.2) < 1e-6


def test_without_a_process_group_the_local_time_is_used():
    value, ms = RP.job_throughput(1000, 50.0, 1)
    assert ms == 50.0 and abs(value - 20000.0) < 1e-9


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "small", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "queries/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_once():
    """Under torchrun (2 ranks on the CPU) only rank 0 runs and prints the reference
    line; the other rank exits 0 without work."""
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", "29533", os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--workload", "small", "--steps", "1",
                        "--warmup", "1", "--gpus", "2"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2

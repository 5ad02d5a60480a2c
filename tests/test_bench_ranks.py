"""The N > 1 path of bench.py on CPU: world_size 2 over gloo (127.0.0.1).

The bench runs replicas (one independent solve per rank, no collective on the data path).
Its only cross-rank steps are the barrier around the timed region and the maximum of the
per-rank timings; the whole-job value is the units all ranks processed over that time.
The reference arm runs on rank 0 alone, and the other ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.0 + rank, 10.0 - rank, 5.0]   # per-rank times (s)
        dist.barrier()
        got = bench.max_over_ranks(local, dist)
        ref = bench.run_reference(None, rank, world) if rank != 0 else "rank0"
        q.put((rank, got, ref))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, ref in res:
        assert got == [2.0, 10.0, 5.0]          # the slowest rank's time, on every rank
        if rank != 0:
            assert ref is None                   # the reference arm: rank 0 only
    # whole-job throughput: 5 steps on each of 2 ranks in 2 s (the max over ranks)
    assert bench.job_rate(5, 2, 2.0) == 5.0
    assert bench.max_over_ranks([3.0, 4.0], None) == [3.0, 4.0]


def test_reference_arm_under_torchrun_world_size_2():
    """`bench.py --impl reference` launched like the driver's N > 1 runs: one JSON line from
    rank 0 with impl = reference and n_gpus = 2; both ranks exit 0."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["e2e"]["h2d_bytes_per_step"] == 0

"""Multi-rank (replicas) host logic of bench.py on CPU with the gloo backend.

The engine runs one replica per GPU with no data-path collective; the only
cross-rank step is the timing reduction (max over ranks of each rank's time for
its own iterations), covered here with world_size 2 on CPU.  The reference arm
under torchrun prints one line from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    v = bench.job_ms_per_iteration(local_ms[rank], steps, world, "cpu")
    q.put((rank, v))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_slowest_rank_over_all_iterations():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, steps = 2, 5
    local_ms = [40.0, 55.0]  # each rank's total time for its `steps` iterations
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, local_ms, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # whole job: 2 x 5 iterations in the slowest rank's 55 ms
    assert got[0] == pytest.approx(55.0 / (steps * world))
    assert got[1] == got[0]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_ms_per_iteration(12.0, 4, 1) == pytest.approx(3.0)


def test_reference_arm_prints_from_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "square4", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0

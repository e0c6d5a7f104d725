"""Multi-rank host logic of bench.py on CPU with gloo, world size 2 (the
GPU runs are replicas: one process per GPU, no data-path collective).  The
timing reduction takes the slowest rank, the whole-job rate counts every
rank's units, and the reference arm runs and prints on rank 0 only."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
    dist.barrier()
    q.put((rank, ms, bench.job_rate(1000, world, ms)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 15.0                       # the slower rank's time
        assert rate == pytest.approx(2 * 1000 / 15e-3)


def test_reference_arm_prints_on_rank_zero_only():
    base = [sys.executable, "bench.py", "--impl", "reference", "--workload", "batch64",
            "--steps", "1", "--warmup", "0", "--gpus", "2"]
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r1 = subprocess.run(base, cwd=ROOT, env=dict(env, RANK="1", LOCAL_RANK="1"),
                        capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(base, cwd=ROOT, env=dict(env, RANK="0", LOCAL_RANK="0"),
                        capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0

"""Replicas-only multi-GPU logic of bench.py, run as two gloo ranks on the CPU: disjoint replica seeds,
max-over-ranks time, whole-job throughput; and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 * (rank + 1)          # rank 1 is the slow one
    value, ms_max = bench.aggregate(ms_local, m=8, K=10, world=world, dist=dist)
    q.put((rank, bench.rank_seed(rank), value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_with_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, v0, t0), (r1, s1, v1, t1) = out
    assert s0 != s1                                   # disjoint replicas
    assert t0 == t1 == 200.0                          # both ranks see the slowest rank's time
    assert abs(v0 - 2 * 8 * 10 / 0.2) < 1e-9 and v0 == v1


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "updates/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

"""The multi-rank bench path on CPU: two gloo ranks, max-over-ranks timing and whole-job
throughput of independent replicas; the reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
r = dist.get_rank()
ms = 100.0 * (r + 1)                       # rank 1 is the slowest
v, mx = bench.job_throughput(50.0, ms)     # 50 sweeps per rank
print(json.dumps({"rank": r, "value": v, "ms": mx}))
dist.destroy_process_group()
"""


def _spawn(world, port, code, extra_env=None, args=()):
    procs = []
    for rank in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_two_gloo_ranks_take_the_slowest_and_sum_the_work():
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _spawn(2, 29611, WORKER)]
    for o in outs:
        assert o["ms"] == 200.0                 # max over ranks
        assert o["value"] == pytest.approx(2 * 50.0 / 0.2)  # all ranks' sweeps / slowest time


def test_single_process_without_group():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.job_throughput(10.0, 500.0)
    assert ms == 500.0 and v == pytest.approx(20.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""

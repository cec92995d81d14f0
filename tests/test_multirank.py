"""The multi-process harness of bench.py on CPU with gloo, world size 2: each rank draws its own
queries, the step time is the max over ranks, and the job throughput counts every rank's queries."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import bench
from synth import WORKLOADS, interior_box, make_rng, uniform_points
rk = bench.Ranks("gloo")
wl = WORKLOADS["bcc_quintic_128"]
lo, hi = interior_box(wl.spline, wl.dims)
pts = uniform_points(make_rng(rk.query_seed(wl.seed), 0), 64, lo, hi)
my_ms = 10.0 + 5.0 * rk.rank                      # rank 1 is the slow one
rk.barrier()
mx = rk.max_over_ranks(my_ms)
out = {"rank": rk.rank, "world": rk.world, "first": pts[0].tolist(), "max_ms": mx,
       "throughput": rk.job_throughput(len(pts), mx)}
rk.close()
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_gloo():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(__import__("json").loads(o.strip().splitlines()[-1]))
    a, b = sorted(outs, key=lambda d: d["rank"])
    assert a["world"] == b["world"] == 2
    assert a["first"] != b["first"]                 # independent query shards
    assert a["max_ms"] == b["max_ms"] == 15.0       # the slowest rank's time
    assert a["throughput"] == b["throughput"] == 2 * 64 / 15e-3

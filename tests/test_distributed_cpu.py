"""Host-side multi-process logic of bench.py on CPU (gloo, world size 2).

The predictor shards over elements with no data-path collective; across ranks
the bench only needs a barrier and the max of the timed region. These tests
run that logic as two gloo processes, and the reference arm under two ranks
(rank 0 alone prints; the other exits without work).
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank()
world = dist.get_world_size()
bench.barrier(world)
m = bench.max_over_ranks(10.0 + rank, world)
# the bench's weak-scaling value: units of all ranks / max time
value = 1000 * world / m
print(json.dumps({{"rank": rank, "max": m, "value": value}}), flush=True)
dist.destroy_process_group()
"""


def run_ranks(code: str, world: int = 2, extra_env=None):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_max_over_ranks_and_weak_scaling_value_gloo():
    outs = run_ranks(WORKER.format(root=ROOT))
    recs = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in recs) == [0, 1]
    for r in recs:
        assert r["max"] == 11.0
        assert r["value"] == pytest.approx(2000 / 11.0)


def test_reference_arm_two_ranks_only_rank0_prints():
    code = ("import sys; sys.argv = ['bench.py', '--impl', 'reference', '--gpus', '2', "
            "'--steps', '1', '--warmup', '0', '--workload', 'order3', '--reference-sample', '16']; "
            f"sys.path.insert(0, {ROOT!r}); import bench; bench.main()")
    outs = run_ranks(code, extra_env={"OMP_NUM_THREADS": "2"})
    lines = [o.strip() for o in outs]
    assert lines[1] == ""  # rank 1 exits without work
    rec = json.loads(lines[0].splitlines()[-1])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["n_gpus"] == 2
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0

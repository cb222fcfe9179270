"""Host-side logic of the multi-rank benchmark (one replica per rank, barrier, max over
ranks, whole-job value) on two CPU processes over gloo; the reference arm runs on rank 0
only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys, types
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
world, rank, local = bench.dist_setup()
bench.barrier(world)
slow = bench.max_over_ranks(100.0 + 50.0 * rank, world)   # rank 1 is the slow one
value = bench.whole_job_value(1000, 4, world, slow)
bench.run_reference(types.SimpleNamespace(workload="tiny", warmup=0, steps=1, gpus=world)) if rank != 0 else None
import torch.distributed as dist
dist.destroy_process_group()
print(json.dumps({"world": world, "rank": rank, "slow": slow, "value": value}), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_over_gloo():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-2000:]
        lines = [l for l in out.splitlines() if l.startswith("{")]
        assert len(lines) == 1, out  # rank 1's reference arm printed nothing
        outs.append(json.loads(lines[0]))
    outs.sort(key=lambda d: d["rank"])
    for d in outs:
        assert d["world"] == 2
        assert d["slow"] == 150.0              # the max over ranks reaches every rank
        assert d["value"] == pytest.approx(2 * 1000 * 4 / 0.150)   # both replicas, slowest rank's time

"""bench.py host logic on CPU: the reference arm and the multi-rank aggregation.

Reads are independent, so N ranks run N replicas; torch.distributed (gloo)
carries only the barrier and the max / sum of the per-rank figures. These tests
run two gloo ranks on CPU and check that rank 0 alone prints one JSON line,
that the others exit 0, and that the whole-job value is the sum of the ranks'
bases over the slowest rank's time.
"""
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


def json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


REF_ARGS = ["--impl", "reference", "--workload", "tiny_1mbp_short", "--n-reads", "2000", "--steps", "1",
            "--warmup", "0"]


def test_reference_arm_single_rank():
    r = subprocess.run([sys.executable, "bench.py", *REF_ARGS], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    L = lines[0]
    assert L["impl"] == "reference" and L["value"] > 0 and L["higher_is_better"] is True
    assert L["unit"] == L["e2e"]["unit"] == L["cpu_baseline"]["unit"] == "read bases/s"
    assert L["e2e"]["value"] == L["value"] == L["cpu_baseline"]["value"]
    assert L["e2e"]["h2d_bytes_per_step"] == 0 and L["e2e"]["d2h_bytes_per_step"] == 0
    assert L["cpu_baseline"]["kind"] == "oracle" and L["cpu_baseline"]["cores"] >= 1
    assert L["config"]["workload"] == "tiny_1mbp_short" and L["config"]["reads"] == 2000
    # every step runs the whole batch: the timed steps fit in the measured wall time
    assert L["ms_per_step"] * L["steps"] <= L["timed_wall_s"] * 1e3 * 1.01


def test_reference_arm_two_ranks_rank0_only():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2", *REF_ARGS]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"


WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
ws, rank, local = bench.dist_setup()
assert ws == 2 and rank in (0, 1)
bench.barrier(ws)
ms = [12.0, 20.0][rank]          # per-rank mean step time
bases = [1.0e9, 3.0e9][rank]     # per-rank read bases
ms_max = bench.dist_max(ms, ws)
total = bench.dist_sum(bases, ws)
bench.barrier(ws)
print(json.dumps({"rank": rank, "ms_max": ms_max, "total": total, "value": total / (ms_max / 1e3)}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def test_gloo_aggregation_two_ranks():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("gloo rank did not finish")
        assert p.returncode == 0, e
        outs.extend(json_lines(o))
    assert len(outs) == 2
    for o in outs:
        assert o["ms_max"] == 20.0
        assert o["total"] == 4.0e9
        assert o["value"] == pytest.approx(4.0e9 / 0.020)

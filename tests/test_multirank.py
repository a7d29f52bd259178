"""The multi-process path of bench.py on CPU: two ranks over gloo.

With N GPUs the solve runs as N independent replicas (it does not shard);
the job's time is the slowest rank's and its value counts every rank's
units.  These tests run that host logic in two processes on the CPU: the
max-over-ranks reduction, the whole-job rate, the reference arm, which
only rank 0 runs and prints, and the bounded host barrier, which a rank that
raised or never arrives turns into an error on the others.
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


_WORKER = r"""
import os, sys, json
sys.path.insert(0, %r)
import torch, torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank, world = dist.get_rank(), dist.get_world_size()
# rank r reports times 10 + r and 20 - r: the job takes the largest of each
ms, e2e = bench.max_over_ranks([10.0 + rank, 20.0 - rank], world, "cpu")
rate = bench.whole_job_rate(world, 3, 1000.0, ms)
print(json.dumps({"rank": rank, "ms": ms, "e2e": e2e, "rate": rate}), flush=True)
dist.destroy_process_group()
"""


def _run_ranks(code, world=2, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code] if isinstance(code, str) else code,
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_max_over_ranks_and_rate_gloo():
    outs = _run_ranks(_WORKER % ROOT)
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for row in rows:
        assert row["ms"] == 11.0 and row["e2e"] == 20.0
        assert row["rate"] == pytest.approx(2 * 3 * 1000.0 / 0.011)


def test_reference_arm_prints_on_rank0_only():
    outs = _run_ranks([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                       "--cpu-n", "16", "--steps", "1", "--warmup", "3"])
    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "DOF/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


_FAIL_WORKER = r"""
import os, sys, json, time
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank = dist.get_rank()
mode = os.environ["FAIL_MODE"]
if rank == 1:
    if mode == "raise":
        raise RuntimeError("rank 1: a failed solve")
    time.sleep(120)          # alive, but never reaches the barrier
    sys.exit(0)
t0 = time.perf_counter()
try:
    bench.host_barrier(2, 3.0)
    out = {"raised": False}
except RuntimeError as e:
    out = {"raised": True, "msg": str(e)[:300]}
out["s"] = time.perf_counter() - t0
print(json.dumps(out), flush=True)
os._exit(0)
"""


@pytest.mark.parametrize("mode", ["raise", "absent"])
def test_host_barrier_detects_a_failed_or_absent_rank(mode):
    """A rank that raised or never arrives: the other rank's bounded host
    barrier raises within seconds instead of blocking (gloo, two ranks)."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r), FAIL_MODE=mode)
        procs.append(subprocess.Popen([sys.executable, "-c", _FAIL_WORKER % ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    try:
        o, e = procs[0].communicate(timeout=90)
    finally:
        procs[1].kill()
        procs[1].communicate()
    assert procs[0].returncode == 0, e[-2000:]
    row = json.loads(o.strip().splitlines()[-1])
    assert row["raised"], row
    assert row["s"] < 30.0, row
    assert "Ranks 1 " in row["msg"], row   # the error names the missing rank

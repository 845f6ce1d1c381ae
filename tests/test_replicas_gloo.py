"""The multi-GPU path is replicas only (one independent DAG per rank): the
ranks share the timing.  Two gloo ranks on the CPU check the job time (the
slowest rank's), the whole-job value, that only rank 0 reports, and that the
reference arm's other ranks exit without output."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
from paper_2012_09646_gb300 import replicas as RP
rank, world, local = RP.rank_env()
dist.init_process_group("gloo")
ms_local = [3.0, 5.0][rank]
ms = RP.job_time_ms(dist, ms_local)
dist.barrier()
out = {"rank": rank, "world": world, "local": local, "ms": ms, "value": RP.job_value(world, 1, ms),
       "reports": RP.reports(rank)}
print("RESULT " + json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(code, world=2, extra_args=()):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_job_time_is_the_slowest_rank():
    outs = run_ranks(WORKER)
    res = [json.loads(l[len("RESULT "):]) for o in outs for l in o.splitlines() if l.startswith("RESULT ")]
    assert len(res) == 2
    for r in res:
        assert r["ms"] == 5.0
        assert r["world"] == 2 and r["local"] == r["rank"]
        assert r["value"] == pytest.approx(2 * 1e3 / 5.0)
    assert [r["reports"] for r in sorted(res, key=lambda r: r["rank"])] == [True, False]


def test_single_process_defaults():
    from paper_2012_09646_gb300 import replicas as RP
    old = {k: os.environ.pop(k, None) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    try:
        assert RP.rank_env() == (0, 1, 0)
    finally:
        for k, v in old.items():
            if v is not None:
                os.environ[k] = v
    assert RP.job_time_ms(None, 2.5) == 2.5
    assert RP.job_value(1, 1, 2.5) == pytest.approx(400.0)


REF = r"""
import sys
sys.path.insert(0, sys.argv[1])
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
import bench
bench.main()
"""


def test_reference_arm_only_rank0_prints():
    """Under torchrun the reference arm runs on rank 0 alone; the other ranks
    exit 0 without output (rank 1 is checked here; rank 0's line is the
    oracle's timing)."""
    port = free_port()
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port))
    p = subprocess.run([sys.executable, "-c", REF, ROOT], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, "-c", REF, ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "DAG/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

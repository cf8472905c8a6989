"""The multi-rank logic of bench.py on CPU: two gloo ranks (the GPU runs are
replicas, one per GPU, with no data-path collective; only the timing is reduced)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
sys.argv = ["bench.py"]
import bench
dist.init_process_group("gloo")
rank, world, _ = bench.dist_env()
ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
print(json.dumps({"rank": rank, "world": world, "ms": ms, "rate": bench.whole_job_rate(100, world, ms)}), flush=True)
dist.destroy_process_group()
"""


def _run_ranks(script: str, world: int, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", script, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_timing_is_the_slowest_rank_and_rate_is_whole_job():
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _run_ranks(WORKER, 2)]
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2 and o["ms"] == 15.0  # max over ranks: 10 and 15 ms
        assert o["rate"] == pytest.approx(100 * 2 / 0.015)


def test_reference_arm_prints_on_rank_zero_only():
    script = r"""
import sys
sys.path.insert(0, sys.argv[1])
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
import bench
bench.main()
"""
    # rank 1 of 2 must exit 0 without work or output (rank 0 alone runs the CPU oracle)
    port = _free_port()
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    p = subprocess.run([sys.executable, "-c", script, ROOT], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""

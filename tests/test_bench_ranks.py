"""The replicas path of bench.py at world size 2, on the CPU: two gloo ranks
run the same rank helpers the benchmark uses under NCCL (barriers around the
timed region, the slowest rank's time, the units summed over ranks), and the
reference arm does its work on rank 0 only.
"""
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
import bench
dist.init_process_group("gloo", init_method="env://")
r = dist.get_rank()
ranks = bench.Ranks(dist, "cpu")
ranks.barrier()
ms = [100.0, 250.0][r]
units = [1.0e6, 3.0e6][r]
value, ms_max, total = bench.replica_throughput(ranks, ms, units)
out = {"rank": r, "value": value, "ms_max": ms_max, "total": total,
       "max_rank": ranks.max(r), "sum_launches": ranks.sum(10 + r)}
ranks.barrier()
dist.destroy_process_group()
print(json.dumps(out), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_like_the_benchmark():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        # every rank sees the slowest time and the whole job's units
        assert o["ms_max"] == 250.0
        assert o["total"] == 4.0e6
        assert o["value"] == pytest.approx(4.0e6 / 0.25, rel=1e-15)
        assert o["max_rank"] == 1.0
        assert o["sum_launches"] == 21.0


def test_one_rank_needs_no_process_group():
    import bench
    ranks = bench.Ranks(None)
    ranks.barrier()
    assert ranks.max(3) == 3.0 and ranks.sum(5) == 5.0
    value, ms_max, total = bench.replica_throughput(ranks, 200.0, 1.0e6)
    assert (value, ms_max, total) == (5.0e6, 200.0, 1.0e6)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None) is None  # returns before touching its arguments or the oracle
    assert capsys.readouterr().out == ""

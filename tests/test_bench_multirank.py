"""The host side of bench.py's N-GPU run (replicas: one system per rank, no exchange
in the solver), on CPU with two gloo ranks: process-group setup from the torchrun
environment, the max-over-ranks timing reduction, the barrier, the whole-job
aggregate and the per-rank seeds; and the cost-balanced sharding of the batching
workload's independent systems. No GPU and no library call is involved."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import torch
import bench
rank, world, local, pg = bench.dist_setup(2)
dev = torch.device("cpu")
ms = 100.0 + 50.0 * rank                 # rank 1 is the slower one
bench.barrier(pg, dev)
ms_max = bench.reduce_max(pg, ms, dev)
out = {"rank": rank, "world": world, "local": local, "ms_max": ms_max,
       "value": bench.aggregate_value(world, 10, ms_max), "seed": bench.replica_seed(rank)}
with open(os.path.join(sys.argv[2], "rank%d.json" % rank), "w") as f:
    json.dump(out, f)
pg.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), MINNORM_BENCH_BACKEND="gloo")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT, str(tmp_path)], env=env))
    for p in procs:
        assert p.wait(timeout=120) == 0
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == 2 and d["local"] == r
        assert d["ms_max"] == 150.0                       # the slowest rank's time on every rank
        assert d["value"] == pytest.approx(2 * 10 / 0.150)  # 20 solves in 0.15 s for the whole job
    assert res[0]["seed"] != res[1]["seed"]              # each replica solves its own system


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rank, world, local, pg = bench.dist_setup(1)
    assert (rank, world, local, pg) == (0, 1, 0, None)
    assert bench.reduce_max(None, 3.5, None) == 3.5
    assert bench.aggregate_value(1, 10, 250.0) == pytest.approx(40.0)


def test_batch_partition_is_a_balanced_cover():
    sys.path.insert(0, ROOT)
    import bench
    import synth
    shapes = synth.batch_shapes(256, seed=4000)
    biggest = max(bench.batch_cost(m, n) for m, n in shapes)
    for world in (1, 2, 3, 4, 8):
        parts = bench.partition_batch(shapes, world)
        assert len(parts) == world
        assert sorted(i for p in parts for i in p) == list(range(256))      # every system exactly once
        loads = [sum(bench.batch_cost(*shapes[i]) for i in p) for p in parts]
        assert max(loads) - min(loads) <= biggest                           # greedy longest-first bound
    assert bench.partition_batch(shapes, 1)[0] == list(range(256))

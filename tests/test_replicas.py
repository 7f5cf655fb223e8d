"""The multi-rank path of bench.py on the host, with two gloo ranks.

Each rank of `bench.py --gpus N` solves its own seeded replica of the workload (no
data-path collective); the ranks meet only to time the step. The whole-job value is the
sigma-vectors of all ranks over the slowest rank's time. Checked here without a GPU:
the rank environment, the barrier, the max / sum reductions behind the value, and that
the replicas draw different seeded systems of the same shape.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo")
# rank r evaluated 10 + r sigma-vectors in 1 + r seconds
value, t_max, total = bench.aggregate(10 + rank, 1.0 + rank, world)
bench.barrier(world)
spec = bench.rank_spec(rank)
print(json.dumps({{"rank": rank, "world": world, "local": local, "value": value, "t_max": t_max,
                  "total": total, "seed": spec.seed, "n_mo": spec.n_mo, "n_chol": spec.n_chol}}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_aggregate_and_replicas():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    out = []
    for p in procs:
        so, se = p.communicate(timeout=120)
        assert p.returncode == 0, se
        out.append(json.loads(so.strip().splitlines()[-1]))
    out.sort(key=lambda d: d["rank"])
    for d in out:
        assert d["world"] == 2 and d["local"] == d["rank"]
        assert d["t_max"] == 2.0 and d["total"] == 21.0
        assert d["value"] == pytest.approx(21.0 / 2.0)
    assert out[0]["seed"] != out[1]["seed"]
    assert out[0]["n_mo"] == out[1]["n_mo"] and out[0]["n_chol"] == out[1]["n_chol"]

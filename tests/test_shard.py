"""Host side of the J-sharded Jacobian transformation (mlcc_sigma_partial), without a GPU:

  * shard_range tiles [0, n_chol) with contiguous ranges in rank order whose sizes differ by
    at most one, for every split tried;
  * two gloo ranks run sharded_sum over a stand-in for the partial sigma (a sum over J of
    per-vector terms plus terms that do not sum over J): the all-reduced result equals the
    unsplit sum on both ranks, and only rank 0 contributes the terms outside the J sum.
The same path on the GPU (each rank's mlcc_sigma_partial, the gloo sum, against mlcc_sigma
and the oracle) is tests/test_gpu_shard.py.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_ranges_tile_the_cholesky_index():
    from paper_2006_05226_gb300 import mlcc
    for n_chol in (1, 2, 7, 200, 1500, 2501):
        for world in range(1, min(9, n_chol + 1)):
            rs = [mlcc.shard_range(n_chol, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n_chol
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [j1 - j0 for j0, j1 in rs]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        mlcc.shard_range(10, 2, 2)
    with pytest.raises(ValueError):
        mlcc.shard_range(3, 0, 4)                   # an empty range for some rank


WORKER = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch, torch.distributed as dist
from paper_2006_05226_gb300 import mlcc
rank, world = int(sys.argv[1]), int(sys.argv[2])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=rank, world_size=world)
nj = 37
x = np.random.default_rng(4).standard_normal((nj, 5))   # a term per Cholesky vector
rest = np.arange(5.0)                                     # the terms outside the J sum
calls = []
def partial(j0, j1, with_rest):
    calls.append((j0, j1, with_rest))
    return torch.as_tensor(x[j0:j1].sum(axis=0) + (rest if with_rest else 0.0))
out = mlcc.sharded_sum(partial, nj, rank, world)
print(json.dumps({{"rank": rank, "out": out.tolist(), "want": (x.sum(axis=0) + rest).tolist(), "calls": calls}}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_sum_their_shards():
    port = _free_port()
    src = WORKER.format(root=ROOT, port=port)
    procs = [subprocess.Popen([sys.executable, "-c", src, str(r), "2"], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    res = []
    for p in procs:
        so, se = p.communicate(timeout=120)
        assert p.returncode == 0, se
        res.append(json.loads(so.strip().splitlines()[-1]))
    res.sort(key=lambda d: d["rank"])
    for d in res:
        assert max(abs(a - b) for a, b in zip(d["out"], d["want"])) < 1e-12
    assert res[0]["calls"] == [[0, 19, True]] and res[1]["calls"] == [[19, 37, False]]

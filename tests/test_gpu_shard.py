"""The Jacobian transformation split over the Cholesky index (mlcc_sigma_partial; Sec. 2.4,
every integral a sum over J): the partial results of ranges that tile [0, n_chol), one of
them with the terms that do not sum over J, add up to mlcc_sigma and to the oracle's sigma,
element by element (binary64 and MLCC_FP64E, 1e-10 relative):

  * in one process over three uneven ranges, on MLCCSD, three-level, MLCC2 and CCS/CCSD
    partitions (the 7-orbital system, the 48-orbital workload and a ragged 37-orbital one),
    and on a CCSD block of 10 / 60 whose ladder runs on the tensor cores;
  * with two gloo ranks (two processes sharing this GPU, no kernel waiting on another rank)
    that each evaluate their half and sum the halves through host memory.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from gpu_helpers import Layout
from oracle.mlcc import MLCCSystem, sigma, solve_ground_state
from test_gpu_parity import PARTITIONS
from tiny_systems import tiny

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    from paper_2006_05226_gb300 import mlcc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mlcc.Context(0)
    yield c
    c.close()


def _inputs(case):
    from synth import CONFIGS, make_system
    from synth.generator import SystemSpec, default_scale
    if case.startswith("tiny:"):
        t = tiny()
        return t.L, t.F, t.k, np.array(dict(PARTITIONS)[case[5:]], dtype=np.int8)
    if case == "small":
        s = make_system(CONFIGS["small"])
    elif case == "ragged":
        s = make_system(SystemSpec("ragged", 6, 31, 29, 5.8, 5, 21, 2, 7, 3, 4, default_scale(5.8)))
    else:   # a CCSD block of 10 / 60: the ladder on the tensor cores in MLCC_FP64E
        s = make_system(SystemSpec("ccsd_rows", 12, 90, 300, 60.0, 12, 90, 10, 60, 3, 7, default_scale(60.0)))
    return s.L, s.fock, s.spec.n_occ, s.level


@pytest.mark.parametrize("case", ["tiny:ccsd", "tiny:three_level", "tiny:mlcc2_ccs_outer", "tiny:ccs_ccsd",
                                  "small", "ragged", "ccsd_10_60"])
def test_partial_sigmas_add_up(ctx, case):
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = _inputs(case)
    g = mlcc.System(ctx, torch.as_tensor(L, device="cuda"), torch.as_tensor(F, device="cuda"), no, lev)
    o = MLCCSystem(L, F, no, lev)
    lay = Layout(g, o)
    rng = np.random.default_rng(17)
    t1 = 0.03 * rng.standard_normal((o.nv, o.no))
    x2 = 0.03 * rng.standard_normal(o.doubles_shape())
    x2 = x2 + x2.transpose(2, 3, 0, 1)
    g.jacobian_prepare(torch.as_tensor(lay.t1(t1), device="cuda"), torch.as_tensor(lay.x2(x2).ravel(), device="cuda"))
    cs, refs = [], []
    for _ in range(2):
        c1 = rng.standard_normal((o.nv, o.no))
        c2 = rng.standard_normal(o.doubles_shape())
        c2 = c2 + c2.transpose(2, 3, 0, 1)
        s1, s2 = sigma(o, t1, x2, c1, c2)
        cs.append(lay.vec(c1, c2))
        refs.append(lay.vec(s1, s2))
    c = torch.as_tensor(np.stack(cs), device="cuda")
    ref = np.stack(refs)
    nj = L.shape[0]
    cuts = [0, max(1, nj // 5), max(2, (2 * nj) // 3), nj]
    for prec in (mlcc.MLCC_FP64, mlcc.MLCC_FP64E):
        whole = g.sigma(c, precision=prec).cpu().numpy()
        parts = [g.sigma_partial(c, cuts[k], cuts[k + 1], k == 1, prec).cpu().numpy() for k in range(3)]
        total = parts[0] + parts[1] + parts[2]
        scale = float(np.abs(ref).max())
        assert np.abs(total - whole).max() <= 1e-10 * scale, (prec, float(np.abs(total - whole).max()))
        assert np.abs(total - ref).max() <= 1e-10 * scale
        # a one-vector range with the rest terms plus the remaining range without them
        a = g.sigma_partial(c, 0, 1, True, prec).cpu().numpy()
        b = g.sigma_partial(c, 1, nj, False, prec).cpu().numpy()
        assert np.abs(a + b - whole).max() <= 1e-10 * scale
    from paper_2006_05226_gb300 import mlcc as m
    with pytest.raises(m.MLCCError) as e:
        g.sigma_partial(c, 3, 3, True)
    assert e.value.status == m.MLCC_E_ARG
    # the unsplit sigma after partial calls is unchanged (the window is restored)
    assert np.array_equal(g.sigma(c).cpu().numpy(), g.sigma(c).cpu().numpy())
    assert np.abs(g.sigma(c).cpu().numpy() - ref).max() <= 1e-10 * float(np.abs(ref).max())
    g.close()


WORKER = r"""
import json, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np, torch, torch.distributed as dist
from paper_2006_05226_gb300 import mlcc
from synth import CONFIGS, make_system
from oracle.mlcc import MLCCSystem, solve_ground_state, sigma
from gpu_helpers import Layout
rank, world = int(sys.argv[1]), int(sys.argv[2])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=rank, world_size=world)
s = make_system(CONFIGS["small"])
no = s.spec.n_occ
ctx = mlcc.Context(0)
g = mlcc.System(ctx, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, s.level)
o = MLCCSystem(s.L, s.fock, no, s.level)
gs = solve_ground_state(o)
lay = Layout(g, o)
g.jacobian_prepare(torch.as_tensor(lay.t1(gs.t1), device="cuda"), torch.as_tensor(lay.x2(gs.x2).ravel(), device="cuda"))
rng = np.random.default_rng(2)
c1 = rng.standard_normal((o.nv, o.no)); c2 = rng.standard_normal(o.doubles_shape()); c2 = c2 + c2.transpose(2, 3, 0, 1)
c = torch.as_tensor(lay.vec(c1, c2), device="cuda").reshape(1, -1)
out = g.sigma_sharded(c, rank, world).cpu().numpy()[0]
whole = g.sigma(c).cpu().numpy()[0]
s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
ref = lay.vec(s1, s2)
scale = float(np.abs(ref).max())
print(json.dumps({{"rank": rank, "vs_whole": float(np.abs(out - whole).max()) / scale,
                  "vs_oracle": float(np.abs(out - ref).max()) / scale, "range": mlcc.shard_range(g.n_chol, rank, world)}}))
g.close(); ctx.close()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_on_one_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    src = WORKER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), port=_free_port())
    procs = [subprocess.Popen([sys.executable, "-c", src, str(r), "2"], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    res = []
    for p in procs:
        so, se = p.communicate(timeout=600)
        assert p.returncode == 0, se[-3000:]
        res.append(json.loads(so.strip().splitlines()[-1]))
    res.sort(key=lambda d: d["rank"])
    assert res[0]["range"] == [0, 100] and res[1]["range"] == [100, 200]
    for d in res:
        assert d["vs_whole"] < 1e-10 and d["vs_oracle"] < 1e-10, d

"""Left eigenvectors on the GPU (mlcc_sigma_left, mlcc_excited_states_left) against the
oracle (oracle/left.py):

  * rho = A^T l element by element against the oracle's dense adjoint on the 7-orbital
    system's partitions without a CCSD level (binary64 and MLCC_FP64E, 1e-10 relative);
  * on a 48-orbital MLCC2 system and a ragged 37-orbital MLCC2 system with CCS outer
    orbitals (too large for a dense Jacobian): the adjoint identity <rho(l), c> = <l, A c>
    with A c from the oracle's sigma, for random symmetric l and c;
  * the left Davidson solve gives the right solve's roots (1e-8 Ha), left vectors with
    |A^T l - w l| small, and with the right vectors passed in, <l_k, r_m> = delta_km;
  * a system with a CCSD level is refused (MLCC_E_ARG).
"""
from dataclasses import replace

import numpy as np
import pytest

from gpu_helpers import Layout
from oracle import left as oleft
from oracle.mlcc import MLCCSystem, sigma, solve_ground_state
from test_gpu_parity import PARTITIONS
from tiny_systems import tiny

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2006_05226_gb300 import mlcc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mlcc.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _prepared(ctx, L, F, no, lev):
    from paper_2006_05226_gb300 import mlcc
    o = MLCCSystem(L, F, no, lev)
    gs = solve_ground_state(o)
    g = mlcc.System(ctx, _dev(L), _dev(F), no, lev)
    lay = Layout(g, o)
    g.jacobian_prepare(_dev(lay.t1(gs.t1)), _dev(lay.x2(gs.x2).ravel()))
    return g, o, gs, lay


def _rand(o, rng):
    c1 = rng.standard_normal((o.nv, o.no))
    c2 = rng.standard_normal(o.doubles_shape())
    return c1, c2 + c2.transpose(2, 3, 0, 1)


@pytest.mark.parametrize("name", ["cc2", "mlcc2_ccs_outer"])
@pytest.mark.parametrize("precision", [0, 4])
def test_left_transformation_against_the_dense_adjoint(ctx, name, precision):
    t = tiny()
    lev = np.array(dict(PARTITIONS)[name], dtype=np.int8)
    g, o, gs, lay = _prepared(ctx, t.L, t.F, t.k, lev)
    parts = oleft.dense(o, gs)
    rng = np.random.default_rng(4)
    ls, refs = [], []
    for _ in range(3):
        l1, l2 = _rand(o, rng)
        r1, r2 = oleft.left_transform(o, gs, l1, l2, parts)
        ls.append(lay.vec(l1, l2))
        refs.append(lay.vec(r1, r2))
    out = g.sigma_left(_dev(np.stack(ls)), precision=precision).cpu().numpy()
    ref = np.stack(refs)
    assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max()
    g.close()


def _mlcc2_systems():
    from synth import CONFIGS, make_system
    from synth.generator import SystemSpec, default_scale
    small = make_system(replace(CONFIGS["small"], name="small_mlcc2", t_occ=0, t_vir=0))
    ragged = make_system(SystemSpec("ragged_mlcc2", 6, 31, 29, 5.8, 5, 21, 0, 0, 3, 4, default_scale(5.8)))
    return {"small_mlcc2": small, "ragged_mlcc2": ragged}


@pytest.fixture(scope="module")
def mlcc2():
    return _mlcc2_systems()


@pytest.mark.parametrize("case", ["small_mlcc2", "ragged_mlcc2"])
def test_adjoint_identity(ctx, mlcc2, case):
    s = mlcc2[case]
    g, o, gs, lay = _prepared(ctx, s.L, s.fock, s.spec.n_occ, s.level)
    rng = np.random.default_rng(7)
    l1, l2 = _rand(o, rng)
    lv = lay.vec(l1, l2)
    for prec in (0, 4):
        rho = g.sigma_left(_dev(lv), precision=prec).cpu().numpy()[0]
        for _ in range(3):
            c1, c2 = _rand(o, rng)
            s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
            lhs = float(rho @ lay.vec(c1, c2))
            rhs = float(lv @ lay.vec(s1, s2))
            assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs)), (prec, lhs, rhs)
    g.close()


@pytest.mark.parametrize("case", ["small_mlcc2", "ragged_mlcc2"])
def test_left_eigenpairs(ctx, mlcc2, case):
    from paper_2006_05226_gb300 import mlcc
    s = mlcc2[case]
    g, o, gs, lay = _prepared(ctx, s.L, s.fock, s.spec.n_occ, s.level)
    opts = mlcc.default_options(n_roots=3)
    w, R, _ = g.excited_states(opts)
    wl, Lv, info = g.excited_states_left(opts, right=R)
    assert info.converged and np.abs(wl - w).max() < 1e-8
    Lh, Rh = Lv.cpu().numpy(), R.cpu().numpy()
    ov = Lh @ Rh.T
    assert np.abs(ov - np.eye(3)).max() < 1e-6
    res = g.sigma_left(Lv).cpu().numpy() - wl[:, None] * Lh
    assert np.abs(res).max() < 1e-6 * np.abs(Lh).max()
    g.close()


def test_a_ccsd_level_is_refused(ctx):
    from paper_2006_05226_gb300 import mlcc
    t = tiny()
    lev = np.array(dict(PARTITIONS)["three_level"], dtype=np.int8)
    g, o, gs, lay = _prepared(ctx, t.L, t.F, t.k, lev)
    with pytest.raises(mlcc.MLCCError) as e:
        g.sigma_left(torch.zeros(1, g.dims.vector_len, dtype=torch.float64, device="cuda"))
    assert e.value.status == mlcc.MLCC_E_ARG
    g.close()

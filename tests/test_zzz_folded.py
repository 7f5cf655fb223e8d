"""The folded CC2 Jacobian on the GPU (mlcc_sigma_eff, mlcc_fold_window) against the
oracle's sigma_eff / sigma_eff_domega (oracle/folded.py, pinned to the dense fold of the
Jacobian), element by element at the oracle's ground state, for several omega below the
lowest P_S denominator: singles and P_T rows of A_eff(omega) c, zero P_S rows, and the
singles of dA_eff/domega c. Also the window itself (min eps_aibj over P_S) and the
argument checks; and the folded eigensolver (mlcc_excited_states_folded) against the
oracle's unfolded Davidson roots and, through the oracle's sigma, its unfolded vectors.
Collected after the other GPU tests, so that a failure here cannot hide their results.
"""
import numpy as np
import pytest

from oracle.folded import sigma_eff, sigma_eff_domega
from oracle.mlcc import solve_ground_state
from test_gpu_parity import PARTITIONS, _close, _dev, _host, _make
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


def _inputs(case):
    if case.startswith("tiny:"):
        t = tiny()
        return t.L, t.F, t.k, np.array(dict(PARTITIONS)[case[5:]], dtype=np.int8)
    from synth import CONFIGS, make_system
    from synth.generator import SystemSpec, default_scale
    if case == "small":
        s = make_system(CONFIGS["small"])
    else:
        s = make_system(SystemSpec("ragged", 6, 31, 29, 5.8, 5, 21, 2, 7, 3, 4, default_scale(5.8)))
    return s.L, s.fock, s.spec.n_occ, s.level


@pytest.mark.parametrize("case", ["tiny:three_level", "tiny:mlcc2_ccs_outer", "small", "ragged"])
@pytest.mark.parametrize("precision", [0, 4])
def test_sigma_eff_matches_the_oracle(ctx, case, precision):
    L, F, no, lev = _inputs(case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    g.jacobian_prepare(_dev(lay.t1(gs.t1)), _dev(lay.x2(gs.x2)))
    top = g.fold_window()
    want_top = float(o.eps_aibj[o.mask_S].min()) if o.mask_S.any() else 1e300
    assert abs(top - want_top) <= 1e-12 * max(1.0, abs(want_top))
    rng = np.random.default_rng(11)
    cs, omegas, refs, drefs = [], [], [], []
    for frac in (0.0, 0.4, 0.8):
        c1 = rng.standard_normal((o.nv, o.no))
        c2 = rng.standard_normal(o.doubles_shape())
        c2 = c2 + c2.transpose(2, 3, 0, 1)
        w = frac * min(top, 1.0)
        s1, s2 = sigma_eff(o, gs, c1, c2, w)
        d1 = sigma_eff_domega(o, gs, c1, w)
        cs.append(lay.vec(c1, c2))
        omegas.append(w)
        refs.append(lay.vec(s1, s2))
        drefs.append(lay.t1(d1).ravel())
    out, dout = g.sigma_eff(_dev(np.stack(cs)), omegas, precision=precision, derivative=True)
    out, dout = _host(out), _host(dout)
    for k in range(len(cs)):
        _close(out[k], refs[k])
        _close(dout[k], drefs[k])


def test_sigma_eff_argument_checks(ctx):
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = _inputs("tiny:three_level")
    g, o, lay = _make(ctx, L, F, no, lev)
    c = _dev(np.zeros((1, g.dims.vector_len)))
    with pytest.raises(mlcc.MLCCError) as e:
        g.sigma_eff(c, [0.1])                   # before the Jacobian is prepared
    assert e.value.status == mlcc.MLCC_E_STATE
    gs = solve_ground_state(o)
    g.jacobian_prepare(_dev(lay.t1(gs.t1)), _dev(lay.x2(gs.x2)))
    top = g.fold_window()
    with pytest.raises(mlcc.MLCCError) as e:
        g.sigma_eff(c, [top])                   # on the lowest pole
    assert e.value.status == mlcc.MLCC_E_ARG
    assert float(_host(g.sigma_eff(c, [0.5 * top])).max()) == 0.0   # linear: zero in, zero out


@pytest.mark.parametrize("case", ["small", "tiny:three_level"])
def test_folded_eigensolver(ctx, case):
    from oracle.davidson import excited_states
    from oracle.folded import excited_states_folded
    from oracle.mlcc import sigma
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = _inputs(case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    g.jacobian_prepare(_dev(lay.t1(gs.t1)), _dev(lay.x2(gs.x2)))
    if case == "small":
        want = excited_states(o, gs, 3, res_tol=1e-9).omega
    else:
        want = excited_states_folded(o, gs, 3)
        if want.size < 3:
            pytest.skip("fewer than three roots below the lowest P_S denominator")
    w, R, info = g.excited_states_folded(mlcc.default_options(n_roots=3, es_res_tol=1e-9))
    assert info.converged and info.n_sigma > 0
    assert np.abs(w - want).max() < 1e-8
    R = _host(R)
    n1 = o.nv * o.no
    for k in range(3):
        assert abs(np.linalg.norm(R[k]) - 1.0) < 1e-12
        c1 = lay.t1_back(R[k][:n1], (o.nv, o.no))
        c2 = lay.x2_back(R[k][n1:], o.doubles_shape())
        s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
        res = np.sqrt(np.sum((s1 - w[k] * c1) ** 2) + np.sum((s2 - w[k] * c2) ** 2))
        assert res < 1e-6

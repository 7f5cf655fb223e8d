"""Parity of libmlcc (through the C ABI) with the FP64 oracle, element by element.

Tolerances (binary64 path): residuals, dressed vectors, Fock matrices and sigma agree to
1e-10 relative to the largest element (the two sides sum in different orders; the
arithmetic is otherwise identical); energies and excitation energies to 1e-8 Ha.
"""
import numpy as np
import pytest

from gpu_helpers import Layout
from oracle.davidson import excited_states as oracle_es
from oracle.mlcc import (MLCCSystem, energy, fock_t1, omega, sigma, solve_ground_state,
                         t1_transform)
from tiny_systems import tiny

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-10
E_TOL = 1e-8

PARTITIONS = [
    ("ccsd", [2, 2, 2, 2, 2, 2, 2]),
    ("cc2", [1, 1, 1, 1, 1, 1, 1]),
    ("mlcc2_ccs_outer", [1, 1, 1, 1, 1, 1, 0]),
    ("ccs_ccsd", [0, 2, 2, 2, 2, 0, 0]),
    ("three_level", [1, 2, 2, 2, 1, 1, 0]),
    ("three_level_inactive_occ", [0, 2, 2, 2, 1, 0, 0]),
    ("ccs_only", [0, 0, 0, 0, 0, 0, 0]),
]


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


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _close(a, b, rel=REL):
    scale = max(1.0, float(np.abs(b).max()) if b.size else 1.0)
    err = float(np.abs(a - b).max()) if b.size else 0.0
    assert err <= rel * scale, f"max error {err:.3e} > {rel:.1e} * {scale:.3e}"


def _make(ctx, L, F, no, level):
    from paper_2006_05226_gb300 import mlcc
    gsys = mlcc.System(ctx, _dev(L), _dev(F), no, level)
    osys = MLCCSystem(L, F, no, np.asarray(level, dtype=np.int8))
    return gsys, osys, Layout(gsys, osys)


def _random_amps(osys, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    t1 = scale * rng.standard_normal((osys.nv, osys.no))
    x2 = scale * rng.standard_normal(osys.doubles_shape())
    return t1, x2 + x2.transpose(2, 3, 0, 1)


@pytest.fixture(scope="module")
def sys7():
    return tiny()


@pytest.fixture(scope="module")
def small():
    from synth import CONFIGS, make_system
    return make_system(CONFIGS["small"])


@pytest.fixture(scope="module")
def ragged():
    # odd sizes: 37 orbitals, 6 occupied, 29 Cholesky vectors; CC2 5 / 21, CCSD 2 / 7
    from synth.generator import SystemSpec, default_scale, make_system
    spec = SystemSpec("ragged", 6, 31, 29, 5.8, 5, 21, 2, 7, 3, 4, default_scale(5.8))
    return make_system(spec)


def _systems(request, name):
    if name.startswith("tiny:"):
        t = request.getfixturevalue("sys7")
        lev = dict(PARTITIONS)[name[5:]]
        return t.L, t.F, t.k, np.array(lev, dtype=np.int8)
    s = request.getfixturevalue(name)
    return s.L, s.fock, s.spec.n_occ, s.level


CASES = [f"tiny:{p[0]}" for p in PARTITIONS] + ["small", "ragged"]


@pytest.mark.parametrize("case", ["small", "ragged", "tiny:three_level"])
def test_dressing_and_fock(ctx, request, case):
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    t1, _ = _random_amps(o, 1)
    Lt = _host(g.t1_transform(_dev(lay.t1(t1))))
    _close(Lt, lay.mo(t1_transform(o.L, t1, no)))
    Ft = _host(g.fock_t1(_dev(lay.t1(t1))))
    ref = fock_t1(t1_transform(o.h, t1, no), t1_transform(o.L, t1, no), no)
    _close(Ft, lay.mo(ref))


@pytest.mark.parametrize("case", CASES)
def test_omega_and_energy(ctx, request, case):
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    for seed in (2, 3):
        t1, x2 = _random_amps(o, seed)
        om1, om2, e = g.omega(_dev(lay.t1(t1)), _dev(lay.x2(x2)))
        r1, r2 = omega(o, t1, x2)
        _close(_host(om1).reshape(o.nv, o.no), lay.t1(r1))
        _close(_host(om2), lay.x2(r2).ravel())
        assert abs(float(_host(e)[0]) - energy(o, t1, x2)) < 1e-10


@pytest.mark.parametrize("case", CASES)
def test_ground_state(ctx, request, case):
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    assert gs.converged
    t1, x2, info = g.ground_state()
    assert info.converged
    assert abs(info.e_corr - gs.energy) < E_TOL
    _close(_host(t1).reshape(o.nv, o.no), lay.t1(gs.t1), rel=1e-7)
    if o.so and o.sv:
        _close(_host(x2), lay.x2(gs.x2).ravel(), rel=1e-7)


@pytest.mark.parametrize("case", CASES)
def test_sigma(ctx, request, case):
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    g.jacobian_prepare(_dev(lay.t1(gs.t1)), _dev(lay.x2(gs.x2)))
    rng = np.random.default_rng(4)
    cs, refs = [], []
    for _ in range(2):
        c1 = rng.standard_normal((o.nv, o.no))
        c2 = rng.standard_normal(o.doubles_shape())
        c2 = c2 + c2.transpose(2, 3, 0, 1)
        cs.append(lay.vec(c1, c2))
        s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
        refs.append(lay.vec(s1, s2))
    out = _host(g.sigma(_dev(np.stack(cs))))
    for k in range(2):
        _close(out[k], refs[k])


@pytest.mark.parametrize("case", ["small", "ragged", "tiny:three_level", "tiny:ccsd", "tiny:ccs_only"])
def test_excited_states(ctx, request, case):
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    ref = oracle_es(o, gs, 3, res_tol=1e-9)
    assert ref.converged
    g.ground_state()
    w, R, info = g.excited_states(mlcc.default_options(n_roots=3))
    assert info.converged and not info.complex_pair
    assert np.abs(w - ref.omega).max() < E_TOL
    # the returned vectors are eigenvectors of the oracle Jacobian
    Rh = _host(R)
    n1 = o.nv * o.no
    for k in range(3):
        c1 = lay.t1_back(Rh[k, :n1], (o.nv, o.no))
        c2 = lay.x2_back(Rh[k, n1:], o.doubles_shape())
        s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
        res = np.sqrt(np.sum((s1 - w[k] * c1) ** 2) + np.sum((s2 - w[k] * c2) ** 2))
        assert res < 1e-6


def test_solve_from_host_memory(ctx, small):
    from paper_2006_05226_gb300 import mlcc
    o = MLCCSystem(small.L, small.fock, small.spec.n_occ, small.level)
    gs = solve_ground_state(o)
    ref = oracle_es(o, gs, 3, res_tol=1e-9)
    sol = mlcc.solve(ctx, small.L, small.fock, small.spec.n_occ, small.level,
                     mlcc.default_options(n_roots=3))
    assert abs(sol.gs.e_corr - gs.energy) < E_TOL
    assert np.abs(sol.omega - ref.omega).max() < E_TOL


def test_invalid_inputs_are_rejected(ctx, sys7):
    from paper_2006_05226_gb300 import mlcc
    L, F = sys7.L.copy(), sys7.F.copy()
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.System(ctx, _dev(L), _dev(F), 2, np.array([1, 1, 3, 1, 1, 1, 1], np.int8))
    assert e.value.status == -1
    Lb = L.copy()
    Lb[0, 1, 2] += 1e-3
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.System(ctx, _dev(Lb), _dev(F), 2, np.ones(7, np.int8))
    assert e.value.status == -1
    Fb = F.copy()
    Fb[3, 4] += 1e-3                                # not symmetric
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.System(ctx, _dev(L), _dev(Fb), 2, np.ones(7, np.int8))
    assert e.value.status == -1
    Fb = F.copy()
    Fb[3, 3] = np.nan
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.System(ctx, _dev(L), _dev(Fb), 2, np.ones(7, np.int8))
    assert e.value.status == mlcc.MLCC_E_NAN
    g = mlcc.System(ctx, _dev(L), _dev(F), 2, np.ones(7, np.int8))
    with pytest.raises(mlcc.MLCCError) as e:
        g.sigma(torch.zeros(1, g.dims.vector_len, dtype=torch.float64, device="cuda"))
    assert e.value.status == -9


# mixed precision: bound of max|sigma_lowp - sigma_fp64| / max|sigma_fp64|
LOWP = [(1, 3e-2), (2, 1e-3), (3, 1e-4)]


@pytest.mark.parametrize("case", ["small", "ragged", "tiny:three_level"])
@pytest.mark.parametrize("prec,tol", LOWP)
def test_sigma_low_precision(ctx, request, case, prec, tol):
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    g.jacobian_prepare(_dev(lay.t1(gs.t1)), _dev(lay.x2(gs.x2)))
    rng = np.random.default_rng(8)
    c = rng.standard_normal((2, g.dims.vector_len))
    ref = _host(g.sigma(_dev(c)))
    out = _host(g.sigma(_dev(c), precision=prec))
    rel = np.abs(out - ref).max() / np.abs(ref).max()
    print(f"precision {prec}: max relative sigma error {rel:.3e}")
    assert rel < tol


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_davidson_refined_to_fp64(ctx, small, prec):
    """Low-precision Davidson followed by binary64 refinement reaches the oracle roots."""
    from paper_2006_05226_gb300 import mlcc
    o = MLCCSystem(small.L, small.fock, small.spec.n_occ, small.level)
    gs = solve_ground_state(o)
    ref = oracle_es(o, gs, 3, res_tol=1e-9)
    g, _, _ = _make(ctx, small.L, small.fock, small.spec.n_occ, small.level)
    g.ground_state()
    w, _, info = g.excited_states(mlcc.default_options(n_roots=3, precision=prec, refine_fp64=1000,
                                                       lowp_res_tol=1e-3), want_vectors=False)
    assert info.converged and info.n_sigma_lowp > 0
    assert np.abs(w - ref.omega).max() < E_TOL
    # one binary64 Rayleigh-Ritz sweep on the low-precision Ritz vectors: within 1e-6 Ha
    # from split-bf16 vectors; plain bf16 (sigma noise near 1e-4) stops a little short
    w1, _, info1 = g.excited_states(mlcc.default_options(n_roots=3, precision=prec, refine_fp64=1,
                                                         lowp_res_tol=1e-4 if prec > 1 else 1e-3),
                                    want_vectors=False)
    assert info1.converged and info1.fp64_sweeps == 1
    assert np.abs(w1 - ref.omega).max() < (5e-6 if prec == 1 else 1e-6)


@pytest.mark.parametrize("case", ["small", "tiny:three_level"])
def test_mixed_ground_state(ctx, request, case):
    """Ground state iterated with tensor-core contractions (split bfloat16), then polished
    in binary64: the oracle energy to 1e-8 Ha; without the polish to 1e-6 Ha."""
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = _systems(request, case)
    g, o, lay = _make(ctx, L, F, no, lev)
    gs = solve_ground_state(o)
    for refine, tol in ((1, E_TOL), (0, 1e-6)):
        opts = mlcc.default_options(gs_precision=mlcc.MLCC_BF16X6, refine_fp64=refine)
        t1, x2, info = g.ground_state(opts)
        assert info.converged
        assert abs(info.e_corr - gs.energy) < tol

"""The whole-solve boundary (mlcc_solve / mlcc_solve_device, mlcc_result) through the C ABI:

  * semicanonicalisation (Sec. 2.1-2.2): inputs rotated by random orthogonal matrices inside
    each level's occupied and virtual blocks (F no longer diagonal there) give the energies
    and excitation energies of the canonical input, which match the oracle's; the returned
    orbitals undo the rotation, and the amplitudes agree up to the orbital signs;
  * every output of mlcc_result: per-root residual norms, the converged singles and doubles
    (equal to mlcc_ground_state's), the right eigenvectors (eigenvectors of the oracle's
    Jacobian), from host and from device memory alike;
  * the device-memory budget of a context: a system or solve above it is refused with
    MLCC_E_OOM before anything is allocated.
"""
import numpy as np
import pytest

from oracle.davidson import excited_states as oracle_es
from oracle.mlcc import MLCCSystem, sigma, solve_ground_state
from gpu_helpers import Layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
E_TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    from paper_2006_05226_gb300 import mlcc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mlcc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def three_level():
    """A 40-orbital system with all three levels and a ragged shape: 7 occupied / 33 virtual,
    CCSD 2/6 inside CC2 5/20, CCS rest."""
    from synth.generator import SystemSpec, default_scale, make_system
    return make_system(SystemSpec("boundary", 7, 33, 90, 18.0, 5, 20, 2, 6, 3, 5, default_scale(18.0)))


def _level_blocks(no, level):
    """Caller-order index sets of each level's occupied and virtual orbitals."""
    lev = np.asarray(level)
    out = []
    for lo, hi in ((0, no), (no, lev.size)):
        for v in (0, 1, 2):
            idx = lo + np.nonzero(lev[lo:hi] == v)[0]
            if idx.size:
                out.append(idx)
    return out


def _rotation(no, level, seed):
    rng = np.random.default_rng(seed)
    n = len(level)
    U = np.eye(n)
    for idx in _level_blocks(no, level):
        if idx.size > 1:
            Q, _ = np.linalg.qr(rng.standard_normal((idx.size, idx.size)))
            U[np.ix_(idx, idx)] = Q
    return U


def test_semicanonicalisation_inside_the_library(ctx, three_level):
    from paper_2006_05226_gb300 import mlcc
    s = three_level
    no, lev = s.spec.n_occ, s.level
    U = _rotation(no, lev, 3)
    Fr = U.T @ s.fock @ U
    Lr = np.einsum("pk,Jpq,ql->Jkl", U, s.L, U, optimize=True)
    blocks = _level_blocks(no, lev)
    assert max(np.abs(Fr[np.ix_(b, b)] - np.diag(np.diag(Fr[np.ix_(b, b)]))).max() for b in blocks) > 1e-3
    opts = mlcc.default_options(n_roots=3)
    can = mlcc.solve(ctx, s.L, s.fock, no, lev, opts, t1=True, orbitals=True)
    rot = mlcc.solve(ctx, Lr, Fr, no, lev, opts, t1=True, orbitals=True)
    # the oracle on the canonical input
    o = MLCCSystem(s.L, s.fock, no, lev)
    gs = solve_ground_state(o)
    ref = oracle_es(o, gs, 3, res_tol=1e-9)
    assert abs(can.gs.e_corr - gs.energy) < E_TOL and np.abs(can.omega - ref.omega).max() < E_TOL
    assert abs(rot.gs.e_hf - can.gs.e_hf) < 1e-10
    assert abs(rot.gs.e_corr - can.gs.e_corr) < 1e-10
    assert np.abs(rot.omega - can.omega).max() < 1e-9
    # orbitals: canonical input -> a permutation; rotated input -> U^T of the same orbitals, signed
    n = len(lev)
    P = can.orbitals
    assert np.array_equal(np.abs(P), np.abs(P).round()) and np.allclose(P.T @ P, np.eye(n))
    C = rot.orbitals
    assert np.abs(C.T @ C - np.eye(n)).max() < 1e-12
    D = (U @ C).T @ P          # system orbitals of both solves: D = diag(+-1)
    assert np.abs(np.abs(D) - np.eye(n)).max() < 1e-9
    d = np.sign(np.diag(D))
    nv = n - no
    t_can = can.t1.reshape(nv, no)
    t_rot = rot.t1.reshape(nv, no)
    assert np.abs(t_rot - d[no:, None] * d[None, :no] * t_can).max() < 1e-9


def test_result_outputs(ctx, three_level):
    from paper_2006_05226_gb300 import mlcc
    s = three_level
    no, lev = s.spec.n_occ, s.level
    opts = mlcc.default_options(n_roots=3)
    h = mlcc.solve(ctx, s.L, s.fock, no, lev, opts, t1=True, x2=True, vectors=True, orbitals=True)
    d = mlcc.solve_device(ctx, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"),
                          no, lev, opts, t1=True, x2=True, vectors=True)
    torch.cuda.synchronize()
    assert h.es.converged and np.all(h.residual < opts.es_res_tol) and np.all(h.residual > 0)
    assert np.abs(h.residual.max() - h.es.max_residual) <= 1e-15
    for name in ("t1", "x2", "r"):
        assert np.array_equal(getattr(d, name).cpu().numpy(), getattr(h, name)), name
    assert np.array_equal(d.omega, h.omega) and np.array_equal(d.residual, h.residual)
    # the amplitudes are mlcc_ground_state's
    g = mlcc.System(ctx, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, lev)
    t1, x2, _ = g.ground_state(opts)
    assert np.array_equal(t1.cpu().numpy(), h.t1) and np.array_equal(x2.cpu().numpy(), h.x2)
    assert np.array_equal(g.perm, h.perm)
    # the vectors: unit norm, largest element positive, eigenvectors of the oracle Jacobian
    o = MLCCSystem(s.L, s.fock, no, lev)
    gs = solve_ground_state(o)
    lay = Layout(g, o)
    n1 = o.nv * o.no
    for k in range(3):
        r = h.r[k]
        assert abs(np.linalg.norm(r) - 1.0) < 1e-12 and r[np.argmax(np.abs(r))] > 0
        c1 = lay.t1_back(r[:n1], (o.nv, o.no))
        c2 = lay.x2_back(r[n1:], o.doubles_shape())
        s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
        res = np.sqrt(np.sum((s1 - h.omega[k] * c1) ** 2) + np.sum((s2 - h.omega[k] * c2) ** 2))
        assert res < 1e-7
    g.close()


def test_context_budget(ctx, three_level):
    from paper_2006_05226_gb300 import mlcc
    s = three_level
    no, lev = s.spec.n_occ, s.level
    opts = mlcc.default_options(n_roots=3)
    fp = mlcc.solve_footprint(len(lev), no, s.L.shape[0], lev, opts)
    small = mlcc.Context(0, budget_bytes=fp // 4)
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.solve(small, s.L, s.fock, no, lev, opts)
    assert e.value.status == mlcc.MLCC_E_OOM
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.System(small, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, lev)
    assert e.value.status == mlcc.MLCC_E_OOM
    small.close()
    roomy = mlcc.Context(0, budget_bytes=fp)
    sol = mlcc.solve(roomy, s.L, s.fock, no, lev, opts)
    ref = mlcc.solve(ctx, s.L, s.fock, no, lev, opts)
    assert np.array_equal(sol.omega, ref.omega)
    # a budget that holds one system refuses a second one at the same time
    g1 = mlcc.System(roomy, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, lev)
    ws = g1.dims.workspace_bytes
    tight = mlcc.Context(0, budget_bytes=int(1.5 * ws))
    a = mlcc.System(tight, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, lev)
    with pytest.raises(mlcc.MLCCError) as e:
        mlcc.System(tight, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, lev)
    assert e.value.status == mlcc.MLCC_E_OOM
    a.close()
    b = mlcc.System(tight, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, lev)
    b.close()
    g1.close()
    tight.close()
    roomy.close()
    assert free0 > 0

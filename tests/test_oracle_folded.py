"""Pins of the folded CC2 effective Jacobian (oracle/folded.py) to the dense Jacobian.

The fold rests on the block structure of the three-level model (A_SS = diag(eps_aibj),
A_ST = A_TS = 0), which is checked here on the dense A in the independent parameters
(singles, doubles (ai) <= (bj)) before anything is folded. Then, for every partition:
  * sigma_eff (two applications of sigma) equals A_11 + A_1S (omega - eps_S)^-1 A_S1 and
    the P_T blocks, built from the dense A, at several omega;
  * the folded roots below the lowest P_S denominator are exactly the eigenvalues of A
    in that window;
  * unfolding a folded eigenvector gives an eigenvector of A.
"""
import numpy as np
import pytest

from oracle.folded import excited_states_folded, folded_matrix, packed_T, sigma_eff, unfold
from oracle.mlcc import MLCCSystem, sigma, solve_ground_state
from test_oracle_pins import PARTITIONS, _dense_jacobian
from tiny_systems import tiny

FOLDABLE = [p for p in PARTITIONS if any(v >= 1 for v in p[1])]


@pytest.fixture(scope="module")
def sys7():
    return tiny()


def _setup(t, lev):
    osys = MLCCSystem(t.L, t.F, t.k, np.array(lev, dtype=np.int8))
    gs = solve_ground_state(osys)
    return osys, gs


def _blocks(osys, gs):
    """Dense A and the index sets of singles, P_S and P_T in its packed doubles."""
    A = _dense_jacobian(osys, gs)
    sh = osys.doubles_shape()
    n1 = osys.nv * osys.no
    pk = [(a, i, b, j) for a in range(sh[0]) for i in range(sh[1]) for b in range(sh[2])
          for j in range(sh[3]) if a * sh[1] + i <= b * sh[3] + j]
    isT = np.array([bool(osys.mask_T[p]) for p in pk], dtype=bool)
    one = np.arange(n1)
    S = n1 + np.nonzero(~isT)[0]
    T = n1 + np.nonzero(isT)[0]
    dS = np.array([osys.eps_aibj[p] for p, t in zip(pk, isT) if not t])
    return A, one, S, T, dS


@pytest.mark.parametrize("name,lev", FOLDABLE)
def test_block_structure_of_the_three_level_jacobian(sys7, name, lev):
    osys, gs = _setup(sys7, lev)
    A, one, S, T, dS = _blocks(osys, gs)
    scale = np.abs(A).max()
    if S.size:
        ASS = A[np.ix_(S, S)]
        assert np.abs(ASS - np.diag(dS)).max() < 1e-10 * scale
    if S.size and T.size:
        assert np.abs(A[np.ix_(S, T)]).max() < 1e-10 * scale
        assert np.abs(A[np.ix_(T, S)]).max() < 1e-10 * scale


@pytest.mark.parametrize("name,lev", FOLDABLE)
def test_sigma_eff_is_the_folded_jacobian(sys7, name, lev):
    osys, gs = _setup(sys7, lev)
    A, one, S, T, dS = _blocks(osys, gs)
    keep = np.concatenate([one, T])
    for omega in (0.0, 0.35, -0.2):
        ref = A[np.ix_(keep, keep)].copy()
        if S.size:
            ref[:one.size, :one.size] += A[np.ix_(one, S)] @ np.diag(1.0 / (omega - dS)) @ A[np.ix_(S, one)]
        M = folded_matrix(osys, gs, omega)
        assert M.shape == ref.shape
        assert np.abs(M - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("name,lev", FOLDABLE)
def test_folded_roots_are_jacobian_eigenvalues(sys7, name, lev):
    """Every eigenvalue of A in (0, min eps_S) is a folded root, and nothing else."""
    osys, gs = _setup(sys7, lev)
    A, one, S, T, dS = _blocks(osys, gs)
    w = np.linalg.eigvals(A)
    w = np.sort(w.real[np.abs(w.imag) < 1e-9])
    top = dS.min() if dS.size else np.inf
    want = w[(w > 0) & (w < top)][:3]
    assert want.size >= 1   # the window is not empty for these partitions
    roots = excited_states_folded(osys, gs, 3)
    assert roots.size == want.size
    assert np.abs(roots - want).max() < 1e-9


@pytest.mark.parametrize("name,lev", [("three_level", dict(PARTITIONS)["three_level"])])
def test_unfolded_eigenvector_is_an_eigenvector_of_A(sys7, name, lev):
    osys, gs = _setup(sys7, lev)
    w0 = excited_states_folded(osys, gs, 1)[0]
    assert 0.0 < w0 < osys.eps_aibj[osys.mask_S].min()
    M = folded_matrix(osys, gs, w0)
    ev, V = np.linalg.eig(M)
    k = int(np.argmin(np.abs(ev - w0)))
    v = V[:, k].real
    n1 = osys.nv * osys.no
    pk = packed_T(osys)
    c1 = v[:n1].reshape(osys.nv, osys.no)
    cT = np.zeros(osys.doubles_shape())
    for x, (a, i, b, j) in zip(v[n1:], pk):
        cT[a, i, b, j] = cT[b, j, a, i] = x
    c2 = unfold(osys, gs, c1, cT, w0)
    s1, s2 = sigma(osys, gs.t1, gs.x2, c1, c2)
    r = np.concatenate([(s1 - w0 * c1).ravel(), (s2 - w0 * c2).ravel()])
    assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(np.concatenate([c1.ravel(), c2.ravel()]))
    # and sigma_eff leaves (c1, c_T) with eigenvalue w0
    e1, e2 = sigma_eff(osys, gs, c1, cT, w0)
    assert np.abs(e1 - w0 * c1).max() < 1e-9 and np.abs(e2 - w0 * np.where(osys.mask_T, cT, 0)).max() < 1e-9


def test_iterative_folded_solver_on_the_48_orbital_workload():
    """The iterative solver (linear Davidson on A_eff(omega), fixed point in omega) gives the
    unfolded roots of the 48-orbital, three-level workload, whose P_S denominators (>= 0.96
    Ha) lie far above its roots."""
    from oracle.davidson import excited_states
    from oracle.folded import excited_states_folded_iterative
    from synth import CONFIGS, make_system
    s = make_system(CONFIGS["small"])
    osys = MLCCSystem(s.L, s.fock, s.spec.n_occ, s.level)
    gs = solve_ground_state(osys)
    ref = excited_states(osys, gs, 3, res_tol=1e-9)
    roots, n_eff = excited_states_folded_iterative(osys, gs, 3)
    assert np.abs(roots - ref.omega).max() < 1e-9
    assert osys.eps_aibj[osys.mask_S].min() > 2.5 * roots.max()


def test_linearised_folded_solver_on_the_48_orbital_workload():
    """The folded solver that keeps its subspaces across omega updates (first-order model
    in omega per trial vector) gives the unfolded roots, with fewer applications of A_eff
    than the plain fixed point in omega."""
    from oracle.davidson import excited_states
    from oracle.folded import excited_states_folded_iterative, excited_states_folded_linearised
    from synth import CONFIGS, make_system
    s = make_system(CONFIGS["small"])
    osys = MLCCSystem(s.L, s.fock, s.spec.n_occ, s.level)
    gs = solve_ground_state(osys)
    ref = excited_states(osys, gs, 3, res_tol=1e-9)
    roots, n_lin = excited_states_folded_linearised(osys, gs, 3)
    assert np.abs(roots - ref.omega).max() < 1e-9
    _, n_fixed = excited_states_folded_iterative(osys, gs, 3)
    assert n_lin < n_fixed


@pytest.mark.parametrize("name,lev", FOLDABLE)
def test_linearised_folded_solver_on_the_seven_orbital_partitions(sys7, name, lev):
    """Same roots as the determinant scan wherever the window holds three roots."""
    from oracle.folded import excited_states_folded_linearised
    osys, gs = _setup(sys7, lev)
    want = excited_states_folded(osys, gs, 3)
    if want.size < 3:
        pytest.skip("fewer than three roots below the lowest P_S denominator")
    roots, _ = excited_states_folded_linearised(osys, gs, 3)
    assert np.abs(roots - want).max() < 1e-9


@pytest.mark.parametrize("name,lev", FOLDABLE)
def test_sigma_eff_domega_is_the_omega_derivative(sys7, name, lev):
    """dA_eff/domega c from sigma_eff_domega equals the central difference of sigma_eff in
    omega (singles; the P_T rows do not depend on omega), and equals
    -A_1S diag((omega - eps_S)^-2) A_S1 c1 built from the dense Jacobian."""
    from oracle.folded import sigma_eff_domega
    osys, gs = _setup(sys7, lev)
    A, one, S, T, dS = _blocks(osys, gs)
    rng = np.random.default_rng(5)
    c1 = rng.standard_normal((osys.nv, osys.no))
    cT = rng.standard_normal(osys.doubles_shape())
    cT = cT + cT.transpose(2, 3, 0, 1)
    top = dS.min() if dS.size else 1.0
    for omega in (0.0, 0.3 * top, -0.2):
        d1 = sigma_eff_domega(osys, gs, c1, omega)
        h = 1e-4
        p1, p2 = sigma_eff(osys, gs, c1, cT, omega + h)
        m1, m2 = sigma_eff(osys, gs, c1, cT, omega - h)
        fd = (p1 - m1) / (2 * h)
        assert np.abs(d1 - fd).max() < 1e-6 * max(1.0, np.abs(d1).max())
        assert np.abs(p2 - m2).max() < 1e-12
        if S.size:
            ref = -A[np.ix_(one, S)] @ (((omega - dS) ** -2) * (A[np.ix_(S, one)] @ c1.ravel()))
            assert np.abs(d1.ravel() - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())

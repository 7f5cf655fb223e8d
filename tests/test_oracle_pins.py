"""Pins of the FP64 oracle to things other than itself (no GPU).

* brute-force determinant-space CC (tests/brute_force.py): residual, energy, Jacobian;
* FCI for two-electron systems, where CCSD is exact;
* the CIS closed form (all orbitals at the CCS level) and the MP2 closed form;
* the limits and invariances the paper states (Sec. 2.1).
"""
import numpy as np
import pytest

from brute_force import BruteForceCC
from oracle.davidson import excited_states
from oracle.mlcc import (MLCCSystem, energy, hf_energy, omega, sigma, sigma_mlcc2_paper,
                         solve_ground_state, t1_transform)
from tiny_systems import rotate, tiny

# (name, per-MO level) for the 7-orbital, 2-occupied test system; 2 = CCSD, 1 = CC2, 0 = CCS
PARTITIONS = [
    ("ccsd", [2, 2, 2, 2, 2, 2, 2]),
    ("cc2", [1, 1, 1, 1, 1, 1, 1]),
    ("mlcc2_ccs_outer", [1, 1, 1, 1, 1, 1, 0]),
    ("ccs_ccsd", [0, 2, 2, 2, 2, 0, 0]),
    ("three_level", [1, 2, 2, 2, 1, 1, 0]),
    ("three_level_inactive_occ", [0, 2, 2, 2, 1, 0, 0]),
]


@pytest.fixture(scope="module")
def sys7():
    return tiny()


def _systems(t, lev):
    lev = np.array(lev, dtype=np.int8)
    return MLCCSystem(t.L, t.F, t.k, lev), BruteForceCC(t.h, t.L, t.F, t.k, lev)


def _random_amplitudes(osys, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    t1 = scale * rng.standard_normal((osys.nv, osys.no))
    x2 = scale * rng.standard_normal(osys.doubles_shape())
    return t1, x2 + x2.transpose(2, 3, 0, 1)


def test_reference_energy_and_h(sys7):
    osys, bf = _systems(sys7, PARTITIONS[0][1])
    # Eq. eff_fock inverted: the recovered one-electron matrix is the MO core Hamiltonian
    assert np.abs(osys.h - sys7.h).max() < 1e-10
    assert abs(bf.e_hf - sys7.e_hf) < 1e-10
    assert abs(hf_energy(osys) - sys7.e_hf) < 1e-10


@pytest.mark.parametrize("name,lev", PARTITIONS)
def test_omega_and_energy_match_determinant_cc(sys7, name, lev):
    """Omega and E at random amplitudes, element by element, against Sec. 2.1 evaluated
    literally in the determinant space."""
    osys, bf = _systems(sys7, lev)
    for seed in (1, 2):
        t1, x2 = _random_amplitudes(osys, seed)
        o1, o2 = omega(osys, t1, x2)
        b1, b2, be = bf.residual(t1, x2)
        assert np.abs(o1 - b1).max() < 1e-9 * max(1.0, np.abs(b1).max())
        assert np.abs(o2 - b2).max() < 1e-9 * max(1.0, np.abs(b2).max())
        assert abs(energy(osys, t1, x2) - be) < 1e-9


@pytest.mark.parametrize("name,lev", PARTITIONS)
def test_ground_state_and_jacobian_match_determinant_cc(sys7, name, lev):
    osys, bf = _systems(sys7, lev)
    gs = solve_ground_state(osys)
    assert gs.converged
    b1, b2, be = bf.residual(gs.t1, gs.x2)
    assert np.abs(b1).max() < 1e-9 and np.abs(b2).max() < 1e-9
    assert abs(gs.energy - be) < 1e-9
    # sigma = dOmega/dx along c, against a central difference of the determinant residual
    rng = np.random.default_rng(7)
    c1 = rng.standard_normal(gs.t1.shape)
    c2 = rng.standard_normal(gs.x2.shape)
    c2 = c2 + c2.transpose(2, 3, 0, 1)
    s1, s2 = sigma(osys, gs.t1, gs.x2, c1, c2)
    h = 1e-4
    p1, p2, _ = bf.residual(gs.t1 + h * c1, gs.x2 + h * c2)
    m1, m2, _ = bf.residual(gs.t1 - h * c1, gs.x2 - h * c2)
    assert np.abs(s1 - (p1 - m1) / (2 * h)).max() < 1e-6
    assert np.abs(s2 - (p2 - m2) / (2 * h)).max() < 1e-6


@pytest.mark.parametrize("name,lev", [p for p in PARTITIONS if 2 not in p[1]])
def test_paper_mlcc2_sigma_is_the_jacobian(sys7, name, lev):
    """Appendix A Eq. mlcc_A_ (with its two readings) equals dOmega/dx exactly."""
    osys, _ = _systems(sys7, lev)
    gs = solve_ground_state(osys)
    rng = np.random.default_rng(3)
    for _ in range(2):
        c1 = rng.standard_normal(gs.t1.shape)
        c2 = rng.standard_normal(gs.x2.shape)
        c2 = c2 + c2.transpose(2, 3, 0, 1)
        s1, s2 = sigma(osys, gs.t1, gs.x2, c1, c2)
        q1, q2 = sigma_mlcc2_paper(osys, gs.t1, gs.x2, c1, c2)
        assert np.abs(s1 - q1).max() < 1e-12 * max(1, np.abs(s1).max())
        assert np.abs(s2 - q2).max() < 1e-12 * max(1, np.abs(s2).max())


def _dense_jacobian(osys, gs):
    """A in the independent parameters (singles, doubles ai <= bj), column by column."""
    nv, no = osys.nv, osys.no
    sh = osys.doubles_shape()
    n1 = nv * no
    pk = [(a, i, b, j) for a in range(sh[0]) for i in range(sh[1]) for b in range(sh[2])
          for j in range(sh[3]) if a * sh[1] + i <= b * sh[3] + j]
    cols = []
    for m in range(n1):
        e1 = np.zeros(n1)
        e1[m] = 1.0
        s1, s2 = sigma(osys, gs.t1, gs.x2, e1.reshape(nv, no), np.zeros(sh))
        cols.append(np.concatenate([s1.ravel(), [s2[p] for p in pk]]))
    for (a, i, b, j) in pk:
        e2 = np.zeros(sh)
        e2[a, i, b, j] = e2[b, j, a, i] = 1.0
        s1, s2 = sigma(osys, gs.t1, gs.x2, np.zeros((nv, no)), e2)
        cols.append(np.concatenate([s1.ravel(), [s2[p] for p in pk]]))
    return np.array(cols).T


@pytest.mark.parametrize("name,lev", PARTITIONS)
def test_davidson_matches_dense_eigenvalues(sys7, name, lev):
    osys, _ = _systems(sys7, lev)
    gs = solve_ground_state(osys)
    w = np.linalg.eigvals(_dense_jacobian(osys, gs))
    w = np.sort(w.real[np.abs(w.imag) < 1e-9])
    es = excited_states(osys, gs, 3, res_tol=1e-9)
    assert es.converged and not es.complex_pair
    assert np.abs(es.omega - w[:3]).max() < 1e-9


def test_two_electron_ccsd_is_fci():
    """Two electrons: CCSD is exact (Sec. 2.1 limit), so E and the singlet excitation
    energies equal the FCI ones."""
    t = tiny(n=6, k=1, n_chol=10, tau=5.0, seed=5, scale=0.4)
    lev = np.full(6, 2, dtype=np.int8)
    osys, bf = _systems(t, lev)
    gs = solve_ground_state(osys)
    fci = bf.singlet_fci(5)
    assert abs((bf.e_hf + gs.energy) - fci[0]) < 1e-10
    es = excited_states(osys, gs, 3, res_tol=1e-10)
    assert np.abs(es.omega - (fci[1:4] - fci[0])).max() < 1e-9


def test_singlet_count_two_electrons():
    t = tiny(n=5, k=1, n_chol=6, tau=4.0, seed=2, scale=0.4)
    bf = BruteForceCC(t.h, t.L, t.F, 1, np.full(5, 2, dtype=np.int8))
    w, v = bf.fci()
    S2 = bf.s_squared()
    s2 = np.array([v[:, k] @ (S2 @ v[:, k]) for k in range(len(w))])
    assert np.sum(np.abs(s2) < 1e-8) == 15 and np.sum(np.abs(s2 - 2) < 1e-8) == 10


def test_cis_limit(sys7):
    """All orbitals at the CCS level: t1 = 0 (Brillouin) and A is the singlet CIS matrix
    (eps_a - eps_i) d + 2 g_aijb - g_abji, the CCS sigma of Appendix A at t1 = 0."""
    lev = np.zeros(7, dtype=np.int8)
    osys = MLCCSystem(sys7.L, sys7.F, sys7.k, lev)
    gs = solve_ground_state(osys)
    assert np.abs(gs.t1).max() < 1e-10 and abs(gs.energy) < 1e-12
    no = sys7.k
    g = np.einsum("Kpq,Krs->pqrs", sys7.L, sys7.L)
    nv = 7 - no
    A = np.zeros((nv, no, nv, no))
    e = np.diag(sys7.F)
    for a in range(nv):
        for i in range(no):
            for b in range(nv):
                for j in range(no):
                    A[a, i, b, j] = ((e[no + a] - e[i]) * (a == b) * (i == j)
                                     + 2 * g[no + a, i, j, no + b] - g[no + a, no + b, j, i])
    w = np.linalg.eigvalsh(A.reshape(nv * no, nv * no))
    es = excited_states(osys, gs, 3, res_tol=1e-10)
    assert np.abs(es.omega - w[:3]).max() < 1e-10


def test_mp2_first_iteration(sys7):
    """At t1 = 0 the CC2 amplitudes are first-order and E is the MP2 energy of the active
    pairs: -sum g_aibj (2 g_aibj - g_ajbi) / eps_aibj."""
    lev = np.array([1, 1, 1, 1, 1, 1, 0], dtype=np.int8)
    osys = MLCCSystem(sys7.L, sys7.F, sys7.k, lev)
    gs = solve_ground_state(osys, max_iter=1)
    e_it1 = gs.history[0][0]
    no = sys7.k
    V = no + osys.vs
    g = np.einsum("Kai,Kbj->aibj", sys7.L[:, V][:, :, osys.os], sys7.L[:, V][:, :, osys.os])
    e = np.diag(sys7.F)
    ea = e[V][:, None] - e[osys.os][None, :]
    den = ea[:, :, None, None] + ea[None, None]
    emp2 = -np.sum(g * (2 * g - g.transpose(0, 3, 2, 1)) / den)
    assert abs(e_it1 - emp2) < 1e-12


def test_ccsd_invariant_under_occupied_and_virtual_rotations(sys7):
    """Full CCSD energy and excitation energies do not depend on rotations within the
    occupied and within the virtual space (this exercises the off-diagonal F~ terms)."""
    lev = np.full(7, 2, dtype=np.int8)
    o0 = MLCCSystem(sys7.L, sys7.F, sys7.k, lev)
    g0 = solve_ground_state(o0)
    L, F, _ = rotate(sys7)
    o1 = MLCCSystem(L, F, sys7.k, lev)
    g1 = solve_ground_state(o1, max_iter=400)
    assert g0.converged and g1.converged
    assert abs(g0.energy - g1.energy) < 1e-10
    e0 = excited_states(o0, g0, 3, res_tol=1e-9)
    e1 = excited_states(o1, g1, 3, res_tol=1e-9)
    assert np.abs(e0.omega - e1.omega).max() < 1e-8


def test_dressing_leaves_ov_block_and_integral_symmetry(sys7):
    rng = np.random.default_rng(0)
    no = sys7.k
    t1 = 0.2 * rng.standard_normal((7 - no, no))
    Lt = t1_transform(sys7.L, t1, no)
    # L~_ov = L_ov exactly: g~_iajb = g_iajb
    assert np.array_equal(Lt[:, :no, no:], sys7.L[:, :no, no:])
    g = np.einsum("Kpq,Krs->pqrs", sys7.L, sys7.L)
    assert np.abs(g - g.transpose(2, 3, 0, 1)).max() < 1e-13
    assert np.abs(g - g.transpose(1, 0, 2, 3)).max() < 1e-13
    # (1 - t) (1 + t) = 1: dressing by t then by -t gives back L
    back = t1_transform(Lt, -t1, no)
    assert np.abs(back - sys7.L).max() < 1e-13


def test_limits_reduce_between_models(sys7):
    """CCS/CCSD with the CC2 level equal to the CCSD level is MLCCSD; an empty CCSD
    level gives MLCC2 (Sec. 2.1): the three-level code must reproduce both, and a CCSD
    level that spans only occupied (or only virtual) orbitals must give the MLCC2 energy
    and Jacobian spectrum."""
    lev_a = np.array([0, 2, 2, 2, 2, 0, 0], dtype=np.int8)
    o = MLCCSystem(sys7.L, sys7.F, sys7.k, lev_a)
    assert not o.mask_S.any()
    lev_b = np.array([1, 1, 1, 1, 1, 1, 0], dtype=np.int8)
    o2 = MLCCSystem(sys7.L, sys7.F, sys7.k, lev_b)
    assert not o2.mask_T.any()
    ga = solve_ground_state(o)
    gb = solve_ground_state(o2)
    assert ga.converged and gb.converged
    # a CCSD level with occupied orbitals only (or virtual orbitals only) holds no doubles
    # with all four indices CCSD-active: the model is MLCC2 on the same CC2 set
    for lev_c in ([2, 1, 1, 1, 1, 1, 0], [1, 1, 2, 2, 1, 1, 0]):
        oc = MLCCSystem(sys7.L, sys7.F, sys7.k, np.array(lev_c, dtype=np.int8))
        assert not oc.mask_T.any()
        gc = solve_ground_state(oc)
        assert abs(gc.energy - gb.energy) < 1e-12
        wc = np.sort_complex(np.linalg.eigvals(_dense_jacobian(oc, gc)))
        wb = np.sort_complex(np.linalg.eigvals(_dense_jacobian(o2, gb)))
        assert np.abs(wc - wb).max() < 1e-9


@pytest.mark.parametrize("name,lev", PARTITIONS)
def test_invariant_under_relabelling_the_orbitals(sys7, name, lev):
    """The equations do not depend on the order in which the caller lists the orbitals of
    each level (Sec. 2.1 defines the levels as sets): permuting the occupied and the
    virtual orbitals, with their levels, leaves the correlation energy, the reference
    energy and the whole spectrum of the Jacobian unchanged."""
    t = sys7
    lev = np.array(lev, dtype=np.int8)
    o = MLCCSystem(t.L, t.F, t.k, lev)
    g = solve_ground_state(o)
    rng = np.random.default_rng(3)
    n, k = t.F.shape[0], t.k
    p = np.concatenate([rng.permutation(k), k + rng.permutation(n - k)])
    o2 = MLCCSystem(t.L[:, p][:, :, p], t.F[np.ix_(p, p)], k, lev[p])
    g2 = solve_ground_state(o2)
    assert abs(g.energy - g2.energy) < 1e-12
    assert abs(hf_energy(o) - hf_energy(o2)) < 1e-12
    # the whole Jacobian spectrum (a relabelling is a similarity transformation of A)
    w = np.linalg.eigvals(_dense_jacobian(o, g))
    w2 = np.linalg.eigvals(_dense_jacobian(o2, g2))
    key = lambda z: np.lexsort((np.round(z.imag, 8), np.round(z.real, 8)))
    assert np.abs(w[key(w)] - w2[key(w2)]).max() < 1e-9

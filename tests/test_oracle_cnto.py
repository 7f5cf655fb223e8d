"""Pins of the CNTO oracle (oracle/cnto.py, Sec. 2.2), each against something other than the
formula it restates:

  * gbar (Eq. approx_double_2) is the derivative of the X1-dressed integrals
    g~_aibj(t1 = h R) = sum_J L~^J_ai L~^J_bj at h = 0, evaluated by the complex step
    through the oracle's dressing (a different code path: the dressing of the whole L);
  * the CCS excitation energies and vectors are those of the CIS closed form
    (eps_a - eps_i) delta + 2 g_aijb - g_abji, diagonalised by LAPACK;
  * trace M = trace N = |R1|^2 + sum over independent doubles (ai <= bj) of R_aibj^2 for
    any symmetric doubles: the (1 + delta) factors of Eqs. M and N count each independent
    amplitude once (a dropped or misplaced delta breaks it);
  * with the doubles removed, M = R1^T R1 and N = R1 R1^T: the natural transition orbitals,
    whose non-zero eigenvalues are the squared singular values of R1 (LAPACK SVD);
  * the approximate doubles are symmetric under (ai) <-> (bj), and on the diagonal pairs
    they carry the extra 1/2 of Eq. approx_double_1;
  * Eq. select_CNTOs on the paper's proportionality.
"""
import numpy as np
import pytest

from oracle import cnto
from oracle.mlcc import MLCCSystem, gtilde_vovo, t1_transform


@pytest.fixture(scope="module")
def small():
    from synth import CONFIGS, make_system
    return make_system(CONFIGS["small"])


def _rng_R(nv, no, seed):
    R = np.random.default_rng(seed).standard_normal((nv, no))
    return R / np.linalg.norm(R)


def test_gbar_is_the_t1_derivative_of_the_dressed_integrals(small):
    no = small.spec.n_occ
    n = small.fock.shape[0]
    sys = MLCCSystem(small.L, small.fock, no, np.ones(n, dtype=np.int8))   # every orbital active
    R = _rng_R(n - no, no, 1)
    h = 1e-20
    Lt = t1_transform(small.L, 1j * h * R, no)
    dg = gtilde_vovo(sys, Lt).imag / h
    gb = cnto.gbar(small.L, no, R)
    assert np.abs(gb - dg).max() < 1e-13 * max(1.0, np.abs(gb).max())
    assert np.abs(gb - gb.transpose(2, 3, 0, 1)).max() == 0.0


def test_ccs_states_are_the_cis_eigenpairs(small):
    no = small.spec.n_occ
    L, F = small.L, small.fock
    nv = F.shape[0] - no
    eps = np.diag(F)
    g = np.einsum("Jpq,Jrs->pqrs", L, L, optimize=True)
    A = (np.diag((eps[no:, None] - eps[None, :no]).ravel())
         + (2.0 * np.einsum("aijb->aibj", g[no:, :no, :no, no:])
            - np.einsum("abji->aibj", g[no:, no:, :no, :no])).reshape(nv * no, nv * no))
    w, V = np.linalg.eigh(A)
    omega, R = cnto.ccs_states(L, F, no, 3)
    assert np.abs(omega - w[:3]).max() < 1e-10
    for k in range(3):
        assert abs(abs(R[k].ravel() @ V[:, k]) - 1.0) < 1e-9


def _packed_norm2(R2):
    nv, no = R2.shape[:2]
    m = R2.reshape(nv * no, nv * no)
    return float(np.sum(np.triu(m) ** 2))


@pytest.mark.parametrize("seed", [0, 1])
def test_traces_count_each_independent_amplitude_once(seed):
    rng = np.random.default_rng(seed)
    nv, no = 7, 4
    R1 = rng.standard_normal((nv, no))
    R2 = rng.standard_normal((nv, no, nv, no))
    R2 = R2 + R2.transpose(2, 3, 0, 1)
    M, N = cnto.cnto_matrices(R1, R2)
    want = float(np.sum(R1 ** 2)) + _packed_norm2(R2)
    assert abs(np.trace(M) - want) < 1e-12 * want
    assert abs(np.trace(N) - want) < 1e-12 * want
    assert np.abs(M - M.T).max() < 1e-14 and np.abs(N - N.T).max() < 1e-14
    assert np.linalg.eigvalsh(M).min() > -1e-12 and np.linalg.eigvalsh(N).min() > -1e-12


def test_without_doubles_the_cntos_are_the_ntos():
    R1 = _rng_R(9, 5, 3)
    M, N = cnto.cnto_matrices(R1, np.zeros((9, 5, 9, 5)))
    s = np.linalg.svd(R1, compute_uv=False)
    wm = np.sort(np.linalg.eigvalsh(M))[::-1]
    wn = np.sort(np.linalg.eigvalsh(N))[::-1]
    assert np.abs(wm - s ** 2).max() < 1e-14
    assert np.abs(wn[:5] - s ** 2).max() < 1e-14 and np.abs(wn[5:]).max() < 1e-14


def test_approximate_doubles(small):
    no = small.spec.n_occ
    omega, R = cnto.ccs_states(small.L, small.fock, no, 1)
    R2 = cnto.approx_doubles(small.L, small.fock, no, R[0], omega[0])
    assert np.abs(R2 - R2.transpose(2, 3, 0, 1)).max() == 0.0
    gb = cnto.gbar(small.L, no, R[0])
    eps = np.diag(small.fock)
    a, i = 3, 2
    den = 2.0 * (eps[no + a] - eps[i]) - omega[0]
    assert abs(R2[a, i, a, i] + gb[a, i, a, i] / (2.0 * den)) < 1e-15
    b, j = 5, 1
    den = eps[no + a] + eps[no + b] - eps[i] - eps[j] - omega[0]
    assert abs(R2[a, i, b, j] + gb[a, i, b, j] / den) < 1e-15


def test_selection_and_the_whole_construction(small):
    assert cnto.n_active_virtual(3, 8, 40) == 15
    assert cnto.n_active_virtual(1, 60, 500) == 8
    assert cnto.n_active_virtual(70, 60, 500) == 500
    r = cnto.cntos(small.L, small.fock, small.spec.n_occ, 2, 3)
    assert r.n_vir_active == 15
    assert np.all(np.diff(r.occ_values) <= 0) and np.all(np.diff(r.vir_values) <= 0)
    V = r.vir_vectors
    assert np.abs(V.T @ V - np.eye(V.shape[0])).max() < 1e-12
    # two unit-norm states: the traces are 2 plus the doubles' packed norms
    assert abs(np.trace(r.M) - np.trace(r.N)) < 1e-12 and np.trace(r.M) > 2.0

"""CNTO construction on the GPU (mlcc_cnto, Sec. 2.2) against the oracle (oracle/cnto.py),
and the paper's reduced-space workflow through the C ABI:

  * CCS energies, M and N (Eqs. M, N with the approximate doubles of Eqs. approx_double_1
    and approx_double_2) element by element, their eigenvalues and eigenvectors, and the
    active counts of Eq. select_CNTOs, in binary64 and MLCC_FP64E to 1e-10 relative and in
    BF16X3 to 1e-5; with the doubles built in row blocks of 50 (a ragged last block) and in
    one block;
  * an MLCC2 calculation in the CNTO basis (the active CNTOs CC2, the rest CCS): the orbitals
    rotated by the CNTOs give a Fock matrix that is not diagonal inside the levels, which the
    library semicanonicalises; its energies and excitation energies equal the oracle's on the
    same orbitals made semicanonical inside each level by numpy.
"""
import numpy as np
import pytest

from oracle import cnto as ocnto
from oracle.davidson import excited_states as oracle_es
from oracle.mlcc import MLCCSystem, solve_ground_state

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


@pytest.fixture(scope="module")
def small():
    from synth import CONFIGS, make_system
    return make_system(CONFIGS["small"])


@pytest.fixture(scope="module")
def ref(small):
    return ocnto.cntos(small.L, small.fock, small.spec.n_occ, 2, 3)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _vec_close(got, want, tol):
    """Columns equal up to sign where the eigenvalue is well separated."""
    for k in range(want.shape[1]):
        assert abs(abs(got[:, k] @ want[:, k]) - 1.0) < tol, k


@pytest.mark.parametrize("precision,block_rows,tol", [(0, 0, 1e-10), (0, 50, 1e-10), (4, 50, 1e-10),
                                                       (2, 0, 1e-5)])
def test_cnto_matrices_match_the_oracle(ctx, small, ref, precision, block_rows, tol):
    from paper_2006_05226_gb300 import mlcc
    no = small.spec.n_occ
    r = mlcc.cnto(ctx, _dev(small.L), _dev(small.fock), no, 2, 3, precision=precision, block_rows=block_rows)
    assert np.abs(r.omega - ref.omega).max() < 1e-10
    for got, want in ((r.m, ref.M), (r.n, ref.N), (r.occ_values, ref.occ_values), (r.vir_values, ref.vir_values)):
        assert np.abs(got - want).max() <= tol * np.abs(want).max()
    assert r.n_occ_active == 3 and r.n_vir_active == ref.n_vir_active == 15
    # eigenvectors of the separated eigenvalues (the leading ones that select the space)
    _vec_close(r.occ_vectors[:, :4], ref.occ_vectors[:, :4], 1e-6 if precision != 2 else 1e-3)
    _vec_close(r.vir_vectors[:, :6], ref.vir_vectors[:, :6], 1e-6 if precision != 2 else 1e-3)
    V = r.vir_vectors
    assert np.abs(V.T @ V - np.eye(V.shape[0])).max() < 1e-12


def _semicanonical(L, F, no, level):
    """numpy: diagonalise F inside each level's occupied and virtual blocks and rotate L."""
    n = F.shape[0]
    U = np.eye(n)
    for lo, hi in ((0, no), (no, n)):
        for v in (0, 1, 2):
            idx = lo + np.nonzero(level[lo:hi] == v)[0]
            if idx.size > 1:
                _, Q = np.linalg.eigh(F[np.ix_(idx, idx)])
                U[np.ix_(idx, idx)] = Q
    return np.einsum("pk,Jpq,ql->Jkl", U, L, U, optimize=True), U.T @ F @ U


def test_mlcc2_in_the_cnto_basis(ctx, small):
    from paper_2006_05226_gb300 import mlcc
    no = small.spec.n_occ
    n = small.fock.shape[0]
    r = mlcc.cnto(ctx, _dev(small.L), _dev(small.fock), no, 2, 3)
    C = np.zeros((n, n))
    C[:no, :no] = r.occ_vectors
    C[no:, no:] = r.vir_vectors
    Lc = np.einsum("pk,Jpq,ql->Jkl", C, small.L, C, optimize=True)
    Fc = C.T @ small.fock @ C
    level = np.zeros(n, dtype=np.int8)
    level[:r.n_occ_active] = 1                         # the leading CNTOs are CC2-active
    level[no:no + r.n_vir_active] = 1
    opts = mlcc.default_options(n_roots=2)
    sol = mlcc.solve(ctx, Lc, Fc, no, level, opts)
    Ls, Fs = _semicanonical(Lc, Fc, no, level)
    o = MLCCSystem(Ls, Fs, no, level)
    gs = solve_ground_state(o)
    es = oracle_es(o, gs, 2, res_tol=1e-9)
    assert abs(sol.gs.e_corr - gs.energy) < 1e-8
    assert np.abs(sol.omega - es.omega).max() < 1e-8
    # the reduced space recovers part of the full MLCC2 correlation energy
    full = mlcc.solve(ctx, small.L, small.fock, no, np.ones(n, dtype=np.int8), opts)
    assert full.gs.e_corr < sol.gs.e_corr < 0.0

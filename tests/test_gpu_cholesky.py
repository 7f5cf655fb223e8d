"""The MO-screened Cholesky decomposition and Algorithm 1 on the GPU (mlcc_mo_screening,
mlcc_cholesky_decompose, mlcc_cholesky_mo_vectors; Sec. 2.4) against the oracle
(oracle/cholesky.py): the same basis (pivot pairs in order), the vectors and the final
diagonal to 1e-10 relative, with and without MO screening, and the MO Cholesky vectors of
Algorithm 1 to 1e-10 relative; a cap on the number of vectors is respected.
"""
import numpy as np
import pytest

from oracle import cholesky as och

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


def _system(n_ao, n_aux, seed):
    from synth.generator import draw_model_hamiltonian
    ham = draw_model_hamiltonian(n_ao, n_aux, n_aux / 5.0, seed, 1.0)
    g = och.ao_integrals(ham.L)
    rng = np.random.default_rng(seed + 100)
    n_loc, n_act = max(2, n_ao // 3), max(2, n_ao // 4)
    C = np.zeros((n_ao, n_act))
    C[:n_loc] = rng.standard_normal((n_loc, n_act))
    C[n_loc:] = 1e-3 * rng.standard_normal((n_ao - n_loc, n_act))
    C_act = np.linalg.qr(C)[0]
    C_all = np.linalg.qr(rng.standard_normal((n_ao, n_ao)))[0][:, : n_ao - 2]
    return g, C_act, C_all


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n_ao,n_aux,seed", [(14, 60, 3), (40, 300, 4)])
@pytest.mark.parametrize("screened", [False, True])
def test_decomposition_matches_the_oracle(ctx, n_ao, n_aux, seed, screened):
    from paper_2006_05226_gb300 import mlcc
    g, C_act, C_all = _system(n_ao, n_aux, seed)
    tau = 1e-8
    w = och.mo_screening(C_act) if screened else None
    piv, L, D = och.pivoted_cholesky(g, tau, screen=w)
    gd = _dev(g)
    wd = mlcc.mo_screening(ctx, _dev(C_act)) if screened else None
    if screened:
        assert np.abs(wd.cpu().numpy() - w).max() <= 1e-15 * w.max()
    p2, L2, D2 = mlcc.cholesky_decompose(ctx, gd, tau, w=wd)
    assert p2 == piv
    scale = float(np.abs(L).max())
    assert np.abs(L2.cpu().numpy() - L).max() <= 1e-10 * scale
    assert np.abs(D2.cpu().numpy() - D).max() <= 1e-10 * float(np.diag(g).max())
    # Algorithm 1 on the basis found
    Lmo = och.mo_vectors(g, piv, C_all)
    Lmo2 = mlcc.cholesky_mo_vectors(ctx, gd, p2, _dev(C_all)).cpu().numpy()
    assert np.abs(Lmo2 - Lmo).max() <= 1e-10 * float(np.abs(Lmo).max())


def test_vector_cap(ctx):
    from paper_2006_05226_gb300 import mlcc
    g, _, _ = _system(14, 60, 3)
    piv, L, _ = och.pivoted_cholesky(g, 0.0, max_vectors=7)
    p2, L2, _ = mlcc.cholesky_decompose(ctx, _dev(g), 0.0, max_vectors=7)
    assert len(p2) == 7 and p2 == piv
    assert np.abs(L2.cpu().numpy() - L).max() <= 1e-10 * float(np.abs(L).max())

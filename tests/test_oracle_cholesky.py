"""Pins of the MO-screened Cholesky oracle (oracle/cholesky.py, Sec. 2.4), each against
something other than the loop it restates:

  * with tau = 0 on a positive definite matrix the factor reproduces it exactly, and its
    pivot rows are LAPACK's Cholesky factor of the pivoted matrix;
  * at termination the whole error matrix g - L L^T is positive semi-definite with its
    diagonal below tau, so every element is below tau (the decomposition's bound);
  * the factor equals the RI form g[:, B] Q^-T with S = g[B, B] = Q Q^T (the identity behind
    Algorithm 1), and Algorithm 1's MO vectors equal the MO transform of the factor;
  * MO screening: the diagonal of the MO-weighted matrix is bounded by nu_a nu_b D (Eq.
    mo_screening), the screened basis is smaller than the standard one on localised active
    orbitals, and every active MO pair's integral error obeys the Cauchy-Schwarz bound of
    the positive semi-definite residual built from the final diagonal.
"""
import numpy as np
import pytest

from oracle import cholesky as och


def _ao_system(n_ao=14, n_aux=60, seed=3):
    from synth.generator import draw_model_hamiltonian
    ham = draw_model_hamiltonian(n_ao, n_aux, 12.0, seed, 1.0)
    return och.ao_integrals(ham.L)


def _localised_active(n_ao, n_act, n_loc, seed):
    rng = np.random.default_rng(seed)
    C = np.zeros((n_ao, n_act))
    C[:n_loc] = rng.standard_normal((n_loc, n_act))
    C[n_loc:] = 1e-3 * rng.standard_normal((n_ao - n_loc, n_act))
    Q, _ = np.linalg.qr(C)
    return Q


def test_full_rank_exact_and_lapack():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 20))
    g = A @ A.T + 0.1 * np.eye(20)
    piv, L, D = och.pivoted_cholesky(g, 0.0)
    assert len(piv) == 20 and sorted(piv) == list(range(20))
    assert np.abs(L @ L.T - g).max() < 1e-12 * np.abs(g).max()
    Lp = np.linalg.cholesky(g[np.ix_(piv, piv)])
    assert np.abs(L[piv] - Lp).max() < 1e-12 * np.abs(Lp).max()


@pytest.mark.parametrize("tau", [1e-4, 1e-6, 1e-8])
def test_termination_bound(tau):
    g = _ao_system()
    piv, L, D = och.pivoted_cholesky(g, tau)
    R = g - L @ L.T
    assert np.linalg.eigvalsh(R).min() > -1e-12 * np.abs(g).max()
    assert np.abs(np.diag(R) - D).max() < 1e-11 * np.abs(g).max()
    assert D.max() < tau and np.abs(R).max() <= tau * (1 + 1e-9)
    assert len(piv) < g.shape[0]


def test_ri_form_and_algorithm_1():
    g = _ao_system()
    piv, L, _ = och.pivoted_cholesky(g, 1e-8)
    Q = np.linalg.cholesky(g[np.ix_(piv, piv)])
    ri = g[:, piv] @ np.linalg.inv(Q).T
    assert np.abs(ri - L).max() < 1e-9 * np.abs(L).max()
    n_ao = 14
    C = np.linalg.qr(np.random.default_rng(5).standard_normal((n_ao, 9)))[0]
    Lmo = och.mo_vectors(g, piv, C)
    direct = np.einsum("ap,bq,abJ->Jpq", C, C, L.reshape(n_ao, n_ao, -1), optimize=True)
    assert np.abs(Lmo - direct).max() < 1e-9 * np.abs(direct).max()
    # and the MO integrals to the decomposition's accuracy
    g_mo = np.einsum("ap,bq,abcd,cr,ds->pqrs", C, C, g.reshape(n_ao, n_ao, n_ao, n_ao), C, C, optimize=True)
    approx = np.einsum("Jpq,Jrs->pqrs", Lmo, Lmo)
    assert np.abs(g_mo - approx).max() < 1e-6


def test_mo_screening():
    n_ao = 14
    g = _ao_system()
    C = _localised_active(n_ao, 4, 5, 7)
    w = och.mo_screening(C)
    # the bound behind Eq. mo_screening: C_ap C_bq D_ab C_ap C_bq <= nu_a nu_b D_ab
    D = np.diag(g)
    Cab = np.einsum("ap,bq->abpq", C, C).reshape(n_ao * n_ao, -1) ** 2
    assert np.all(Cab * D[:, None] <= (w * D)[:, None] * (1 + 1e-12))
    tau = 1e-6
    piv_s, L_s, D_s = och.pivoted_cholesky(g, tau, screen=w)
    piv_0, _, _ = och.pivoted_cholesky(g, tau)
    assert len(piv_s) < len(piv_0)
    assert (w * D_s).max() < tau
    # active MO pair integrals: error <= the Cauchy-Schwarz bound of the PSD residual
    R = g - L_s @ L_s.T
    c = np.einsum("ap,bq->pqab", C, C).reshape(16, n_ao * n_ao)
    err = np.abs(np.einsum("xa,ab,yb->xy", c, R, c))
    bound = (np.abs(c) @ np.sqrt(np.maximum(D_s, 0.0))) ** 2
    assert np.all(np.diag(err) <= bound * (1 + 1e-9) + 1e-15)
    assert np.all(err <= np.sqrt(np.outer(bound, bound)) * (1 + 1e-9) + 1e-15)

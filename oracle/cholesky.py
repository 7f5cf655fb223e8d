"""MO-screened pivoted Cholesky decomposition of the AO two-electron integral matrix and the
construction of MO Cholesky vectors from the resulting basis (Sec. 2.4).

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy, in the paper's order:

  * g is the AO integral matrix with rows and columns indexed by AO pairs (alpha beta),
    g[(ab), (cd)] = (ab|cd); it is positive semi-definite.
  * Decomposition (Sec. 2.4): the updated diagonal D_(ab) = g_(ab)(ab) - sum_J (L^J_(ab))^2;
    the next basis element is the pair with the largest diagonal, and the procedure stops
    when that largest value is below tau (Eq. standard_cholesky). With MO screening the
    selection and the stop use the screened diagonal D~_(ab) = nu_a D_(ab) nu_b
    (Eq. cd_screening), nu_a = max_p (C^a_ap)^2 over the active MO coefficients
    (Eq. mo_screening). Each new vector is the pivot column minus the projection on the
    vectors so far, divided by the square root of the (unscreened) pivot diagonal.
  * MO vectors from the basis (Algorithm 1, the RI expression): S = g[B, B] = Q Q^T (lower
    Cholesky factor Q), X_pqK = sum_ab C_ap C_bq (ab|K), L^J_pq = sum_K X_pqK [Q^-T]_KJ.
"""
import numpy as np


def ao_integrals(B):
    """g[(ab), (cd)] = sum_P B^P_ab B^P_cd for factors B [P][n][n] (the synthetic stand-in for
    AO integrals: positive semi-definite by construction)."""
    P, n, _ = B.shape
    Bm = B.reshape(P, n * n)
    return Bm.T @ Bm


def mo_screening(C_active):
    """Eq. mo_screening and Eq. cd_screening: the weights nu_a nu_b of the screened diagonal,
    nu_a = max_p C_ap^2 over the active MOs (columns of C_active [n_ao][n_active])."""
    nu = np.max(C_active ** 2, axis=1)
    return np.outer(nu, nu).ravel()


def pivoted_cholesky(g, tau, screen=None, max_vectors=None):
    """(pivots, L [n_pairs][N_J], final diagonal D) of the decomposition of g (Sec. 2.4).
    screen: the weights of the screened diagonal (None: the standard decomposition)."""
    m = g.shape[0]
    w = np.ones(m) if screen is None else np.asarray(screen, dtype=np.float64)
    D = np.diag(g).astype(np.float64).copy()
    cols, piv = [], []
    limit = m if max_vectors is None else int(max_vectors)
    while len(piv) < limit:
        Dt = w * D
        K = int(np.argmax(Dt))
        if not Dt[K] >= tau or D[K] <= 0.0:
            break
        col = g[:, K].astype(np.float64).copy()
        for Lj in cols:
            col -= Lj * Lj[K]
        Lk = col / np.sqrt(D[K])
        D -= Lk ** 2
        D[K] = 0.0
        cols.append(Lk)
        piv.append(K)
    L = np.stack(cols, axis=1) if cols else np.zeros((m, 0))
    return piv, L, D


def mo_vectors(g, pivots, C):
    """Algorithm 1: L^J_pq [N_J][n_mo][n_mo] from the basis (pivots) and MO coefficients
    C [n_ao][n_mo]: X_pqK = sum_ab C_ap C_bq (ab|K), S = g[B, B] = Q Q^T, L = X Q^-T."""
    n_ao, n_mo = C.shape
    S = g[np.ix_(pivots, pivots)]
    Q = np.linalg.cholesky(S)
    cols = g[:, pivots].reshape(n_ao, n_ao, len(pivots))
    X = np.einsum("ap,bq,abK->pqK", C, C, cols, optimize=True)
    Qinv_T = np.linalg.inv(Q).T                  # [Q^-T]_KJ
    L = np.einsum("pqK,KJ->Jpq", X, Qinv_T, optimize=True)
    return L

"""Restricted closed-shell Hartree-Fock on a Cholesky-factorised model Hamiltonian.

Input preparation only: the multilevel CC method takes the canonical MO quantities this
produces (the orbitals in which Sec. 2.3 builds the Fock matrix). Orthonormal basis
(S = I), Roothaan iterations with Pulay DIIS on the commutator FD - DF, aufbau occupation
of the lowest n_occ orbitals.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class RHFResult:
    energy: float          # E_HF = sum_pq D_pq (h_pq + F_pq)
    C: np.ndarray          # [n, n] canonical orbitals, columns sign-fixed
    eps: np.ndarray        # [n] orbital energies, ascending
    fock: np.ndarray       # [n, n] AO Fock matrix at convergence
    iterations: int
    gradient: float        # max |FD - DF| at convergence
    converged: bool


def _fock(h, L, D):
    # J_pq = sum_K L^K_pq (L^K . D);  K_pq = sum_K (L^K D L^K)_pq
    coul = np.einsum("kpq,kpq->k", L, D[None, :, :], optimize=True)
    J = np.tensordot(coul, L, axes=(0, 0))
    LD = np.matmul(L, D)                      # [K, n, n]
    Kx = np.einsum("kpr,krq->pq", LD, L, optimize=True)
    return h + 2.0 * J - Kx


def _sign_fix(C):
    # largest-|.| coefficient of each column positive
    idx = np.argmax(np.abs(C), axis=0)
    s = np.sign(C[idx, np.arange(C.shape[1])])
    s[s == 0] = 1.0
    return C * s


def rhf(h, L, n_occ, tol=1e-10, max_iter=500, diis_dim=8, chunk=None):
    """Closed-shell RHF with density D = C_occ C_occ^T (per spin)."""
    n = h.shape[0]
    eps, C = np.linalg.eigh(h)
    D = C[:, :n_occ] @ C[:, :n_occ].T
    errs, focks = [], []
    grad = np.inf
    for it in range(1, max_iter + 1):
        F = _fock(h, L, D)
        err = F @ D - D @ F
        grad = float(np.max(np.abs(err)))
        if grad < tol:
            E = float(np.sum(D * (h + F)))
            eps, C = np.linalg.eigh(F)
            return RHFResult(E, _sign_fix(C), eps, F, it, grad, True)
        errs.append(err)
        focks.append(F)
        if len(errs) > diis_dim:
            errs.pop(0)
            focks.pop(0)
        m = len(errs)
        if m >= 2:
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for a in range(m):
                for b in range(m):
                    B[a, b] = np.sum(errs[a] * errs[b])
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                coef = np.linalg.solve(B, rhs)[:m]
                F = sum(c * f for c, f in zip(coef, focks))
            except np.linalg.LinAlgError:
                pass
        eps, C = np.linalg.eigh(F)
        D = C[:, :n_occ] @ C[:, :n_occ].T
    F = _fock(h, L, D)
    E = float(np.sum(D * (h + F)))
    eps, C = np.linalg.eigh(F)
    return RHFResult(E, _sign_fix(C), eps, F, max_iter, grad, False)

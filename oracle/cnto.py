"""Correlated natural transition orbitals (CNTOs) from CCS excitation vectors (Sec. 2.2).

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy, in the paper's order:

  1. CCS excitation vectors R_ai and energies omega (the Jacobian of the all-CCS partition;
     at the Hartree-Fock reference t1 = 0 and it is the CIS matrix).
  2. Approximate doubles (Eqs. approx_double_1 and approx_double_2, after Baudin and
     Kristensen's CIS(D)-based construction):
        gbar_aibj = P^{ab}_{ij} ( sum_{cJ} R_ci L^J_bj L^J_ac - sum_{kJ} R_bk L^J_kj L^J_ai )
        R_aibj    = - gbar_aibj / ((1 + delta_{ai,bj}) (eps_a + eps_b - eps_i - eps_j - omega))
     with P^{ab}_{ij} I_{ai,bj} = I_{ai,bj} + I_{bj,ai}; all orbitals, not only active ones.
  3. The matrices of Eqs. M and N,
        M_ij = sum_a R_ai R_aj + 1/2 sum_abk (1 + delta_{ai,bk} delta_ij) R_aibk R_ajbk
        N_ab = sum_i R_ai R_bi + 1/2 sum_ijc (1 + delta_{ai,cj} delta_ab) R_aicj R_bicj
     summed over the states considered together (Sec. 2.2, last paragraph).
  4. Their eigenvectors are the occupied and virtual CNTOs; the active ones are those of
     the largest eigenvalues, n_v^a = (N_v / N_o) n_o^a (Eq. select_CNTOs).

Readings: R_ai is normalised to unit 2-norm before step 2 (the paper does not state a
normalisation; the selection only orders eigenvalues, so a common scale changes nothing);
n_v^a of Eq. select_CNTOs is rounded to the nearest integer, at least 1 and at most N_v.
"""
import numpy as np

from .davidson import excited_states
from .mlcc import MLCCSystem, solve_ground_state


def ccs_states(L, F, no, n_states, res_tol=1e-11):
    """(omega [n_states], R [n_states, N_v, N_o]) of the CCS Jacobian, R unit 2-norm."""
    n = F.shape[0]
    sys = MLCCSystem(L, F, no, np.zeros(n, dtype=np.int8))
    gs = solve_ground_state(sys)
    res = excited_states(sys, gs, n_states, res_tol=res_tol)
    R = res.vectors.T.reshape(n_states, n - no, no)
    R = R / np.linalg.norm(R.reshape(n_states, -1), axis=1)[:, None, None]
    return res.omega, R


def gbar(L, no, R):
    """Eq. approx_double_2: gbar_aibj for one CCS singles vector R [N_v, N_o]."""
    L_vo = L[:, no:, :no]
    L_vv = L[:, no:, no:]
    L_oo = L[:, :no, :no]
    first = np.einsum("ci,Jbj,Jac->aibj", R, L_vo, L_vv, optimize=True)
    second = np.einsum("bk,Jkj,Jai->aibj", R, L_oo, L_vo, optimize=True)
    X = first - second
    return X + X.transpose(2, 3, 0, 1)


def approx_doubles(L, F, no, R, omega):
    """Eq. approx_double_1: R_aibj = -gbar_aibj / ((1 + delta_{ai,bj}) (eps^{ab}_{ij} - omega))."""
    eps = np.diag(F)
    e_ai = eps[no:, None] - eps[None, :no]
    den = e_ai[:, :, None, None] + e_ai[None, None, :, :] - omega
    R2 = -gbar(L, no, R) / den
    nv = R.shape[0]
    a, i = np.meshgrid(np.arange(nv), np.arange(no), indexing="ij")
    R2[a, i, a, i] *= 0.5          # 1 / (1 + delta_{ai,bj}) on the diagonal pairs
    return R2


def cnto_matrices(R1, R2):
    """Eqs. M and N for one state: R1 [N_v, N_o], R2 [N_v, N_o, N_v, N_o]."""
    nv, no = R1.shape
    M = R1.T @ R1 + 0.5 * np.einsum("aibk,ajbk->ij", R2, R2, optimize=True)
    N = R1 @ R1.T + 0.5 * np.einsum("aicj,bicj->ab", R2, R2, optimize=True)
    # the (1 + delta) factors: the diagonal doubles element R_aiai enters M_ii and N_aa twice
    a, i = np.meshgrid(np.arange(nv), np.arange(no), indexing="ij")
    d = R2[a, i, a, i] ** 2        # [N_v, N_o]
    M[np.arange(no), np.arange(no)] += 0.5 * d.sum(axis=0)
    N[np.arange(nv), np.arange(nv)] += 0.5 * d.sum(axis=1)
    return M, N


def n_active_virtual(n_occ_active, no, nv):
    """Eq. select_CNTOs, n_v^a = (N_v / N_o) n_o^a, rounded to the nearest integer."""
    return int(min(nv, max(1, int(np.floor(nv / no * n_occ_active + 0.5)))))


class CNTOs:
    def __init__(self, omega, M, N, occ_values, occ_vectors, vir_values, vir_vectors, n_occ_active,
                 n_vir_active):
        self.omega, self.M, self.N = omega, M, N
        self.occ_values, self.occ_vectors = occ_values, occ_vectors
        self.vir_values, self.vir_vectors = vir_values, vir_vectors
        self.n_occ_active, self.n_vir_active = n_occ_active, n_vir_active


def cntos(L, F, no, n_states, n_occ_active, n_vir_active=None):
    """The whole construction: CCS states, approximate doubles, M and N summed over the
    states, their eigenpairs in descending order of eigenvalue (columns of the vectors),
    and the active counts (n_vir_active None: Eq. select_CNTOs)."""
    omega, R = ccs_states(L, F, no, n_states)
    nv = F.shape[0] - no
    M = np.zeros((no, no))
    N = np.zeros((nv, nv))
    for k in range(n_states):
        R2 = approx_doubles(L, F, no, R[k], omega[k])
        Mk, Nk = cnto_matrices(R[k], R2)
        M += Mk
        N += Nk
    wo, Vo = np.linalg.eigh(M)
    wv, Vv = np.linalg.eigh(N)
    wo, Vo = wo[::-1], Vo[:, ::-1]
    wv, Vv = wv[::-1], Vv[:, ::-1]
    if n_vir_active is None:
        n_vir_active = n_active_virtual(n_occ_active, no, nv)
    return CNTOs(omega, M, N, wo, Vo, wv, Vv, n_occ_active, n_vir_active)

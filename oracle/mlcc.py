"""FP64 reference implementation of the MLCC2 / MLCCSD ground state and Jacobian transformation.

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy, written term by term
in the notation of arXiv 2006.05226 Appendix A: indices A, B, C (I, J, K as orbitals) run
over all virtual (occupied) orbitals, a, b, c (i, j, k, l) over active ones; K or J in
einsum strings is the Cholesky index. Storage conventions:

  t1[A, I]                 singles amplitudes x_AI, all virtuals x all occupied
  x2[a, i, b, j]           doubles amplitudes x^{ab}_{ij} on the CC2-active orbitals,
                           symmetric under (ai) <-> (bj); X2 = 1/2 sum x_aibj E_ai E_bj
  omega / sigma doubles    the same layout: the coefficient of E_ai E_bj |HF> (times 2 on
                           the ai = bj diagonal), i.e. the biorthonormal projection

Three orbital levels (Sec. 2.1): CCSD-active subset of CC2-active subset of all orbitals.
Doubles live on D_CC2 (all four indices CC2-active). P_T is the part with all four
indices CCSD-active, P_S the rest. Reading for the three-level model, which the paper
names but does not write out: rows in P_S obey the CC2 doubles equation
(g~_aibj + eps_aibj x_aibj = 0), rows in P_T the CCSD doubles equation built from the
P_T amplitudes only, and the singles, the energy and u = 2x - x^T use all of x2. With no
CCSD level this is MLCC2, with CCSD = CC2 it is the CCS/CCSD model of the paper, and with
everything active it is CC2 or CCSD.
"""
import numpy as np

LEVEL_CCS, LEVEL_CC2, LEVEL_CCSD = 0, 1, 2


def _es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


class MLCCSystem:
    """MO Cholesky vectors L^K_PQ, Fock matrix F_PQ and the orbital partition.

    Occupied orbitals come first. level[P] is 0 (CCS), 1 (CC2) or 2 (CCSD); the levels
    must nest (CCSD-active orbitals are also CC2-active).
    """

    def __init__(self, L, fock, n_occ, level):
        self.L = np.asarray(L, dtype=np.float64)
        self.F = np.asarray(fock, dtype=np.float64)
        self.no = int(n_occ)
        self.n = self.F.shape[0]
        self.nv = self.n - self.no
        level = np.asarray(level)
        self.level = level
        no = self.no
        # CC2-active sets (ascending orbital order) and the CCSD subset inside them
        self.os = np.nonzero(level[:no] >= LEVEL_CC2)[0]
        self.vs = np.nonzero(level[no:] >= LEVEL_CC2)[0]
        self.ot = np.nonzero(level[:no][self.os] == LEVEL_CCSD)[0]
        self.vt = np.nonzero(level[no:][self.vs] == LEVEL_CCSD)[0]
        self.so, self.sv = self.os.size, self.vs.size
        self.to, self.tv = self.ot.size, self.vt.size
        mo = np.zeros(self.so, bool)
        mo[self.ot] = True
        mv = np.zeros(self.sv, bool)
        mv[self.vt] = True
        self.mask_T = (mv[:, None, None, None] & mo[None, :, None, None]
                       & mv[None, None, :, None] & mo[None, None, None, :])
        self.mask_S = ~self.mask_T
        self.eps = np.diag(self.F).copy()
        eo, ev = self.eps[:no], self.eps[no:]
        self.eps_ai = ev[:, None] - eo[None, :]
        ea = self.eps_ai[np.ix_(self.vs, self.os)]
        self.eps_aibj = ea[:, :, None, None] + ea[None, None, :, :]
        self.h = h_eff(self.L, self.F, no)

    # index helpers --------------------------------------------------------------
    @property
    def V(self):
        return self.no + self.vs

    @property
    def O(self):
        return self.os

    def tbox(self):
        """Global orbital indices of the CCSD-active occupied and virtual orbitals."""
        return self.os[self.ot], self.no + self.vs[self.vt]

    def doubles_shape(self):
        return (self.sv, self.so, self.sv, self.so)

    def vector_len(self):
        return self.nv * self.no + self.sv * self.so * self.sv * self.so


def h_eff(L, F, no):
    """One-electron matrix of the reduced space, Sec. 2.3 Eq. eff_fock.

    F = h + sum_i (2 g_pqii - g_piiq) + F^e with i over the occupied orbitals of the
    reduced space; the frozen-environment part F^e is absorbed into the returned h.
    """
    coul = np.einsum("Kii->K", L[:, :no, :no])
    J = np.tensordot(coul, L, axes=(0, 0))
    Kx = np.einsum("Kpi,Kiq->pq", L[:, :, :no], L[:, :no, :], optimize=True)
    return F - (2.0 * J - Kx)


def t1_matrix(t1, no, n):
    T = np.zeros((n, n), dtype=t1.dtype)
    T[no:, :no] = t1
    return T


def t1_transform(M, t1, no):
    """X1-basis transformation (Sec. 2.1, Appendix A): M~ = (1 - t1) M (1 + t1).

    t1 is placed in the virtual-occupied block of an n x n matrix T; exp(-X1) E_pq exp(X1)
    maps a one-index-pair operator with matrix M to exp(-T) M exp(T) = (1 - T) M (1 + T)
    because T is nilpotent (T^2 = 0). Applies to h and to every Cholesky vector L^K.
    """
    n = M.shape[-1]
    T = t1_matrix(t1, no, n)
    I = np.eye(n)
    return np.matmul(np.matmul(I - T, M), I + T)


def fock_t1(h_t, Lt, no):
    """Fock matrix in the X1 basis (Appendix A):
    F~_PQ = h~_PQ + 2 L~^K_PQ L~^K_II - L~^K_PI L~^K_IQ   (sum over all occupied I).
    Reading: the printed formula omits the one-electron term h~; it is added here.
    """
    coul = np.einsum("KII->K", Lt[:, :no, :no])
    return (h_t + 2.0 * np.tensordot(coul, Lt, axes=(0, 0))
            - np.einsum("KPI,KIQ->PQ", Lt[:, :, :no], Lt[:, :no, :], optimize=True))


def u_of(x2):
    """u^{ab}_{ij} = 2 x^{ab}_{ij} - x^{ab}_{ji}  (Appendix A, below Eq. mlcc2_omega_codable)."""
    return 2.0 * x2 - x2.transpose(0, 3, 2, 1)


def gtilde_vovo(sys, Lt):
    """g~_aibj = L~^K_ai L~^K_bj on the CC2-active orbitals (Appendix A)."""
    Lvo = Lt[:, sys.V][:, :, sys.O]
    n_ai = sys.sv * sys.so
    Lm = Lvo.reshape(Lvo.shape[0], n_ai)
    return (Lm.T @ Lm).reshape(sys.doubles_shape())


def cc2_amplitudes(sys, gt):
    """Analytic CC2 doubles on P_S, Appendix A: s^{ab}_{ij} = -g~_aibj / (F_aa+F_bb-F_ii-F_jj)."""
    s = np.zeros(sys.doubles_shape(), dtype=gt.dtype)
    s[sys.mask_S] = -gt[sys.mask_S] / sys.eps_aibj[sys.mask_S]
    return s


def omega_singles(sys, Lt, Ft, x2):
    """Omega_AI, Appendix A Eq. mlcc2_omega_codable (same expression for MLCCSD with t):

    Omega_AI = F~_AI + ((u^{bc}_{ij} L~^K_jc) L~^K_Ab) d_Ii - (u^{ab}_{jk} g~_kbjI) d_Aa
               + (u^{ab}_{ij} F~_jb) d_{AI,ai}
    """
    no, O, V = sys.no, sys.O, sys.V
    u = u_of(x2)
    om = Ft[no:, :no].copy().astype(np.result_type(Ft, x2))
    L_jc = Lt[:, O][:, :, V]                    # L~^K_jc   [K, j, c]
    L_Ab = Lt[:, no:][:, :, V]                  # L~^K_Ab   [K, A, b]
    L_jI = Lt[:, O][:, :, :no]                  # L~^K_jI   [K, j, I]
    # Z^K_bi = u^{bc}_{ij} L~^K_jc, shared by the second and third term
    Z = _es("bicj,Kjc->Kbi", u, L_jc)
    om[:, O] += _es("KAb,Kbi->Ai", L_Ab, Z)
    # u^{ab}_{jk} g~_kbjI = (u^{ab}_{jk} L~^K_kb) L~^K_jI = Z^K_aj L~^K_jI
    om[sys.vs, :] -= _es("Kaj,KjI->aI", Z, L_jI)
    F_jb = Ft[O][:, V]
    om[np.ix_(sys.vs, O)] += _es("aibj,jb->ai", u, F_jb)
    return om


def omega_ccsd_doubles(sys, Lt, Ft, t):
    """MLCCSD doubles residual on P_T, Appendix A (Omega_aibj below Eq. mlcc2_omega2).

    t[a, i, b, j] = t^{ab}_{ij} over the CCSD-active orbitals only. Readings of the
    printed equation (all indices CCSD-active, all integrals in the X1 basis):
      * g_aikc, g_kiac printed without tilde are read as g~;
      * Y_aick = g~_kiac - 1/2 t^{ad}_{li} g~_kdlc (the printed contraction index pattern
        is garbled);
      * the occupied Fock-like term is -t^{ab}_{ik} (F~_kj + g~_ldkc u^{dc}_{lj}) (the
        printed minus in front of g~ is a sign slip; the brute-force pin fixes it);
      * the operator P^{ab}_{ij} X_aibj = X_aibj + X_bjai applies to the C, D and E lines
        (the terms with Y, with u and with F~), the first line is symmetric already.
    """
    o, v = sys.tbox()
    L_ai = Lt[:, v][:, :, o]
    L_ac = Lt[:, v][:, :, v]
    L_ki = Lt[:, o][:, :, o]
    L_kc = Lt[:, o][:, :, v]
    g_aibj = _es("Kai,Kbj->aibj", L_ai, L_ai)
    g_acbd = _es("Kac,Kbd->acbd", L_ac, L_ac)
    g_kilj = _es("Kki,Klj->kilj", L_ki, L_ki)
    g_kcld = _es("Kkc,Kld->kcld", L_kc, L_kc)
    g_kiac = _es("Kki,Kac->kiac", L_ki, L_ac)
    g_aikc = _es("Kai,Kkc->aikc", L_ai, L_kc)
    Lg_ldkc = 2.0 * g_kcld - g_kcld.transpose(0, 3, 2, 1)     # L~_ldkc = 2g~_ldkc - g~_lckd
    F_bc = Ft[v][:, v]
    F_kj = Ft[o][:, o]
    u = u_of(t)

    om = (g_aibj
          + _es("acbd,cidj->aibj", g_acbd, t)
          + _es("akbl,kilj->aibj", t, g_kilj + _es("cidj,kcld->kilj", t, g_kcld)))
    Y = g_kiac.transpose(2, 1, 3, 0) - 0.5 * _es("aldi,kdlc->aick", t, g_kcld)
    C = -0.5 * _es("bkcj,aick->aibj", t, Y) - _es("bkci,ajck->aibj", t, Y)
    D = (-0.5 * _es("bjck,kiac->aibj", u, g_kiac)
         + 0.25 * _es("bjck,ldkc,aidl->aibj", u, Lg_ldkc, u)
         + _es("bjck,aikc->aibj", u, g_aikc))
    E = (_es("aicj,bc->aibj", t, F_bc - _es("ldkc,bkdl->bc", g_kcld, u))
         - _es("aibk,kj->aibj", t, F_kj + _es("ldkc,dlcj->kj", g_kcld, u)))
    CDE = C + D + E
    return om + CDE + CDE.transpose(2, 3, 0, 1)


def _tbox_index(sys):
    return np.ix_(sys.vt, sys.ot, sys.vt, sys.ot)


def omega(sys, t1, x2, return_parts=False):
    """Ground-state residual Omega(x) with t1 and the doubles x2 as independent variables.

    Singles: Omega_AI (Eq. mlcc2_omega_codable). Doubles on P_S: the CC2 equation
    <mu2|H~ + [F, S2]|HF> = g~_aibj + eps_aibj x_aibj in the semicanonical basis
    (Eq. mlcc2_2). Doubles on P_T: the MLCCSD residual (Eq. mlccsd_2).
    """
    Lt = t1_transform(sys.L, t1, sys.no)
    ht = t1_transform(sys.h, t1, sys.no)
    Ft = fock_t1(ht, Lt, sys.no)
    return _omega_dressed(sys, t1, x2, Lt, Ft, return_parts)


def _omega_dressed(sys, t1, x2, Lt, Ft, return_parts=False, gt=None):
    dt = np.result_type(Lt, x2)
    om2 = np.zeros(sys.doubles_shape(), dtype=dt)
    if sys.mask_S.any():
        if gt is None:
            gt = gtilde_vovo(sys, Lt)
        om2[sys.mask_S] = gt[sys.mask_S] + sys.eps_aibj[sys.mask_S] * x2[sys.mask_S]
    if sys.to and sys.tv:
        ix = _tbox_index(sys)
        om2[ix] = omega_ccsd_doubles(sys, Lt, Ft, x2[ix])
    om1 = omega_singles(sys, Lt, Ft, x2)
    if return_parts:
        return om1, om2, Lt, Ft
    return om1, om2


def energy(sys, t1, x2):
    """Correlation energy, Appendix A Eq. mlcc_energy, with L_PQRS = 2 g_PQRS - g_PSRQ:

    E = x^A_I x^B_J L_IAJB + x^{ab}_{ij} L_iajb, the first term evaluated as
    2 (L^K_IA x_AI)(L^K_JB x_BJ) - (L^K_IB x_BJ)(L^K_JA x_AI).
    """
    no = sys.no
    L_IA = sys.L[:, :no, no:]
    a = np.einsum("KIA,AI->K", L_IA, t1)
    M = np.einsum("KIB,BJ->KIJ", L_IA, t1)
    e1 = 2.0 * (a @ a) - np.einsum("KIJ,KJI->", M, M)
    L_ia = sys.L[:, sys.O][:, :, sys.V]
    g = _es("Kia,Kjb->iajb", L_ia, L_ia)
    Lg = 2.0 * g - g.transpose(0, 3, 2, 1)
    e2 = np.einsum("aibj,iajb->", x2, Lg)
    return float(np.real(e1 + e2))


def hf_energy(sys):
    """E_HF = sum_I (h_II + F_II) of the reduced space (x2 spin), from h of Eq. eff_fock."""
    no = sys.no
    return float(np.trace(sys.h[:no, :no]) + np.trace(sys.F[:no, :no]))


class GroundState:
    def __init__(self, t1, x2, energy, omega_norm, iterations, converged, history):
        self.t1, self.x2, self.energy = t1, x2, energy
        self.omega_norm, self.iterations, self.converged = omega_norm, iterations, converged
        self.history = history


def solve_ground_state(sys, tol=1e-11, e_tol=1e-12, max_iter=200, diis_dim=8, verbose=False):
    """DIIS-accelerated quasi-Newton solver for Omega = 0 (Sec. 2.1).

    Each iteration: X1-dress L and h, build F~, build the CC2 doubles on P_S analytically
    from the current t1 (Appendix A, s = -g~/eps), evaluate the residual, the energy and
    the norm, then take the quasi-Newton step x <- x - Omega / eps_mu on the singles and
    the P_T doubles and extrapolate with DIIS over the last diis_dim pairs of updated
    amplitudes and quasi-Newton steps Omega / eps_mu.
    """
    no, nv = sys.no, sys.nv
    t1 = np.zeros((nv, no))
    x2 = np.zeros(sys.doubles_shape())
    ix = _tbox_index(sys) if (sys.to and sys.tv) else None
    tT = np.zeros((sys.tv, sys.to, sys.tv, sys.to))
    epsT = sys.eps_aibj[ix] if ix is not None else None
    vecs, errs, hist = [], [], []
    e_old = 0.0
    for it in range(1, max_iter + 1):
        Lt = t1_transform(sys.L, t1, no)
        ht = t1_transform(sys.h, t1, no)
        Ft = fock_t1(ht, Lt, no)
        gt = gtilde_vovo(sys, Lt) if sys.mask_S.any() else None
        x2 = cc2_amplitudes(sys, gt) if gt is not None else np.zeros(sys.doubles_shape())
        if ix is not None:
            x2[ix] = tT
        om1, om2 = _omega_dressed(sys, t1, x2, Lt, Ft, gt=gt)
        e = energy(sys, t1, x2)
        nrm = np.sqrt(np.sum(om1 ** 2) + (np.sum(om2[ix] ** 2) if ix is not None else 0.0))
        hist.append((e, nrm))
        if verbose:
            print(f"GS it {it:3d}  E = {e:.14f}  |Omega| = {nrm:.3e}")
        if nrm < tol and abs(e - e_old) < e_tol:
            return GroundState(t1, x2, e, nrm, it, True, hist)
        e_old = e
        t1n = t1 - om1 / sys.eps_ai
        vec = [t1n.ravel()]
        err = [(om1 / sys.eps_ai).ravel()]
        if ix is not None:
            vec.append((tT - om2[ix] / epsT).ravel())
            err.append((om2[ix] / epsT).ravel())
        vecs.append(np.concatenate(vec))
        errs.append(np.concatenate(err))
        if len(vecs) > diis_dim:
            vecs.pop(0)
            errs.pop(0)
        m = len(vecs)
        p = vecs[-1]
        if m > 1:
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            B[:m, :m] = np.array([[ea @ eb for eb in errs] for ea in errs])
            B[:m, :m] /= np.max(np.abs(np.diag(B[:m, :m])))
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
            p = sum(ci * vi for ci, vi in zip(c, vecs))
        t1 = p[: nv * no].reshape(nv, no).copy()
        if ix is not None:
            tT = p[nv * no:].reshape(tT.shape).copy()
    return GroundState(t1, x2, e, nrm, max_iter, False, hist)


def sigma(sys, t1, x2, c1, c2, h=1e-20):
    """Jacobian transformation sigma = A c with A_mu,nu = dOmega_mu / dx_nu (Sec. 2.1).

    The Jacobian is the derivative of the residual defined in omega() with respect to the
    amplitudes (singles and the D_CC2 doubles taken as independent). sigma is its
    directional derivative along c, evaluated exactly (to rounding) by the complex step
    Im Omega(x + i h c) / h: Omega is a polynomial in the amplitudes, so no truncation
    error remains at h = 1e-20.
    """
    om1, om2 = omega(sys, t1 + 1j * h * c1, x2 + 1j * h * c2)
    return om1.imag / h, om2.imag / h


def sigma_mlcc2_paper(sys, t1, x2, c1, c2):
    """The paper's explicit MLCC2 Jacobian transformation (Appendix A, Eq. mlcc_A_ and the
    sigma^MLCC2_aibj equation). Valid when there are no CCSD-active doubles.

    Readings of the printed singles equation (fixed by comparison with sigma()):
      * the doubles-to-singles term (2c - c^T)^{bc}_{ij} g~_Abjc (the derivative of the
        second term of Eq. mlcc2_omega_codable) is missing in print and is added;
      * the term -L_jbki c_akbj is read as -L~_jbkI c_akbj with I unrestricted
        (derivative of the third term), L~_pqrs = 2 g~_pqrs - g~_psrq;
      * the doubles part carries P^{ab}_{ij}: sigma_aibj = X_aibj + X_bjai + eps c_aibj.
    """
    no, O, V, vs = sys.no, sys.O, sys.V, sys.vs
    Lt = t1_transform(sys.L, t1, no)
    ht = t1_transform(sys.h, t1, no)
    Ft = fock_t1(ht, Lt, no)
    u = u_of(x2)
    F_AB, F_JI = Ft[no:, no:], Ft[:no, :no]
    L_JB, L_AI = Lt[:, :no, no:], Lt[:, no:, :no]
    L_AB, L_JI = Lt[:, no:, no:], Lt[:, :no, :no]
    # CCS terms
    s1 = F_AB @ c1 - c1 @ F_JI
    s1 += 2.0 * np.tensordot(np.einsum("KJB,BJ->K", L_JB, c1), L_AI, axes=(0, 0))
    s1 -= _es("KAB,BJ,KJI->AI", L_AB, c1, L_JI)
    # MLCC2 singles terms from t1-dependence of F~_kc and L~
    L_kc = Lt[:, O][:, :, V]
    L_kB = Lt[:, O][:, :, no:]
    L_Jc = Lt[:, :no][:, :, V]
    dF_kc = (2.0 * _es("KJB,BJ,Kkc->kc", L_JB, c1, L_kc)
             - _es("KkB,BJ,KJc->kc", L_kB, c1, L_Jc))
    s1[np.ix_(vs, O)] += _es("kc,aick->ai", dF_kc, u)
    X_Ji = _es("KJb,Kkc,ckbi->Ji", Lt[:, :no][:, :, V], L_kc, u)
    Y_aB = _es("Kkc,KjB,ajck->aB", L_kc, Lt[:, O][:, :, no:], u)
    s1[:, O] -= c1 @ X_Ji
    s1[vs, :] -= Y_aB @ c1
    # doubles -> singles
    uc = u_of(c2)
    Zc = _es("bicj,Kjc->Kbi", uc, L_kc)
    s1[:, O] += _es("KAb,Kbi->Ai", Lt[:, no:][:, :, V], Zc)
    s1[vs, :] -= _es("Kaj,KjI->aI", Zc, Lt[:, O][:, :, :no])
    s1[np.ix_(vs, O)] += _es("jb,aibj->ai", Ft[O][:, V], uc)
    # doubles: (L~^K_bC c_Cj - c_bK L~^K_Kj) L~^K_ai, symmetrised, + eps c
    L_ai = Lt[:, V][:, :, O]
    Vb = (_es("KbC,Cj->Kbj", Lt[:, V][:, :, no:], c1[:, O])
          - _es("bM,KMj->Kbj", c1[vs, :], Lt[:, :no][:, :, O]))
    W = _es("Kai,Kbj->aibj", L_ai, Vb)
    s2 = W + W.transpose(2, 3, 0, 1) + sys.eps_aibj * c2
    return s1, s2

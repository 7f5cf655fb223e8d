"""Brute-force determinant-space coupled cluster: the independent pin for the oracle.

Nothing here shares code or formulas with oracle/. Operators are built as sparse matrices
over all Sz = 0 determinants of 2k electrons in n spatial orbitals:

  E_pq = sum_sigma a+_{p sigma} a_{q sigma}                       (singlet excitation op.)
  H    = sum_pq h_pq E_pq + 1/2 sum_pqrs g_pqrs (E_pq E_rs - d_qr E_ps)

The cluster operator is X = sum t_ai E_ai + 1/2 sum x_aibj E_ai E_bj (x symmetric under
(ai) <-> (bj)), and exp(+-X) is applied to vectors by its (finite) power series. The
projected equations of Sec. 2.1 are evaluated literally:

  singles rows    <mu1| exp(-X) H exp(X) |HF>
  CC2 rows        <mu2| H~ + [F, X2] |HF>,   H~ = exp(-X1) H exp(X1), F the MO Fock operator
  CCSD rows       <mu2| exp(-T2) H~ exp(T2) |HF>  with T2 the CCSD-active part of X2

A projection <mu~| is read off as the coefficient of the vector in the (non-orthogonal)
basis {E_ai |HF>} or {E_ai E_bj |HF>, ai <= bj} of its excitation level (least squares
on that level), which is the biorthonormal projection. Doubles coefficients are returned
in the symmetric convention (coefficient of 1/2 sum_{aibj} Omega_aibj E_ai E_bj |HF>).
"""
from itertools import combinations
from math import comb

import numpy as np
import scipy.sparse as sp


class DeterminantSpace:
    def __init__(self, n, k):
        self.n, self.k = n, k
        self.strings = [sum(1 << p for p in c) for c in combinations(range(n), k)]
        self.index = {s: i for i, s in enumerate(self.strings)}
        self.ns = len(self.strings)
        assert self.ns == comb(n, k)
        self.dim = self.ns * self.ns
        self._e1 = {}
        self._E = {}

    def _string_op(self, p, q):
        """a+_p a_q on one spin's strings, as a sparse ns x ns matrix with fermion signs."""
        key = (p, q)
        if key in self._e1:
            return self._e1[key]
        rows, cols, vals = [], [], []
        for j, s in enumerate(self.strings):
            if not (s >> q) & 1:
                continue
            sign = (-1) ** bin(s & ((1 << q) - 1)).count("1")
            s1 = s & ~(1 << q)
            if (s1 >> p) & 1:
                continue
            sign *= (-1) ** bin(s1 & ((1 << p) - 1)).count("1")
            s2 = s1 | (1 << p)
            rows.append(self.index[s2])
            cols.append(j)
            vals.append(float(sign))
        m = sp.csr_matrix((vals, (rows, cols)), shape=(self.ns, self.ns))
        self._e1[key] = m
        return m

    def E(self, p, q):
        """Singlet excitation operator E_pq on the product (alpha string, beta string) space."""
        key = (p, q)
        if key not in self._E:
            e = self._string_op(p, q)
            I = sp.identity(self.ns, format="csr")
            self._E[key] = (sp.kron(e, I) + sp.kron(I, e)).tocsr()
        return self._E[key]

    def hf(self):
        v = np.zeros(self.dim)
        s0 = self.index[(1 << self.k) - 1]
        v[s0 * self.ns + s0] = 1.0
        return v

    def one_body(self, M):
        n = self.n
        op = sp.csr_matrix((self.dim, self.dim))
        for p in range(n):
            for q in range(n):
                if M[p, q] != 0.0:
                    op = op + M[p, q] * self.E(p, q)
        return op.tocsr()

    def hamiltonian(self, h, L):
        """H from the one-electron matrix and Cholesky vectors, g_pqrs = sum_J L^J_pq L^J_rs."""
        g_contr = np.einsum("Jpq,Jqs->ps", L, L)           # sum_q g_pqqs
        H = self.one_body(h - 0.5 * g_contr)
        for J in range(L.shape[0]):
            LJ = self.one_body(L[J])
            H = H + 0.5 * (LJ @ LJ)
        return H.tocsr()


def _exp_apply(op, v, sign=1.0, max_terms=64):
    out = v.copy()
    term = v.copy()
    for m in range(1, max_terms):
        term = sign * (op @ term) / m
        if not np.any(term):
            return out
        out = out + term
    raise RuntimeError("excitation series did not terminate")


class BruteForceCC:
    """Closed-shell CC on a small model system; occupied orbitals are 0 .. k-1."""

    def __init__(self, h, L, fock, n_occ, level):
        self.n = h.shape[0]
        self.k = n_occ
        self.nv = self.n - n_occ
        self.ds = DeterminantSpace(self.n, n_occ)
        self.H = self.ds.hamiltonian(h, L)
        self.Fop = self.ds.one_body(fock)
        self.hf = self.ds.hf()
        self.e_hf = float(self.hf @ (self.H @ self.hf))
        level = np.asarray(level)
        no = n_occ
        self.os = np.nonzero(level[:no] >= 1)[0]
        self.vs = np.nonzero(level[no:] >= 1)[0]
        # CCSD-active flags of the CC2-active orbitals, in the order of os / vs
        self.mo_T = level[:no][self.os] == 2
        self.mv_T = level[no:][self.vs] == 2
        self.Eai = {(a, i): self.ds.E(no + a, i) for a in range(self.nv) for i in range(no)}
        pairs = [(a, i) for a in range(self.nv) for i in range(no)]
        self.pairs = pairs
        self.sing_basis = np.stack([self.Eai[p] @ self.hf for p in pairs], axis=1)
        dpairs = [(p, q) for x, p in enumerate(pairs) for y, q in enumerate(pairs) if x <= y]
        self.dpairs = dpairs
        self.doub_basis = np.stack([self.Eai[p] @ (self.Eai[q] @ self.hf) for p, q in dpairs], axis=1)
        self._doub_pinv = np.linalg.pinv(self.doub_basis)

    # operators ----------------------------------------------------------------------
    def X1(self, t1):
        op = sp.csr_matrix((self.ds.dim, self.ds.dim))
        for (a, i), E in self.Eai.items():
            if t1[a, i] != 0.0:
                op = op + t1[a, i] * E
        return op

    def X2_apply(self, x2full, v):
        """(1/2 sum_aibj x_aibj E_ai E_bj) v for a full [nv, no, nv, no] symmetric array."""
        out = np.zeros_like(v)
        for (a, i), Ea in self.Eai.items():
            w = np.zeros_like(v)
            for (b, j), Eb in self.Eai.items():
                c = x2full[a, i, b, j]
                if c != 0.0:
                    w = w + c * (Eb @ v)
            if np.any(w):
                out = out + Ea @ w
        return 0.5 * out

    def embed(self, x2_active, which="all"):
        """Place active-space doubles [sv, so, sv, so] into the full [nv, no, nv, no] array.
        which: 'all', 'T' (all four indices CCSD-active) or 'S' (the rest)."""
        full = np.zeros((self.nv, self.k, self.nv, self.k))
        ix = np.ix_(self.vs, self.os, self.vs, self.os)
        x = x2_active.copy()
        if which != "all":
            mT = self.mask_T()
            x = np.where(mT if which == "T" else ~mT, x, 0.0)
        full[ix] = x
        return full

    def mask_T(self):
        mo, mv = self.mo_T, self.mv_T
        return (mv[:, None, None, None] & mo[None, :, None, None]
                & mv[None, None, :, None] & mo[None, None, None, :])

    def _series(self, apply, v, sign=1.0, max_terms=32):
        out = v.copy()
        term = v.copy()
        for m in range(1, max_terms):
            term = sign * apply(term) / m
            if not np.any(term):
                return out
            out = out + term
        raise RuntimeError("series did not terminate")

    # projections ----------------------------------------------------------------------
    def project_singles(self, v):
        c = (self.sing_basis.T @ v) / 2.0
        return c.reshape(self.nv, self.k)

    def project_doubles(self, v):
        c = self._doub_pinv @ v
        out = np.zeros((self.nv, self.k, self.nv, self.k))
        for (p, q), val in zip(self.dpairs, c):
            if p == q:
                out[p[0], p[1], p[0], p[1]] = 2.0 * val
            else:
                out[p[0], p[1], q[0], q[1]] = val
                out[q[0], q[1], p[0], p[1]] = val
        return out

    # equations ----------------------------------------------------------------------
    def residual(self, t1, x2_active):
        """(Omega_1 [nv, no], Omega_2 on the CC2-active box, energy) for the three-level model."""
        X1 = self.X1(t1)
        Ht = lambda v: _exp_apply(X1, self.H @ _exp_apply(X1, v, 1.0), -1.0)
        x_all = self.embed(x2_active, "all")
        x_T = self.embed(x2_active, "T")
        apply_all = lambda v: self.X2_apply(x_all, v)
        apply_T = lambda v: self.X2_apply(x_T, v)
        # singles and energy: exp(-X) H exp(X) with X = X1 + X2
        w_all = self._series(apply_all, Ht(self._series(apply_all, self.hf, 1.0)), -1.0)
        om1 = self.project_singles(w_all)
        e = float(self.hf @ w_all)
        # CC2 rows: H~ + [F, X2]
        x2hf = apply_all(self.hf)
        fcomm = self.Fop @ x2hf - apply_all(self.Fop @ self.hf)
        om2_cc2 = self.project_doubles(Ht(self.hf) + fcomm)
        # CCSD rows: exp(-T2) H~ exp(T2)
        w_T = self._series(apply_T, Ht(self._series(apply_T, self.hf, 1.0)), -1.0)
        om2_ccsd = self.project_doubles(w_T)
        ix = np.ix_(self.vs, self.os, self.vs, self.os)
        a2, b2 = om2_cc2[ix], om2_ccsd[ix]
        om2 = np.where(self.mask_T(), b2, a2)
        return om1, om2, e - self.e_hf

    def fci(self):
        """All eigenvalues and eigenvectors of H in the determinant space (every spin state)."""
        return np.linalg.eigh(self.H.toarray())

    def singlet_fci(self, n_states=6):
        """Lowest FCI energies of singlet states, selected by <S^2> = 0."""
        w, v = self.fci()
        S2 = self.s_squared()
        out = []
        for k in range(len(w)):
            if abs(v[:, k] @ (S2 @ v[:, k])) < 1e-6:
                out.append(w[k])
            if len(out) >= n_states:
                break
        return np.array(out)

    def s_squared(self):
        """S^2 = S_- S_+ on the Sz = 0 space, S_+ = sum_p a+_{p alpha} a_{p beta}.

        Determinants are a+(alpha string) a+(beta string) |vac>, so a beta operator
        passes the k alpha creators (sign (-1)^k) before acting on the beta string.
        """
        n, k, ns = self.n, self.k, self.ds.ns
        strings, index = self.ds.strings, self.ds.index
        below = lambda s, p: bin(s & ((1 << p) - 1)).count("1")
        rows, cols, vals = [], [], []
        for ia, sa in enumerate(strings):
            for ib, sb in enumerate(strings):
                for p in range(n):
                    if not (sb >> p) & 1 or (sa >> p) & 1:
                        continue
                    sgn1 = (-1) ** (k + below(sb, p)) * (-1) ** below(sa, p)
                    sa1, sb1 = sa | (1 << p), sb & ~(1 << p)
                    for q in range(n):
                        if not (sa1 >> q) & 1 or (sb1 >> q) & 1:
                            continue
                        sgn2 = (-1) ** below(sa1, q) * (-1) ** (k + below(sb1, q))
                        sa2, sb2 = sa1 & ~(1 << q), sb1 | (1 << q)
                        rows.append(index[sa2] * ns + index[sb2])
                        cols.append(ia * ns + ib)
                        vals.append(float(sgn1 * sgn2))
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.ds.dim, self.ds.dim))

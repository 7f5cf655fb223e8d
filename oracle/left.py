"""Left eigenvectors of the MLCC Jacobian (test infrastructure: only tests/ may use this
module).

The excitation energies are eigenvalues of the non-symmetric Jacobian A = dOmega/dx
(Sec. 2.1); transition moments, which the paper names as a motivation (Sec. 1), need the
left eigenvectors as well: l^T A = omega l^T. The amplitudes here are the singles and the
doubles stored symmetric in full, and the inner product is the plain Euclidean one on that
storage (an off-diagonal doubles pair counts twice, a diagonal one once), as in the
Davidson solvers. The left transformation is the adjoint of A in that inner product on the
symmetric vectors:
    <rho(l), c> = <l, A c>   for every admissible c.
It is built here densely from A itself (columns from sigma on the independent parameters,
as in the pins of the Davidson solver), for small systems:
    A_P (packed values -> packed values),  W = the weights of the inner product,
    rho_P = W^-1 A_P^T W l_P.
"""
import numpy as np
import scipy.linalg as sla

from .mlcc import sigma


def packed_pairs(sys):
    sh = sys.doubles_shape()
    return [(a, i, b, j) for a in range(sh[0]) for i in range(sh[1]) for b in range(sh[2])
            for j in range(sh[3]) if a * sh[1] + i <= b * sh[3] + j]


def dense(sys, gs):
    """(A_P, W, pairs): A over the independent parameters (singles, doubles ai <= bj) and the
    diagonal weights of the full-storage inner product in those parameters."""
    nv, no = sys.nv, sys.no
    sh = sys.doubles_shape()
    n1 = nv * no
    pk = packed_pairs(sys)
    cols = []
    for m in range(n1):
        e1 = np.zeros(n1)
        e1[m] = 1.0
        s1, s2 = sigma(sys, gs.t1, gs.x2, e1.reshape(nv, no), np.zeros(sh))
        cols.append(np.concatenate([s1.ravel(), [s2[p] for p in pk]]))
    for (a, i, b, j) in pk:
        e2 = np.zeros(sh)
        e2[a, i, b, j] = e2[b, j, a, i] = 1.0
        s1, s2 = sigma(sys, gs.t1, gs.x2, np.zeros((nv, no)), e2)
        cols.append(np.concatenate([s1.ravel(), [s2[p] for p in pk]]))
    so = sh[1]
    w = np.concatenate([np.ones(n1), [1.0 if a * so + i == b * so + j else 2.0 for (a, i, b, j) in pk]])
    return np.array(cols).T, w, pk


def to_packed(sys, c1, c2, pk):
    return np.concatenate([np.asarray(c1).ravel(), [c2[p] for p in pk]])


def from_packed(sys, v, pk):
    nv, no = sys.nv, sys.no
    n1 = nv * no
    c2 = np.zeros(sys.doubles_shape())
    for val, (a, i, b, j) in zip(v[n1:], pk):
        c2[a, i, b, j] = c2[b, j, a, i] = val
    return v[:n1].reshape(nv, no), c2


def left_transform(sys, gs, l1, l2, dense_parts=None):
    """rho(l) = the adjoint of A applied to the symmetric vector (l1, l2)."""
    A, w, pk = dense_parts or dense(sys, gs)
    lp = to_packed(sys, l1, l2, pk)
    rp = (A.T @ (w * lp)) / w
    return from_packed(sys, rp, pk)


def left_eigenpairs(sys, gs, n_roots, dense_parts=None):
    """(omega, left vectors [n_roots] as (l1, l2), right vectors likewise) of the lowest
    real roots, from the dense problem; left and right scaled so that <l_k, r_k> = 1 and r_k
    has unit norm."""
    A, w, pk = dense_parts or dense(sys, gs)
    wr, vl, vr = sla.eig(A, left=True, right=True)
    order = [k for k in np.argsort(wr.real) if abs(wr[k].imag) < 1e-9][:n_roots]
    omega = wr.real[order]
    lefts, rights = [], []
    for k in order:
        r = vr[:, k].real
        # the eigenvector of A_P^T is W l_P: l_P = W^-1 (left eigenvector of A_P)
        lp = vl[:, k].real / w
        rn = np.sqrt(np.sum(w * r * r))
        r = r / rn
        lp = lp / np.sum(w * lp * r)
        rights.append(from_packed(sys, r, pk))
        lefts.append(from_packed(sys, lp, pk))
    return omega, lefts, rights

"""Davidson solver for the lowest right eigenpairs of the non-symmetric CC Jacobian.

TEST INFRASTRUCTURE ONLY. The paper obtains excitation energies as eigenvalues of the
Jacobian (Sec. 2.1) to a residual threshold (Sec. 3) and does not name the eigensolver;
this is the standard non-symmetric Davidson iteration:

  1. start from 2 n_roots unit singles with the lowest eps_a - eps_i;
  2. Rayleigh-Ritz: G = B^T A B, eigenpairs of G (dense, FP64), lowest n_roots by Re w;
  3. residuals r_k = A B y_k - w_k B y_k, converged when |r_k| < res_tol and the Ritz value
     moved less than w_tol;
  4. new directions (eps_mu - w_k)^-1 r_k (guarded where |eps_mu - w_k| < 1e-8),
     orthonormalised against the basis by two passes of Gram-Schmidt;
  5. when the basis would exceed max_sub vectors it collapses onto 2 n_roots Ritz vectors.

Vectors are flat arrays (singles then the symmetric doubles array); the inner product is
the plain Euclidean one on that storage.
"""
import numpy as np
import scipy.linalg as sla


class DavidsonResult:
    def __init__(self, omega, vectors, residuals, iterations, converged, complex_pair, n_sigma):
        self.omega, self.vectors, self.residuals = omega, vectors, residuals
        self.iterations, self.converged, self.complex_pair = iterations, converged, complex_pair
        self.n_sigma = n_sigma


def _orthonormalise_against(B, v, drop_tol=1e-10):
    nrm0 = np.linalg.norm(v)
    if nrm0 == 0.0:
        return None
    for _ in range(2):
        if B.shape[1]:
            v = v - B @ (B.T @ v)
    nrm = np.linalg.norm(v)
    if nrm < drop_tol * nrm0:
        return None
    return v / nrm


def davidson(apply_A, diag, n_roots, guess, res_tol=1e-8, w_tol=1e-11, max_iter=300,
             max_sub=None, collapse=None, project=None, verbose=False):
    """apply_A(V[:, m]) -> A V[:, m]; diag = eps_mu preconditioner; guess: [dim, m0].

    project(v) maps a vector onto the space of admissible amplitudes (here: doubles
    symmetric under (ai) <-> (bj)); new directions are projected before they enter the
    basis so that rounding noise cannot open up the unphysical complement, whose
    eigenvalues are not excitation energies.
    """
    project = project or (lambda v: v)
    dim = diag.size
    max_sub = max_sub or max(8 * n_roots, 2 * n_roots + 4)
    collapse = collapse or 2 * n_roots
    B = np.zeros((dim, 0))
    for k in range(guess.shape[1]):
        v = _orthonormalise_against(B, guess[:, k].astype(np.float64))
        if v is not None:
            B = np.column_stack([B, v])
    S = apply_A(B)
    n_sigma = B.shape[1]
    w_old = np.full(n_roots, np.inf)
    complex_pair = False
    for it in range(1, max_iter + 1):
        G = B.T @ S
        w, Y = sla.eig(G)
        order = np.argsort(w.real, kind="stable")
        w, Y = w[order], Y[:, order]
        wk = w[:n_roots]
        complex_pair = bool(np.any(np.abs(wk.imag) > 1e-10 * np.maximum(1.0, np.abs(wk.real))))
        Yk = Y[:, :n_roots].real
        X = B @ Yk
        nx = np.linalg.norm(X, axis=0)
        X /= nx
        Yk = Yk / nx
        R = S @ Yk - X * wk.real
        rn = np.linalg.norm(R, axis=0)
        dw = np.abs(wk.real - w_old)
        w_old = wk.real.copy()
        done = (rn < res_tol) & (dw < w_tol)
        if verbose:
            print(f"Davidson it {it:3d} dim {B.shape[1]:3d} w {wk.real} |r| {rn}")
        if np.all(done):
            idx = np.argmax(np.abs(X), axis=0)
            X = X * np.sign(X[idx, np.arange(n_roots)])
            return DavidsonResult(wk.real, X, rn, it, True, complex_pair, n_sigma)
        new = []
        for k in np.nonzero(~done)[0]:
            den = wk[k].real - diag
            den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den + 0.0), den)
            new.append(project(R[:, k] / den))
        if B.shape[1] + len(new) > max_sub:
            Yc = Y[:, :collapse].real
            Bc = B @ Yc
            Sc = S @ Yc
            # re-orthonormalise the collapsed basis with the same transformation on S
            Q, Rq = np.linalg.qr(Bc)
            Rinv = np.linalg.inv(Rq)
            B, S = Q, Sc @ Rinv
        added = []
        for v in new:
            v = _orthonormalise_against(np.column_stack([B] + added) if added else B, v)
            if v is not None:
                added.append(v[:, None])
        if not added:
            # the basis spans an invariant subspace: the Ritz pairs are exact
            idx = np.argmax(np.abs(X), axis=0)
            X = X * np.sign(X[idx, np.arange(n_roots)])
            return DavidsonResult(wk.real, X, rn, it, bool(np.all(rn < res_tol)),
                                  complex_pair, n_sigma)
        Bn = np.column_stack(added)
        Sn = apply_A(Bn)
        n_sigma += Bn.shape[1]
        B = np.column_stack([B, Bn])
        S = np.column_stack([S, Sn])
    idx = np.argmax(np.abs(X), axis=0)
    X = X * np.sign(X[idx, np.arange(n_roots)])
    return DavidsonResult(wk.real, X, rn, it, False, complex_pair, n_sigma)


def excited_states(sys, gs, n_roots, sigma_fn=None, **kw):
    """Lowest n_roots excitation energies of the MLCC Jacobian at the ground state gs."""
    from .mlcc import sigma as sigma_def
    sigma_fn = sigma_fn or sigma_def
    nv, no = sys.nv, sys.no
    n1 = nv * no
    dshape = sys.doubles_shape()

    def apply_A(V):
        out = np.empty_like(V)
        for k in range(V.shape[1]):
            c1 = V[:n1, k].reshape(nv, no)
            c2 = V[n1:, k].reshape(dshape)
            s1, s2 = sigma_fn(sys, gs.t1, gs.x2, c1, c2)
            out[:n1, k] = s1.ravel()
            out[n1:, k] = s2.ravel()
        return out

    def project(v):
        d = v[n1:].reshape(dshape)
        return np.concatenate([v[:n1], (0.5 * (d + d.transpose(2, 3, 0, 1))).ravel()])

    kw.setdefault("project", project)
    diag = np.concatenate([sys.eps_ai.ravel(), sys.eps_aibj.ravel()])
    n_guess = min(2 * n_roots, n1)
    order = np.argsort(sys.eps_ai.ravel(), kind="stable")[:n_guess]
    guess = np.zeros((diag.size, n_guess))
    guess[order, np.arange(n_guess)] = 1.0
    return davidson(apply_A, diag, n_roots, guess, **kw)

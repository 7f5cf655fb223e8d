"""Folded CC2 effective Jacobian (test infrastructure: only tests/ may use this module).

For CC2 the paper points to the strategies of CC2 response theory (Sec. 2.1), where the
doubles are folded into an energy-dependent effective Jacobian. In the three-level model
(rows with all four indices CCSD-active, P_T, obey the CCSD equation built from P_T
amplitudes; the other CC2-active rows, P_S, obey g~ + eps x = 0) the Jacobian blocks on
P_S are
    A_SS = diag(eps_aibj),   A_ST = 0,   A_TS = 0,
so an eigenpair (omega, c) of A has c_S = (omega - eps_S)^-1 A_S1 c1, and (c1, c_T) is an
eigenvector with eigenvalue omega of
    A_eff(omega) = [[A_11 + A_1S (omega - eps_S)^-1 A_S1, A_1T],
                    [A_T1,                                A_TT]].
sigma_eff applies A_eff(omega) with two evaluations of the oracle's sigma (the definition
A = dOmega/dx): one with c2 = 0, whose P_S rows are A_S1 c1, and one with
c2 = c_S(omega) + c_T, whose singles and P_T rows are the result.

excited_states_folded_iterative does it by iteration for larger systems whose roots lie
well below the P_S denominators. On the 48-orbital workload it needs about 4x the
sigma-vector count of the unfolded Davidson (each sigma_eff is two sigma evaluations here),
so a production solver has to reuse its subspace across omega updates.

excited_states_folded_linearised keeps its subspaces across omega updates: each trial
vector b stores A_eff(w_b) b and dA_eff/domega (w_b) b = -A_1S (w_b - eps_S)^-2 A_S1 b1 at
the omega w_b it was applied at, and the projected problem at omega uses the first-order
model A_eff(omega) b ~ A_eff(w_b) b + (omega - w_b) dA_eff/domega b. Stage 1 finds all roots
roughly with every vector applied at one omega; stage 2 refines each root in a subspace of
its own, restarting from the Ritz vector applied exactly at the current omega until the
model is exact at convergence. On the 48-orbital workload it needs fewer applications than
the plain fixed point above.

excited_states_folded solves the nonlinear problem on small systems: its roots below the
lowest P_S denominator are the zeros of det(A_eff(omega) - omega), with A_eff assembled
from sigma applications (fold_parts). A plain fixed-point iteration omega <- lambda_k(omega)
need not converge when the coupling to the doubles is strong (roots near the poles).
"""
import numpy as np

from .mlcc import sigma as sigma_def


def sigma_eff(sys, gs, c1, cT, omega, sigma_fn=None):
    """A_eff(omega) (c1, c_T). cT is a doubles array of which only the P_T entries are
    used; the result is (s1, s2) with s2 zero outside P_T."""
    sigma_fn = sigma_fn or sigma_def
    zero = np.zeros(sys.doubles_shape())
    _, r2 = sigma_fn(sys, gs.t1, gs.x2, c1, zero)          # P_S rows: A_S1 c1
    cS = np.where(sys.mask_S, r2 / (omega - sys.eps_aibj), 0.0)
    c2 = np.where(sys.mask_T, cT, cS)
    s1, s2 = sigma_fn(sys, gs.t1, gs.x2, c1, c2)
    return s1, np.where(sys.mask_T, s2, 0.0)


def unfold(sys, gs, c1, cT, omega, sigma_fn=None):
    """The full doubles vector of a folded vector: c_S(omega) on P_S, c_T on P_T."""
    sigma_fn = sigma_fn or sigma_def
    _, r2 = sigma_fn(sys, gs.t1, gs.x2, c1, np.zeros(sys.doubles_shape()))
    cS = np.where(sys.mask_S, r2 / (omega - sys.eps_aibj), 0.0)
    return np.where(sys.mask_T, cT, cS)


def packed_T(sys):
    """Independent P_T parameters: (a, i, b, j) with (ai) <= (bj), all four CCSD-active."""
    sv, so = sys.sv, sys.so
    return [(a, i, b, j) for a in range(sv) for i in range(so) for b in range(sv) for j in range(so)
            if sys.mask_T[a, i, b, j] and a * so + i <= b * so + j]


def folded_matrix(sys, gs, omega, sigma_fn=None):
    """Dense A_eff(omega) over (singles, packed P_T), column by column."""
    nv, no = sys.nv, sys.no
    sh = sys.doubles_shape()
    n1 = nv * no
    pk = packed_T(sys)
    cols = []
    for m in range(n1 + len(pk)):
        c1 = np.zeros(n1)
        cT = np.zeros(sh)
        if m < n1:
            c1[m] = 1.0
        else:
            a, i, b, j = pk[m - n1]
            cT[a, i, b, j] = cT[b, j, a, i] = 1.0
        s1, s2 = sigma_eff(sys, gs, c1.reshape(nv, no), cT, omega, sigma_fn)
        cols.append(np.concatenate([s1.ravel(), [s2[p] for p in pk]]))
    return np.array(cols).T


def fold_parts(sys, gs, sigma_fn=None):
    """The omega-independent pieces of A_eff, from sigma applications to unit vectors:
    P = [[A_11, A_1T], [A_T1, A_TT]] over (singles, packed P_T); U = A_1S and V = A_S1
    over the packed P_S pairs; d = eps on those pairs. A_eff(omega) = P + the singles
    block U diag(1 / (omega - d)) V."""
    sigma_fn = sigma_fn or sigma_def
    nv, no = sys.nv, sys.no
    n1 = nv * no
    sh = sys.doubles_shape()
    so = sh[1]
    pk_all = [(a, i, b, j) for a in range(sh[0]) for i in range(so) for b in range(sh[2]) for j in range(so)
              if a * so + i <= b * so + j]
    pT = [q for q in pk_all if sys.mask_T[q]]
    pS = [q for q in pk_all if not sys.mask_T[q]]
    zero1, zero2 = np.zeros((nv, no)), np.zeros(sh)
    P = np.zeros((n1 + len(pT), n1 + len(pT)))
    V = np.zeros((len(pS), n1))
    U = np.zeros((n1, len(pS)))
    for m in range(n1):
        e1 = np.zeros(n1)
        e1[m] = 1.0
        s1, s2 = sigma_fn(sys, gs.t1, gs.x2, e1.reshape(nv, no), zero2)
        P[:n1, m] = s1.ravel()
        P[n1:, m] = [s2[q] for q in pT]
        V[:, m] = [s2[q] for q in pS]
    for col, q in enumerate(pT + pS):
        e2 = np.zeros(sh)
        e2[q] = e2[q[2], q[3], q[0], q[1]] = 1.0
        s1, s2 = sigma_fn(sys, gs.t1, gs.x2, zero1, e2)
        if col < len(pT):
            P[:n1, n1 + col] = s1.ravel()
            P[n1:, n1 + col] = [s2[r] for r in pT]
        else:
            U[:, col - len(pT)] = s1.ravel()
    d = np.array([sys.eps_aibj[q] for q in pS])
    return P, U, V, d


def excited_states_folded(sys, gs, n_roots, sigma_fn=None, grid=4000):
    """Lowest solutions omega of A_eff(omega) c = omega c with 0 < omega < min(eps_S), the
    regime below the doubles denominators that the fold is for (at most n_roots, ascending).
    They are the zeros of det(A_eff(omega) - omega): located by sign changes on a grid and
    refined by bisection. Without P_S pairs A_eff is the plain Jacobian."""
    P, U, V, d = fold_parts(sys, gs, sigma_fn)
    n1 = U.shape[0]
    if d.size == 0:
        w = np.linalg.eigvals(P)
        w = np.sort(w.real[np.abs(w.imag) < 1e-9])
        return w[w > 0][:n_roots]

    def f(w):
        M = P.copy()
        M[:n1, :n1] += (U / (w - d)) @ V
        sign, logdet = np.linalg.slogdet(M - w * np.eye(M.shape[0]))
        return sign

    hi = d.min() * (1.0 - 1e-9)
    xs = np.linspace(0.0, hi, grid)
    fs = [f(x) for x in xs]
    roots = []
    for x0, x1, f0, f1 in zip(xs[:-1], xs[1:], fs[:-1], fs[1:]):
        if f0 == 0.0:
            roots.append(x0)
        elif f0 != f1:
            a, b, fa = x0, x1, f0
            for _ in range(200):
                m = 0.5 * (a + b)
                fm = f(m)
                if fm == fa:
                    a, fa = m, fm
                else:
                    b = m
                if b - a < 1e-15 * max(1.0, abs(m)):
                    break
            roots.append(0.5 * (a + b))
        if len(roots) >= n_roots:
            break
    return np.array(roots)


def excited_states_folded_iterative(sys, gs, n_roots, tol=1e-10, res_tol=1e-9, max_macro=40, sigma_fn=None):
    """The folded problem by iteration, for systems whose roots lie well below the P_S
    denominators (then lambda_k(omega) depends weakly on omega):
      1. a linear Davidson for the n_roots lowest eigenpairs of A_eff(omega_0), omega_0 = 0;
      2. per root k, the fixed point omega <- lambda_k(omega), where lambda_k is the k-th
         lowest eigenvalue of A_eff(omega) from a linear Davidson warm-started on the
         previous eigenvectors.
    Vectors are (singles, doubles) with the doubles restricted to P_T. Returns
    (roots ascending, number of sigma_eff applications)."""
    from .davidson import davidson
    nv, no = sys.nv, sys.no
    n1 = nv * no
    sh = sys.doubles_shape()
    maskT = sys.mask_T.ravel()
    count = [0]

    def apply_eff(omega):
        def apply(V):
            out = np.zeros_like(V)
            for k in range(V.shape[1]):
                c1 = V[:n1, k].reshape(nv, no)
                cT = V[n1:, k].reshape(sh)
                s1, s2 = sigma_eff(sys, gs, c1, cT, omega, sigma_fn)
                out[:n1, k] = s1.ravel()
                out[n1:, k] = s2.ravel()
                count[0] += 1
            return out
        return apply

    def project(v):
        d = np.where(maskT, v[n1:], 0.0).reshape(sh)
        return np.concatenate([v[:n1], (0.5 * (d + d.transpose(2, 3, 0, 1))).ravel()])

    # outside P_T the preconditioner denominator is huge: those components stay zero
    diag = np.concatenate([sys.eps_ai.ravel(), np.where(maskT, sys.eps_aibj.ravel(), 1e30)])
    n_guess = min(2 * n_roots, n1)
    order = np.argsort(sys.eps_ai.ravel(), kind="stable")[:n_guess]
    guess = np.zeros((diag.size, n_guess))
    guess[order, np.arange(n_guess)] = 1.0
    first = davidson(apply_eff(0.0), diag, n_roots, guess, res_tol=1e-6, w_tol=1e-8, project=project)
    roots = []
    for k in range(n_roots):
        omega, X = first.omega[k], first.vectors[:, :k + 1]
        for _ in range(max_macro):
            r = davidson(apply_eff(omega), diag, k + 1, X, res_tol=res_tol, w_tol=tol, project=project)
            lam, X = r.omega[k], r.vectors
            done = abs(lam - omega) < tol
            omega = lam
            if done:
                break
        else:
            raise RuntimeError(f"folded root {k}: no fixed point in {max_macro} iterations")
        roots.append(omega)
    return np.sort(np.array(roots)), count[0]


def sigma_eff_domega(sys, gs, c1, omega, sigma_fn=None):
    """dA_eff/domega (c1, c_T) = (-A_1S (omega - eps_S)^-2 A_S1 c1, 0): only the singles
    block of A_eff depends on omega. A_S1 c1 are the P_S rows of sigma(c1, 0); A_1S x_S are
    the singles of sigma(0, x_S)."""
    sigma_fn = sigma_fn or sigma_def
    zero1, zero2 = np.zeros_like(c1), np.zeros(sys.doubles_shape())
    _, r2 = sigma_fn(sys, gs.t1, gs.x2, c1, zero2)
    xS = np.where(sys.mask_S, -r2 / (omega - sys.eps_aibj) ** 2, 0.0)
    d1, _ = sigma_fn(sys, gs.t1, gs.x2, zero1, xS)
    return d1


def excited_states_folded_linearised(sys, gs, n_roots, res_tol=1e-9, max_iter=100, stage1_tol=1e-3,
                                     exact_dw=1e-7, sigma_fn=None):
    """Lowest n_roots solutions of A_eff(omega) c = omega c below the P_S denominators, with
    subspaces kept across omega updates (first-order model in omega per trial vector):

    stage 1 (all roots): trial vectors applied at one omega_0 (the lowest eps_ai); for each
      root the k-th eigenvalue of the projected model V^T (S0 + (omega - omega_0) S1) is
      made self-consistent in omega; new directions are the preconditioned residuals
      (eps_mu - omega_k)^-1 r_k; stop when every model residual is below stage1_tol;
    stage 2 (each root k): a subspace of its own, started from the stage-1 Ritz vector
      applied at omega_k; each step takes the Ritz pair of the projected model (vector b
      applied at w_b contributes S0_b + (omega - w_b) S1_b) that overlaps most with the
      previous one, made self-consistent in omega, and adds its preconditioned residual
      applied at the current omega. When the model residual is below res_tol the root is
      done if every vector of the subspace was applied within exact_dw of omega (the model
      error is second order in omega - w_b); otherwise the subspace restarts from the Ritz
      vector applied exactly at omega.

    Returns (roots ascending, number of A_eff applications)."""
    nv, no = sys.nv, sys.no
    n1 = nv * no
    sh = sys.doubles_shape()
    maskT = sys.mask_T.ravel()
    count = [0]

    def project(v):
        d = np.where(maskT, v[n1:], 0.0).reshape(sh)
        return np.concatenate([v[:n1], (0.5 * (d + d.transpose(2, 3, 0, 1))).ravel()])

    def apply(w, v):
        c1 = v[:n1].reshape(nv, no)
        cT = v[n1:].reshape(sh)
        s1, s2 = sigma_eff(sys, gs, c1, cT, w, sigma_fn)
        d1 = sigma_eff_domega(sys, gs, c1, w, sigma_fn)
        count[0] += 1
        return (np.concatenate([s1.ravel(), s2.ravel()]),
                np.concatenate([d1.ravel(), np.zeros(v.size - n1)]))

    def orth(V, v):
        for _ in range(2):
            if V.shape[1]:
                v = v - V @ (V.T @ v)
        return v

    diag = np.concatenate([sys.eps_ai.ravel(), np.where(maskT, sys.eps_aibj.ravel(), 1e30)])

    def precondition(r, w):
        den = diag - w
        return project(r / np.where(np.abs(den) < 1e-8, 1e-8, den))

    def model_pair(V, S0, S1, wv, w, pick):
        """Self-consistent (omega, y) of the projected first-order model; pick(lam, Y)
        chooses the Ritz pair."""
        G0, G1 = V.T @ S0, V.T @ S1
        for _ in range(100):
            lam, Y = np.linalg.eig(G0 + G1 * (w - wv)[None, :])
            j = pick(lam, Y)
            if abs(lam[j].real - w) < 1e-14 * max(1.0, abs(w)):
                break
            w = lam[j].real
        y = Y[:, j].real
        y = y / np.linalg.norm(y)
        x = V @ y
        r = S0 @ y + S1 @ ((w - wv) * y) - w * x
        return w, y, x, r

    # stage 1
    n_guess = min(2 * n_roots, n1)
    order = np.argsort(sys.eps_ai.ravel(), kind="stable")[:n_guess]
    w0 = float(sys.eps_ai.ravel()[order[0]])
    V = np.zeros((diag.size, n_guess))
    V[order, np.arange(n_guess)] = 1.0
    cols = [apply(w0, V[:, i]) for i in range(n_guess)]
    S0 = np.column_stack([c[0] for c in cols])
    S1 = np.column_stack([c[1] for c in cols])
    om = np.full(n_roots, w0)
    X = [None] * n_roots
    for _ in range(max_iter):
        wv = np.full(V.shape[1], w0)
        R = []
        for k in range(n_roots):
            om[k], _, X[k], r = model_pair(V, S0, S1, wv, om[k],
                                           lambda lam, Y, k=k: int(np.argsort(lam.real)[k]))
            R.append(r)
        if max(np.linalg.norm(r) for r in R) < stage1_tol:
            break
        for k in range(n_roots):
            t = orth(V, precondition(R[k], om[k]))
            nt = np.linalg.norm(t)
            if nt < 1e-10:
                continue
            t /= nt
            a, b = apply(w0, t)
            V, S0, S1 = np.column_stack([V, t]), np.column_stack([S0, a]), np.column_stack([S1, b])
    # stage 2
    roots = []
    for k in range(n_roots):
        w = om[k]

        def restart(x, w):
            x = x / np.linalg.norm(x)
            a, b = apply(w, x)
            return x[:, None], a[:, None], b[:, None], np.array([w]), np.array([1.0])

        V, S0, S1, wv, yprev = restart(X[k], w)
        for _ in range(max_iter):
            def overlap(lam, Y, yprev=yprev):
                Yr = Y.real
                return int(np.argmax(np.abs(Yr[:yprev.size].T @ yprev) / np.linalg.norm(Yr, axis=0)))
            w, y, x, r = model_pair(V, S0, S1, wv, w, overlap)
            if np.linalg.norm(r) < res_tol:
                if np.max(np.abs(w - wv)) < exact_dw:
                    break
                V, S0, S1, wv, yprev = restart(x, w)
                continue
            t = orth(V, precondition(r, w))
            nt = np.linalg.norm(t)
            if nt < 1e-12 or V.shape[1] >= 8 * n_roots:
                V, S0, S1, wv, yprev = restart(x, w)
                continue
            t /= nt
            a, b = apply(w, t)
            V, S0, S1 = np.column_stack([V, t]), np.column_stack([S0, a]), np.column_stack([S1, b])
            wv = np.append(wv, w)
            yprev = np.append(y, 0.0)
        else:
            raise RuntimeError(f"folded root {k}: not converged in {max_iter} iterations")
        roots.append(w)
    return np.sort(np.array(roots)), count[0]

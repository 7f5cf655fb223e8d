"""Small seeded model systems for the oracle pins (test helper, no method arithmetic)."""
import numpy as np

from synth.generator import draw_model_hamiltonian
from synth.rhf import rhf


class Tiny:
    def __init__(self, n, k, n_chol, tau, seed, scale):
        ham = draw_model_hamiltonian(n, n_chol, tau, seed=seed, scale=scale)
        r = rhf(ham.h, ham.L, k, tol=1e-12)
        assert r.converged
        C = r.C
        self.n, self.k = n, k
        self.L = np.matmul(np.matmul(C.T[None], ham.L), C[None])
        F = C.T @ r.fock @ C
        self.F = 0.5 * (F + F.T)
        self.h = C.T @ ham.h @ C
        self.e_hf = r.energy
        self.eps = r.eps


def tiny(n=7, k=2, n_chol=12, tau=6.0, seed=3, scale=0.35):
    return Tiny(n, k, n_chol, tau, seed, scale)


def rotate(sysobj, seed=11):
    """Random orthogonal occ-occ and vir-vir rotation of the MO quantities."""
    rng = np.random.default_rng(seed)
    n, k = sysobj.n, sysobj.k
    U = np.zeros((n, n))
    for lo, hi in ((0, k), (k, n)):
        q, _ = np.linalg.qr(rng.standard_normal((hi - lo, hi - lo)))
        U[lo:hi, lo:hi] = q
    L = np.matmul(np.matmul(U.T[None], sysobj.L), U[None])
    F = U.T @ sysobj.F @ U
    h = U.T @ sysobj.h @ U
    return L, 0.5 * (F + F.T), h

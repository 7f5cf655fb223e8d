"""Seeded model Hamiltonians shaped like the paper's reduced-space workloads.

Recipe (one closed-shell system per seed, orthonormal AO basis):
  * h: diagonal ~ U[-3, 2] Ha, off-diagonal upper triangle (row-major) ~ N(0, 0.05^2),
    mirrored to a symmetric matrix;
  * for J = 0 .. N_J-1 and m <= n (row-major upper triangle):
        L^J_mn = z * exp(-J / tau) * exp(-|m - n| / 6) * scale,   z ~ N(0, 1),
    mirrored, so g_mnrs = sum_J L^J_mn L^J_rs is a positive semidefinite ERI tensor
    with the pq <-> qp and pq <-> rs symmetries of real orbitals;
  * draw order: h diagonal, h off-diagonal, then L one J at a time.
RHF on (h, L) gives canonical orbitals C; the MO inputs of the method are
L^J_MO = C^T L^J C and F = diag(eps) (canonical, hence semicanonical in every block).
Levels (Sec. 2.1, nested active spaces): CCSD-active are the highest t_o occupied and the
lowest t_v virtual orbitals, CC2-active adds the next s_o - t_o occupied and s_v - t_v
virtual orbitals, and every other orbital is CCS (level 0).
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .rhf import rhf

LEVEL_CCS, LEVEL_CC2, LEVEL_CCSD = 0, 1, 2


@dataclass
class ModelHamiltonian:
    h: np.ndarray      # [n, n]
    L: np.ndarray      # [n_chol, n, n]


def draw_model_hamiltonian(n, n_chol, tau, seed, scale=1.0, dist=6.0):
    rng = np.random.default_rng(seed)
    h = np.zeros((n, n))
    h[np.diag_indices(n)] = rng.uniform(-3.0, 2.0, size=n)
    iu1 = np.triu_indices(n, 1)
    off = rng.normal(0.0, 0.05, size=iu1[0].size)
    h[iu1] = off
    h[(iu1[1], iu1[0])] = off
    iu = np.triu_indices(n)
    band = np.array([math.exp(-abs(int(m) - int(q)) / dist) for m, q in zip(*iu)])
    L = np.empty((n_chol, n, n))
    for J in range(n_chol):
        z = rng.standard_normal(iu[0].size)
        v = z * (math.exp(-J / tau) * scale) * band
        LJ = L[J]
        LJ[iu] = v
        LJ[(iu[1], iu[0])] = v
    return ModelHamiltonian(h, L)


@dataclass
class SystemSpec:
    name: str
    n_occ: int
    n_vir: int
    n_chol: int
    tau: float
    s_occ: int         # CC2-active occupied (includes the CCSD-active ones)
    s_vir: int
    t_occ: int         # CCSD-active occupied
    t_vir: int
    n_roots: int
    seed: int = 0
    scale: float = 1.0

    @property
    def n_mo(self):
        return self.n_occ + self.n_vir


def level_map(n_occ, n_vir, s_occ, s_vir, t_occ, t_vir):
    """Per-MO level (0 CCS, 1 CC2, 2 CCSD) for energy-ordered canonical orbitals."""
    assert 0 <= t_occ <= s_occ <= n_occ and 0 <= t_vir <= s_vir <= n_vir
    lev = np.zeros(n_occ + n_vir, dtype=np.int8)
    lev[n_occ - s_occ:n_occ] = LEVEL_CC2
    lev[n_occ - t_occ:n_occ] = LEVEL_CCSD
    lev[n_occ:n_occ + s_vir] = LEVEL_CC2
    lev[n_occ:n_occ + t_vir] = LEVEL_CCSD
    return lev


@dataclass
class MOSystem:
    spec: SystemSpec
    L: np.ndarray          # [n_chol, n_mo, n_mo] MO Cholesky vectors, occupied first
    fock: np.ndarray       # [n_mo, n_mo] MO Fock matrix (diagonal for canonical orbitals)
    eps: np.ndarray        # [n_mo] orbital energies
    e_hf: float            # E_HF = sum_i (h_ii + F_ii) in the MO basis (x2 for spin)
    level: np.ndarray      # [n_mo] int8 levels
    rhf_iterations: int = 0
    rhf_gradient: float = 0.0
    extra: dict = field(default_factory=dict)


def make_system(spec: SystemSpec, rhf_tol=1e-10):
    ham = draw_model_hamiltonian(spec.n_mo, spec.n_chol, spec.tau, spec.seed, spec.scale)
    res = rhf(ham.h, ham.L, spec.n_occ, tol=rhf_tol)
    if not res.converged:
        raise RuntimeError(f"RHF did not converge for {spec.name}: gradient {res.gradient:.3e}")
    C = res.C
    Lmo = np.matmul(np.matmul(C.T[None], ham.L), C[None])
    fock = C.T @ res.fock @ C
    fock = 0.5 * (fock + fock.T)
    lev = level_map(spec.n_occ, spec.n_vir, spec.s_occ, spec.s_vir, spec.t_occ, spec.t_vir)
    return MOSystem(spec, Lmo, fock, res.eps.copy(), res.energy, lev, res.iterations,
                    res.gradient, {"h_mo": C.T @ ham.h @ C})


def default_scale(tau):
    """Uniform rescale of the drawn L^J: 0.5 / sqrt(tau).

    With scale 1 the self-repulsion g_pppp ~ tau / 2 Ha dwarfs the one-electron spread of
    5 Ha: RHF does not converge (small config) or the coupled cluster equations diverge.
    0.5 / sqrt(tau) puts g_pppp near 1/8 Ha for every tau, where RHF converges and the
    CC ground state converges with moderate amplitudes (|t| < 0.2).
    """
    return 0.5 / math.sqrt(tau)


def _spec(name, no, nv, nj, so, sv, to, tv, roots):
    tau = nj / 5.0
    return SystemSpec(name, no, nv, nj, tau, so, sv, to, tv, roots, 0, default_scale(tau))


# Workloads shaped like the paper's (Sec. 3 tables): tau = N_J / 5 (40, 300, 1200, 500).
CONFIGS = {
    # 48 orbitals, 8 occupied, 200 Cholesky vectors; CCSD 3 occ / 12 vir, CC2 the rest
    "small": _spec("small", 8, 40, 200, 8, 40, 3, 12, 3),
    # 340 orbitals, 40 occupied, 1500 vectors; CCSD 10 / 60, CC2 the rest; 4 roots
    "mid": _spec("mid", 40, 300, 1500, 40, 300, 10, 60, 4),
    # 1350 orbitals, 150 occupied, 6000 vectors; CC2 40 / 300, CCS the rest; 6 roots
    "mlcc2_large": _spec("mlcc2_large", 150, 1200, 6000, 40, 300, 0, 0, 6),
    # 560 orbitals, 60 occupied, 2500 vectors; CCSD 20 / 140 in CC2 40 / 300, CCS rest
    "three_level": _spec("three_level", 60, 500, 2500, 40, 300, 20, 140, 4),
    # excited-state parity case: 170 orbitals, 20 occupied, 850 vectors; CCSD 6 / 36 in
    # CC2 16 / 110, CCS rest; 4 roots (its rank GEMMs take the tensor-core paths)
    "es_parity": _spec("es_parity", 20, 150, 850, 16, 110, 6, 36, 4),
}


# Serving mix: independent excitation requests of uneven sizes (one synthetic snapshot
# Hamiltonian each). Request r draws from its own stream (seed_base + r):
#   occupied ~ U{20..80}, virtual ~ U{150..600}, N_J = 5 (occ + vir), tau = N_J / 5;
#   active fraction f ~ U[0.1, 0.3), applied to the occupied and the virtual orbitals
#   (rounded, at least 1);
#   kind: "ccs_ccsd" (two levels: the active orbitals CCSD, the rest CCS) or "mlcc2" (the
#   active orbitals CC2, the rest CCS), each with probability 1/2;
#   4 roots.
# Arrival times: exponential gaps at `rate` requests per second from a stream of their own.
SERVING_OCC = (20, 80)
SERVING_VIR = (150, 600)
SERVING_FRACTION = (0.1, 0.3)


def serving_request_spec(r, seed_base=0):
    rng = np.random.default_rng(seed_base + r)
    no = int(rng.integers(SERVING_OCC[0], SERVING_OCC[1] + 1))
    nv = int(rng.integers(SERVING_VIR[0], SERVING_VIR[1] + 1))
    f = float(rng.uniform(*SERVING_FRACTION))
    kind = "ccs_ccsd" if rng.random() < 0.5 else "mlcc2"
    ao = max(1, int(round(f * no)))
    av = max(1, int(round(f * nv)))
    nj = 5 * (no + nv)
    tau = nj / 5.0
    t_o, t_v = (ao, av) if kind == "ccs_ccsd" else (0, 0)
    spec = SystemSpec(f"serve{r}_{kind}", no, nv, nj, tau, ao, av, t_o, t_v, 4, seed_base + r,
                      default_scale(tau))
    return spec, kind, f


def serving_arrivals(n, rate=20.0, seed=1 << 20):
    """Arrival times (seconds from the first request) of n requests: exponential gaps."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    gaps[0] = 0.0
    return np.cumsum(gaps)

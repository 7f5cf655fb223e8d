"""Writes the stored expected values under tests/golden/ from the oracle alone.

  python tests/golden/make_golden.py small    # seconds
  python tests/golden/make_golden.py mid      # the oracle ground state of the 340-orbital
                                              # workload: tens of minutes on 8 cores
  python tests/golden/make_golden.py three_level   # 560 orbitals, CCS / CC2 / CCSD levels
  python tests/golden/make_golden.py es_parity     # 170 orbitals, three levels, with roots

For each workload: the reference energy E_HF = sum_I (h_II + F_II) of the reduced space,
the MLCC ground-state correlation energy (Eq. mlcc_energy at Omega = 0, DIIS quasi-Newton
of Sec. 2.1), the residual norm and iteration count, and (small and es_parity) the lowest
excitation energies from the oracle's Davidson on A = dOmega/dx. Inputs come from the
seeded generator in synth/ (shared input module, no method arithmetic).
"""
import hashlib
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle.davidson import excited_states  # noqa: E402
from oracle.mlcc import MLCCSystem, hf_energy, solve_ground_state  # noqa: E402
from synth import CONFIGS, draw_model_hamiltonian, make_system  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def draws_sha256(spec):
    """SHA-256 of the raw seeded draws (h then L, little-endian binary64) of a workload."""
    ham = draw_model_hamiltonian(spec.n_mo, spec.n_chol, spec.tau, spec.seed, spec.scale)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ham.h, dtype="<f8").tobytes())
    h.update(np.ascontiguousarray(ham.L, dtype="<f8").tobytes())
    return h.hexdigest()


def main(name):
    spec = CONFIGS[name]
    t0 = time.time()
    s = make_system(spec)
    o = MLCCSystem(s.L, s.fock, spec.n_occ, s.level)
    gs = solve_ground_state(o, verbose=True)
    out = {"workload": name, "n_mo": spec.n_mo, "n_occ": spec.n_occ, "n_chol": spec.n_chol,
           "s_occ": spec.s_occ, "s_vir": spec.s_vir, "t_occ": spec.t_occ, "t_vir": spec.t_vir,
           "seed": spec.seed, "e_hf": float(hf_energy(o)), "e_corr": float(gs.energy),
           "omega_norm": float(gs.omega_norm), "gs_iterations": int(gs.iterations), "gs_converged": bool(gs.converged)}
    if name in ("small", "es_parity"):
        es = excited_states(o, gs, spec.n_roots, res_tol=1e-9)
        out["omega"] = [float(w) for w in es.omega]
        out["es_residuals"] = [float(r) for r in es.residuals]
        out["es_sigma"] = int(es.n_sigma)
    if name == "small":
        out["draws_sha256"] = draws_sha256(spec)
    out["written_by"] = "tests/golden/make_golden.py (oracle/ only)"
    out["host"] = {"machine": platform.machine(), "numpy": np.__version__, "seconds": time.time() - t0}
    path = os.path.join(HERE, f"{name}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, json.dumps(out))


if __name__ == "__main__":
    for n in sys.argv[1:] or ["small"]:
        main(n)

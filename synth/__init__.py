"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds no coupled-cluster arithmetic. It draws a closed-shell model
Hamiltonian (one-electron matrix h and AO Cholesky vectors L^J) from a seed, runs a
restricted Hartree-Fock calculation on it to produce the canonical molecular-orbital
quantities that the multilevel CC method starts from (MO Cholesky vectors L^J_pq and the
Fock matrix F_pq, Sec. 2.3 Eq. eff_fock), and assigns orbitals to the CCS / CC2 / CCSD
levels. Everything downstream (T1-dressing, residuals, Jacobian, Davidson) lives elsewhere.
"""
from .generator import (ModelHamiltonian, draw_model_hamiltonian, SystemSpec, MOSystem, default_scale,
                        make_system, level_map, CONFIGS, serving_request_spec, serving_arrivals)
from .rhf import rhf, RHFResult

__all__ = ["ModelHamiltonian", "draw_model_hamiltonian", "SystemSpec", "MOSystem", "default_scale",
           "make_system", "level_map", "CONFIGS", "serving_request_spec", "serving_arrivals", "rhf",
           "RHFResult"]

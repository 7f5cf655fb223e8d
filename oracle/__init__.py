"""Plain FP64 CPU oracle for the MLCC2 / MLCCSD hot path (arXiv 2006.05226).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this package: only
tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs use it. It
shares no code with the CUDA library; both sides take their inputs from the seeded
generator in synth/.

Contents (each function cites the passage it restates):
  mlcc.MLCCSystem            orbital partition, active index sets, h_eff recovery (Sec. 2.3)
  mlcc.t1_transform          T1-dressing of Cholesky vectors (Sec. 2.1, Appendix A)
  mlcc.fock_t1               Fock matrix in the X1 basis (Appendix A, Eq. for F~)
  mlcc.omega                 ground-state residual: Omega_AI (Eq. mlcc2_omega_codable),
                             CC2 doubles (analytic s), MLCCSD doubles Omega_aibj
  mlcc.energy                correlation energy (Eq. mlcc_energy)
  mlcc.solve_ground_state    quasi-Newton + DIIS (Sec. 2.1)
  mlcc.sigma                 Jacobian transformation sigma = A c, A = dOmega/dx (Sec. 2.1,
                             Appendix A "Jacobian transformation"), as an exact
                             complex-step directional derivative of omega()
  mlcc.sigma_mlcc2_paper     the paper's explicit MLCC2 sigma (Eq. mlcc_A_ and the
                             sigma^MLCC2_aibj equation), for cross-checks
  davidson.davidson          lowest right eigenpairs of the non-symmetric Jacobian

Pins (tests/test_oracle_*.py) tie this code to brute-force determinant-space coupled
cluster, FCI for two-electron systems, the CIS and MP2 closed forms, finite differences
and the limits the paper states. Where the printed equations are garbled or silent, the
reading taken is stated at the function that depends on it.
"""

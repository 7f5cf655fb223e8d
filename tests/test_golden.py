"""Stored expected values (tests/golden/*.json, written by tests/golden/make_golden.py from
the oracle alone) still match what the oracle and the generator produce (no GPU):
  * the raw seeded draws of the 48-orbital workload hash to the stored SHA-256, so the
    generator's stream and draw order are unchanged;
  * the oracle's reference energy, ground-state correlation energy and lowest excitation
    energies of that workload equal the stored ones;
  * the stored files are complete and internally consistent (the 340- and 560-orbital
    files, used by the full-size GPU tests, hold converged ground states of the stated
    workloads).
"""
import json
import os
import platform

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _load(name):
    path = os.path.join(GOLDEN, f"{name}_oracle.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    return json.load(open(path))


def test_generator_draws_unchanged():
    import sys
    sys.path.insert(0, GOLDEN)
    from make_golden import draws_sha256
    from synth import CONFIGS
    g = _load("small")
    if platform.machine() != g["host"]["machine"]:
        pytest.skip("the hash covers exp() results of the host's libm")
    assert draws_sha256(CONFIGS["small"]) == g["draws_sha256"]


def test_oracle_reproduces_the_stored_small_workload():
    from oracle.davidson import excited_states
    from oracle.mlcc import MLCCSystem, hf_energy, solve_ground_state
    from synth import CONFIGS, make_system
    g = _load("small")
    s = make_system(CONFIGS["small"])
    o = MLCCSystem(s.L, s.fock, s.spec.n_occ, s.level)
    gs = solve_ground_state(o)
    assert abs(hf_energy(o) - g["e_hf"]) < 1e-9
    assert abs(gs.energy - g["e_corr"]) < 1e-10
    es = excited_states(o, gs, len(g["omega"]), res_tol=1e-9)
    assert np.abs(es.omega - np.array(g["omega"])).max() < 1e-9


@pytest.mark.parametrize("name", ["small", "mid", "three_level", "es_parity"])
def test_stored_files_describe_their_workload(name):
    from synth import CONFIGS
    g = _load(name)
    s = CONFIGS[name]
    assert (g["n_mo"], g["n_occ"], g["n_chol"], g["seed"]) == (s.n_mo, s.n_occ, s.n_chol, s.seed)
    assert (g["s_occ"], g["s_vir"], g["t_occ"], g["t_vir"]) == (s.s_occ, s.s_vir, s.t_occ, s.t_vir)
    assert g["gs_converged"] and g["omega_norm"] < 1e-10
    assert g["e_corr"] < 0.0 and g["written_by"].startswith("tests/golden/make_golden.py")

"""The three-level workload at full size (560 orbitals, 60 occupied / 500 virtual, 2500
Cholesky vectors; CCSD-active 20 / 140 inside CC2-active 40 / 300, the rest CCS): the
reference and ground-state correlation energies of the binary64 path and of the mixed path
(split bfloat16 iterations polished in MLCC_FP64E) against the oracle's, stored by
tests/golden/make_golden.py, to 1e-8 Ha. This is the only full-size case with all three
levels. Collected after the other GPU tests, so that a failure here cannot hide their
results.
"""
import json
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_ground_state_three_level_against_the_stored_oracle():
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS, make_system
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "three_level_oracle.json")
    ref = json.load(open(path))
    spec = CONFIGS["three_level"]
    s = make_system(spec)
    ctx = mlcc.Context(0)
    L = torch.as_tensor(s.L, device="cuda")
    F = torch.as_tensor(s.fock, device="cuda")
    fp64 = mlcc.default_options(n_roots=spec.n_roots)
    mixed = mlcc.default_options(n_roots=spec.n_roots, precision=mlcc.MLCC_BF16X3, gs_precision=mlcc.MLCC_BF16X3,
                                 refine_fp64=1, lowp_res_tol=1e-5, refine_precision=mlcc.MLCC_FP64E,
                                 gs_tol=1e-9, gs_energy_tol=1e-10)
    try:
        for opts in (fp64, mixed):
            g = mlcc.System(ctx, L, F, spec.n_occ, s.level)
            _, _, info = g.ground_state(opts)
            g.close()
            assert info.converged
            assert abs(info.e_hf - ref["e_hf"]) < 1e-8
            assert abs(info.e_corr - ref["e_corr"]) < 1e-8, (opts.precision, info.e_corr, ref["e_corr"])
    finally:
        del L, F
        ctx.close()

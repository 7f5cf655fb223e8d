"""Excited states against the oracle on a system whose contractions take the tensor-core
paths: 170 orbitals (20 occupied / 150 virtual), 850 Cholesky vectors, CCSD-active 6 / 36
inside CC2-active 16 / 110, CCS the rest (three levels), 4 roots. Its rank GEMMs
(2 d_S^2 N_J = 1.5e10 flop) and CCSD-block contractions run on tcgen05 in MLCC_FP64E and
the split-bfloat16 precisions.

The oracle's ground-state energy and roots (its Davidson on A = dOmega/dx) are stored by
tests/golden/make_golden.py (oracle/ only). Checked here, through the C ABI:
  * the ground-state energy of every path to 1e-8 Ha;
  * the roots of the binary64 path and of MLCC_FP64E to 1e-8 Ha; of the mixed path (the
    benchmark's options: BF16X3 phases, one MLCC_FP64E Rayleigh-Ritz sweep) to 1e-6 Ha, and
    with refinement to convergence to 1e-8 Ha; of the folded CC2 eigensolver to 1e-8 Ha;
  * each returned eigenvector of the binary64 path is an eigenvector of the oracle's
    Jacobian at the oracle's own ground state: |A R - w R| < 1e-7.
"""
import json
import os

import numpy as np
import pytest

from gpu_helpers import Layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def setup():
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS, make_system
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    path = os.path.join(HERE, "golden", "es_parity_oracle.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle values for the excited-state parity case")
    ref = json.load(open(path))
    s = make_system(CONFIGS["es_parity"])
    ctx = mlcc.Context(0)
    L = torch.as_tensor(s.L, device="cuda")
    F = torch.as_tensor(s.fock, device="cuda")
    yield mlcc, ctx, s, L, F, ref
    ctx.close()


def _run(mlcc, ctx, s, L, F, opts, folded=False):
    g = mlcc.System(ctx, L, F, s.spec.n_occ, s.level)
    _, _, gi = g.ground_state(opts)
    if folded:
        w, R, ei = g.excited_states_folded(opts)
    else:
        w, R, ei = g.excited_states(opts)
    return g, gi, w, R, ei


def test_fp64_roots_and_vectors(setup):
    from oracle.mlcc import MLCCSystem, sigma, solve_ground_state
    mlcc, ctx, s, L, F, ref = setup
    opts = mlcc.default_options(n_roots=4)
    g, gi, w, R, ei = _run(mlcc, ctx, s, L, F, opts)
    assert abs(gi.e_corr - ref["e_corr"]) < 1e-8
    assert ei.converged and np.abs(w - np.array(ref["omega"])).max() < 1e-8
    o = MLCCSystem(s.L, s.fock, s.spec.n_occ, s.level)
    gs = solve_ground_state(o)
    lay = Layout(g, o)
    Rh = R.cpu().numpy()
    n1 = o.nv * o.no
    for k in range(4):
        c1 = lay.t1_back(Rh[k, :n1], (o.nv, o.no))
        c2 = lay.x2_back(Rh[k, n1:], o.doubles_shape())
        s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
        res = np.sqrt(np.sum((s1 - w[k] * c1) ** 2) + np.sum((s2 - w[k] * c2) ** 2))
        assert res < 1e-7, (k, res)
    g.close()


@pytest.mark.parametrize("mode", ["fp64e", "mixed", "mixed_refined", "folded"])
def test_roots_of_each_path(setup, mode):
    mlcc, ctx, s, L, F, ref = setup
    want = np.array(ref["omega"])
    if mode == "fp64e":
        opts = mlcc.default_options(n_roots=4, precision=mlcc.MLCC_FP64E, gs_precision=mlcc.MLCC_FP64E)
        tol = 1e-8
    elif mode == "folded":
        opts = mlcc.default_options(n_roots=4, es_res_tol=1e-8)
        tol = 1e-8
    else:
        refine = 1 if mode == "mixed" else 1000
        opts = mlcc.default_options(n_roots=4, precision=mlcc.MLCC_BF16X3, gs_precision=mlcc.MLCC_BF16X3,
                                    refine_fp64=refine, lowp_res_tol=1e-5, refine_precision=mlcc.MLCC_FP64E,
                                    gs_tol=1e-9, gs_energy_tol=1e-10)
        tol = 1e-6 if mode == "mixed" else 1e-8
    g, gi, w, R, ei = _run(mlcc, ctx, s, L, F, opts, folded=(mode == "folded"))
    assert abs(gi.e_corr - ref["e_corr"]) < 1e-8
    err = np.abs(w - want).max()
    print(f"{mode}: max |omega - oracle| = {err:.2e} Ha, {ei.n_sigma} sigma")
    assert err < tol
    g.close()

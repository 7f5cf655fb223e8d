"""Through the C ABI: the library's results do not depend on the order in which the caller
lists the orbitals of each level. The 48-orbital workload with its occupied and its
virtual orbitals permuted (levels permuted with them) gives the same correlation energy
and excitation energies as in canonical order, to the binary64 parity tolerance; the
library's internal level order (mlcc_orbital_order) maps the two back onto each other.
Collected after the other GPU tests, so that a failure here cannot hide their results.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_do_not_depend_on_the_callers_orbital_order():
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS, make_system
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = make_system(CONFIGS["small"])
    n, k = s.fock.shape[0], s.spec.n_occ
    rng = np.random.default_rng(8)
    p = np.concatenate([rng.permutation(k), k + rng.permutation(n - k)])
    ctx = mlcc.Context(0)
    opts = mlcc.default_options(n_roots=3)
    out = []
    for perm in (np.arange(n), p):
        L = torch.as_tensor(np.ascontiguousarray(s.L[:, perm][:, :, perm]), device="cuda")
        F = torch.as_tensor(np.ascontiguousarray(s.fock[np.ix_(perm, perm)]), device="cuda")
        g = mlcc.System(ctx, L, F, k, s.level[perm])
        _, _, gi = g.ground_state(opts)
        w, _, ei = g.excited_states(opts, want_vectors=False)
        out.append((gi.e_corr, w, perm[g.perm]))
        g.close()
    ctx.close()
    (e0, w0, o0), (e1, w1, o1) = out
    assert abs(e0 - e1) < 1e-10
    assert np.abs(w0 - w1).max() < 1e-8
    # both internal orders list the same orbitals level by level
    assert sorted(o0.tolist()) == sorted(o1.tolist()) == list(range(n))
    lev = s.level
    assert np.array_equal(lev[o0], lev[o1])


def test_ccsd_level_without_virtual_orbitals_is_mlcc2():
    """A CCSD level holding only occupied orbitals has no doubles with all four indices
    CCSD-active: the library must then give the MLCC2 results of the same CC2 set."""
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS, make_system
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = make_system(CONFIGS["small"])
    k = s.spec.n_occ
    lev_occ_only = s.level.copy()
    lev_occ_only[k:][lev_occ_only[k:] == 2] = 1
    lev_mlcc2 = lev_occ_only.copy()
    lev_mlcc2[lev_mlcc2 == 2] = 1
    ctx = mlcc.Context(0)
    L = torch.as_tensor(s.L, device="cuda")
    F = torch.as_tensor(s.fock, device="cuda")
    opts = mlcc.default_options(n_roots=3)
    res = []
    for lev in (lev_occ_only, lev_mlcc2):
        g = mlcc.System(ctx, L, F, k, lev)
        assert g.dims.t_vir == 0
        _, _, gi = g.ground_state(opts)
        w, _, _ = g.excited_states(opts, want_vectors=False)
        res.append((gi.e_corr, w))
        g.close()
    ctx.close()
    assert abs(res[0][0] - res[1][0]) < 1e-10
    assert np.abs(res[0][1] - res[1][1]).max() < 1e-8

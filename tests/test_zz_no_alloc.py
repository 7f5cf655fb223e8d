"""The allocation-free entry point (mlcc_fock_t1_noalloc) against the system-based ones.

For callers that cannot let the library allocate device memory (their own memory pool
holds the device, or they cannot accept the synchronisation of cudaMalloc / cudaFree),
mlcc_fock_t1_noalloc works from caller buffers and a fixed static scratch array. Two calls
in a row (the scratch keeps the previous call's contents) must agree with
mlcc_t1_transform and mlcc_fock_t1 to the binary64 parity tolerance. Collected last so
that a failure here cannot hide another test's result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-10


def _close(a, b):
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= REL * scale, f"max error {err:.3e} > {REL:.1e} * {scale:.3e}"


def test_fock_t1_noalloc_matches_system_entry_points():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS, make_system
    s = make_system(CONFIGS["small"])
    n, no, nj = s.spec.n_mo, s.spec.n_occ, s.spec.n_chol
    nv = n - no
    L = torch.as_tensor(s.L, device="cuda")
    F = torch.as_tensor(s.fock, device="cuda")
    ctx = mlcc.Context(0)
    g = mlcc.System(ctx, L, F, no, s.level)
    perm = g.perm
    pv = perm[no:] - no
    po = perm[:no]
    rng = np.random.default_rng(17)
    lt = torch.empty(nj, n, n, dtype=torch.float64, device="cuda")
    ft = torch.empty(n, n, dtype=torch.float64, device="cuda")
    for call in range(2):
        t1_user = 0.05 * rng.standard_normal((nv, no))
        mlcc.fock_t1_noalloc(L, F, no, torch.as_tensor(t1_user, device="cuda"), lt, ft)
        torch.cuda.synchronize()
        t1_int = torch.as_tensor(np.ascontiguousarray(t1_user[np.ix_(pv, po)]), device="cuda")
        ref_lt = g.t1_transform(t1_int).cpu().numpy()
        ref_ft = g.fock_t1(t1_int).cpu().numpy()
        got_lt = lt.cpu().numpy()[:, perm[:, None], perm[None, :]]
        got_ft = ft.cpu().numpy()[perm[:, None], perm[None, :]]
        _close(got_lt, ref_lt)
        _close(got_ft, ref_ft)
    g.close()
    ctx.close()


def test_fock_t1_noalloc_rejects_too_many_cholesky_vectors():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2006_05226_gb300 import mlcc
    lib = mlcc.load()
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    st = lib.mlcc_fock_t1_noalloc(4, 2, 32769, p, p, p, p, p, None)
    assert st == -1 and b"MLCC_NOALLOC_MAX_CHOL" in lib.mlcc_last_error()

"""MLCC_FP64E: binary64 GEMMs from exact integer slices on the tcgen05 tensor cores.

Pins, through the C ABI (mlcc_gemm and the solver entry points):
  1. integer matrices whose digits are exact give the exact integer product bit for bit:
     every fp32 tensor-core chunk sum must be exact and the 64-bit combination lossless;
  2. random binary64 operands with rows and columns of very different scale, zero rows,
     subnormals, alpha / beta and every transpose agree with numpy's binary64 product
     within the error bound of the splitting (8 digits of 7 bits, products kept down to
     2^-49 of the leading one: about 2^-53 of max|row| max|column| per product);
  3. a Cholesky-rank GEMM of the 340-orbital workload (12000 x 12000 x 1500), sampled rows;
  4. through the solver: sigma, the ground state and the excited states agree with the
     binary64 path and the oracle.
"""
import numpy as np
import pytest

from oracle.davidson import excited_states as oracle_es
from oracle.mlcc import MLCCSystem, solve_ground_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    from paper_2006_05226_gb300 import mlcc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mlcc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small():
    from synth import CONFIGS, make_system
    return make_system(CONFIGS["small"])


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _op(x, trans):
    """Stored operand for op(x): x itself, or its transpose laid out row-major."""
    return np.ascontiguousarray(x.T) if trans else np.ascontiguousarray(x)


def _gemm(ctx, A, B, ta, tb, prec, C0=None, alpha=1.0, beta=0.0):
    M, N = A.shape[0], B.shape[1]
    c = _dev(C0) if C0 is not None else torch.zeros((M, N), dtype=torch.float64, device="cuda")
    ctx.gemm(_dev(_op(A, ta)), _dev(_op(B, tb)), c, alpha=alpha, beta=beta, trans_a=ta, trans_b=tb,
             precision=prec)
    return _host(c)


def _bound(A, B):
    """Worst-case error bound of the emulation plus numpy's binary64 error."""
    K = A.shape[1]
    rmax = np.abs(A).max(axis=1)[:, None]
    cmax = np.abs(B).max(axis=0)[None, :]
    return 16 * K * 2.0 ** -53 * 4 * rmax * cmax + 2 * K * 2.0 ** -53 * (np.abs(A) @ np.abs(B))


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_exact_integer_product(ctx, ta, tb):
    """|a|, |b| < 2^20: four digits hold every element, K * 2^40 < 2^53 holds every sum, so
    the emulated product is the exact integer product (several tiles, ragged edges, chunks
    of every group across K = 2100)."""
    from paper_2006_05226_gb300 import mlcc
    rng = np.random.default_rng(11)
    M, N, K = 300, 520, 2100
    A = rng.integers(-(2 ** 20) + 1, 2 ** 20, size=(M, K)).astype(np.float64)
    B = rng.integers(-(2 ** 20) + 1, 2 ** 20, size=(K, N)).astype(np.float64)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    out = _gemm(ctx, A, B, ta, tb, mlcc.MLCC_FP64E)
    assert np.array_equal(out, exact), f"max deviation {np.abs(out - exact).max()}"
    # the binary64 FMA path is exact here too (integer partial sums below 2^53)
    out64 = _gemm(ctx, A, B, ta, tb, mlcc.MLCC_FP64)
    assert np.array_equal(out64, exact)


_EXACT = {}


def _exact_row(A, B, m):
    from fractions import Fraction
    key = (m, A.shape, B.shape)
    if key not in _EXACT:
        a = [Fraction(x) for x in A[m]]
        _EXACT[key] = np.array([float(sum(ak * Fraction(bk) for ak, bk in zip(a, B[:, n]) if ak and bk))
                                for n in range(B.shape[1])])
    return _EXACT[key]


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_random_binary64(ctx, ta, tb):
    from paper_2006_05226_gb300 import mlcc
    rng = np.random.default_rng(12)
    M, N, K = 257, 300, 1500
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-20, 20, (1, N)))
    A[5, :] = 0.0                      # zero row
    A[7, :] *= 1e-300                  # subnormal-scale row
    A[9, 3] = 5e-324                   # smallest subnormal inside a normal row
    B[:, 11] = 0.0                     # zero column
    out = _gemm(ctx, A, B, ta, tb, mlcc.MLCC_FP64E)
    ref = A @ B
    # gradual underflow: every rounding in the subnormal range (numpy's products, the
    # final scaling of ours) costs up to 2^-1075 absolute, below any relative bound
    floor = 4 * K * 2.0 ** -1074
    assert np.all(np.abs(out - ref) <= _bound(A, B) + floor)
    # three rows against the exact rational product (row 7 has subnormal elements, where
    # numpy loses up to 1e-7 relative): the emulation's error relative to max|row| max|col|
    # is a few 1e-16 typically (the same arithmetic run on the CPU gives medians of 7e-16,
    # numpy's are 1e-15) and below 2e-14 everywhere
    cmax = np.abs(B).max(axis=0)
    for m in (0, 7, 100):
        ex = _exact_row(A, B, m)
        sc = np.abs(A[m]).max() * cmax
        err = np.abs(out[m] - ex)
        assert np.all(err <= 4e-14 * sc + 2 * 2.0 ** -1074), m
        assert np.median(err[sc > 0] / sc[sc > 0]) < 2e-15, m
    assert np.all(out[5, :] == 0.0) and np.all(out[:, 11] == 0.0)
    # alpha and beta
    C0 = rng.standard_normal((M, N))
    out = _gemm(ctx, A, B, ta, tb, mlcc.MLCC_FP64E, C0=C0, alpha=-0.75, beta=1.5)
    ref2 = -0.75 * ref + 1.5 * C0
    bound = 0.75 * (_bound(A, B) + floor) + 4 * 2.0 ** -53 * (0.75 * np.abs(ref) + 1.5 * np.abs(C0))
    assert np.all(np.abs(out - ref2) <= bound)


def test_nonfinite_rows_give_nan(ctx):
    from paper_2006_05226_gb300 import mlcc
    rng = np.random.default_rng(13)
    A = rng.standard_normal((128, 200))
    B = rng.standard_normal((200, 96))
    A[3, 17] = np.nan
    B[40, 5] = np.inf
    out = _gemm(ctx, A, B, False, False, mlcc.MLCC_FP64E)
    assert np.all(np.isnan(out[3, :])) and np.all(np.isnan(out[:, 5]))
    mask = np.ones_like(out, dtype=bool)
    mask[3, :] = False
    mask[:, 5] = False
    assert np.all(np.isfinite(out[mask]))


def test_shapes_outside_the_path_are_rejected(ctx):
    from paper_2006_05226_gb300 import mlcc
    A = np.ones((8, 100))
    B = np.ones((100, 256))
    with pytest.raises(mlcc.MLCCError) as e:
        _gemm(ctx, A, B, False, False, mlcc.MLCC_FP64E)
    assert e.value.status == -1


def test_rank_gemm_of_the_340_orbital_workload(ctx):
    """C = A^T B with A, B [1500][12000] (the sigma outer product of the 340-orbital, 1500-
    vector workload); 16 sampled rows against numpy's binary64 product."""
    from paper_2006_05226_gb300 import mlcc
    nj, dS = 1500, 12000
    g = torch.Generator(device="cuda").manual_seed(14)
    A = torch.randn((nj, dS), generator=g, dtype=torch.float64, device="cuda") * 0.05
    B = torch.randn((nj, dS), generator=g, dtype=torch.float64, device="cuda") * 0.05
    C = torch.empty((dS, dS), dtype=torch.float64, device="cuda")
    ctx.gemm(A, B, C, trans_a=True, precision=mlcc.MLCC_FP64E)
    rows = np.random.default_rng(15).choice(dS, 16, replace=False)
    Ah, Bh = _host(A), _host(B)
    out = _host(C[torch.as_tensor(rows, device="cuda")])
    ref = Ah[:, rows].T @ Bh
    bound = _bound(Ah[:, rows].T, Bh)
    assert np.all(np.abs(out - ref) <= bound)
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-13


@pytest.fixture(scope="module")
def small_prepared(ctx, small):
    from paper_2006_05226_gb300 import mlcc
    o = MLCCSystem(small.L, small.fock, small.spec.n_occ, small.level)
    gs = solve_ground_state(o)
    g = mlcc.System(ctx, _dev(small.L), _dev(small.fock), small.spec.n_occ, small.level)
    g.ground_state()
    return g, o, gs


def test_sigma_fp64e_matches_binary64(ctx, small_prepared):
    from paper_2006_05226_gb300 import mlcc
    g, _, _ = small_prepared
    rng = np.random.default_rng(16)
    c = rng.standard_normal((2, g.dims.vector_len))
    ref = _host(g.sigma(_dev(c)))
    ctx.kernel_timing(True)
    out = _host(g.sigma(_dev(c), precision=mlcc.MLCC_FP64E))
    n, _, _ = ctx.kernel_time("rank_gemm_f64e")
    ctx.kernel_timing(False)
    assert n > 0, "the rank GEMMs did not take the emulated tensor-core path"
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-12


def test_ground_state_fp64e(ctx, small_prepared):
    from paper_2006_05226_gb300 import mlcc
    g, _, gs = small_prepared
    t1, x2, info = g.ground_state(mlcc.default_options(gs_precision=mlcc.MLCC_FP64E))
    assert info.converged and abs(info.e_corr - gs.energy) < E_TOL
    # split-bfloat16 phase, then the polish in FP64E
    t1, x2, info = g.ground_state(mlcc.default_options(gs_precision=mlcc.MLCC_BF16X3, refine_fp64=1,
                                                       refine_precision=mlcc.MLCC_FP64E))
    assert info.converged and abs(info.e_corr - gs.energy) < E_TOL


def test_excited_states_fp64e(ctx, small_prepared):
    from paper_2006_05226_gb300 import mlcc
    g, o, gs = small_prepared
    g.ground_state()
    ref = oracle_es(o, gs, 3, res_tol=1e-9)
    w, _, info = g.excited_states(mlcc.default_options(n_roots=3, precision=mlcc.MLCC_FP64E),
                                  want_vectors=False)
    assert info.converged and info.n_sigma_lowp == 0
    assert np.abs(w - ref.omega).max() < E_TOL
    w, _, info = g.excited_states(mlcc.default_options(n_roots=3, precision=mlcc.MLCC_BF16X3,
                                                       refine_fp64=1000, lowp_res_tol=1e-4,
                                                       refine_precision=mlcc.MLCC_FP64E),
                                  want_vectors=False)
    assert info.converged and info.n_sigma_lowp > 0 and info.fp64_sweeps >= 1
    assert np.abs(w - ref.omega).max() < E_TOL


@pytest.mark.parametrize("prec,tol", [(1, 3e-2), (2, 1e-3), (3, 1e-4)])
def test_split_bf16_precisions(ctx, prec, tol):
    """The split-bfloat16 precisions of the same engine (fp32 accumulation): relative error
    against numpy within the bounds the sigma-vectors meet (BF16 ~ 2^-8, BF16X3 and BF16X6
    limited by fp32 accumulation over K)."""
    rng = np.random.default_rng(17)
    M, N, K = 300, 520, 1500
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    out = _gemm(ctx, A, B, False, False, prec)
    ref = A @ B
    rel = np.abs(out - ref).max() / np.abs(ref).max()
    assert rel < tol, rel
    if prec > 1:   # the extra pieces help
        out1 = _gemm(ctx, A, B, False, False, 1)
        assert rel < np.abs(out1 - ref).max() / np.abs(ref).max()

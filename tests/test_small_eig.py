"""The host-side small dense solvers of the DIIS and Davidson loops (csrc/small_eig.cpp),
compiled on their own with g++ and checked against LAPACK through numpy (no GPU):
  * solve_linear (Gaussian elimination with partial pivoting) against numpy.linalg.solve;
  * eig_nonsym (Hessenberg reduction, complex shifted QR, inverse iteration): every
    eigenvalue of random non-symmetric matrices (complex pairs included) and of
    Davidson-like subspace matrices, eigenvalues sorted by real part, and right
    eigenvectors with A v = lambda v.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_05226_gb300", "csrc")

SHIM = r"""
#include "small_eig.h"
#include <complex>
#include <vector>
extern "C" int t_solve(int n, const double* A, const double* b, double* x) {
  std::vector<double> a(A, A + n * n), bb(b, b + n), xx;
  if (!mlcc::solve_linear(n, a, bb, xx)) return 0;
  for (int i = 0; i < n; ++i) x[i] = xx[i];
  return 1;
}
extern "C" int t_eig(int n, const double* A, double* wr, double* wi, int nv, double* vr, double* vi) {
  std::vector<double> a(A, A + n * n);
  std::vector<std::complex<double>> w;
  std::vector<std::vector<std::complex<double>>> v;
  if (!mlcc::eig_nonsym(n, a, w, nv > 0 ? &v : nullptr, nv)) return 0;
  for (int i = 0; i < n; ++i) { wr[i] = w[i].real(); wi[i] = w[i].imag(); }
  for (int k = 0; k < nv; ++k)
    for (int i = 0; i < n; ++i) { vr[k * n + i] = v[k][i].real(); vi[k * n + i] = v[k][i].imag(); }
  return 1;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("small_eig")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libsmall_eig_test.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", f"-I{CSRC}", str(shim),
                    os.path.join(CSRC, "small_eig.cpp"), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    P = ctypes.POINTER(ctypes.c_double)
    L.t_solve.argtypes = [ctypes.c_int, P, P, P]
    L.t_eig.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P, P]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _eig(lib, A, nv):
    n = A.shape[0]
    A = np.ascontiguousarray(A, dtype=np.float64)
    wr, wi = np.zeros(n), np.zeros(n)
    vr, vi = np.zeros(max(nv, 1) * n), np.zeros(max(nv, 1) * n)
    assert lib.t_eig(n, _p(A), _p(wr), _p(wi), nv, _p(vr), _p(vi)) == 1
    return wr + 1j * wi, (vr + 1j * vi).reshape(max(nv, 1), n)[:nv]


@pytest.mark.parametrize("n", [1, 4, 17, 40])
def test_solve_linear(lib, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
    b = rng.standard_normal(n)
    x = np.zeros(n)
    assert lib.t_solve(n, _p(np.ascontiguousarray(A)), _p(b), _p(x)) == 1
    ref = np.linalg.solve(A, b)
    assert np.abs(x - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()) * np.linalg.cond(A)


def _check_spectrum(A, w, V):
    ref = np.linalg.eigvals(A)
    scale = max(1.0, np.abs(ref).max())
    # same multiset of eigenvalues
    for lam in ref:
        assert np.abs(w - lam).min() < 1e-9 * scale
    # sorted by real part
    assert np.all(np.diff(w.real) >= -1e-12 * scale)
    # right eigenvectors of the leading ones
    for k in range(V.shape[0]):
        v = V[k]
        assert np.linalg.norm(A @ v - w[k] * v) < 1e-9 * scale * np.linalg.norm(v)


@pytest.mark.parametrize("n,seed", [(2, 0), (6, 1), (25, 2), (64, 3)])
def test_eig_random_nonsymmetric(lib, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    w, V = _eig(lib, A, min(n, 6))
    _check_spectrum(A, w, V)
    if n >= 6:
        assert np.any(np.abs(w.imag) > 1e-6)   # complex pairs were exercised


@pytest.mark.parametrize("n,seed", [(8, 4), (32, 5)])
def test_eig_davidson_like_subspace(lib, n, seed):
    """B^T A B with a mildly non-symmetric A: close real eigenvalues, as in Davidson."""
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(0.01, 2.0, n))
    A = np.diag(d) + 0.02 * rng.standard_normal((n, n))
    w, V = _eig(lib, A, 4)
    _check_spectrum(A, w, V)


SYM_SHIM = r"""
#include "small_eig.h"
#include <vector>
extern "C" int t_eig_sym(int n, const double* A, double* w, double* V) {
  std::vector<double> a(A, A + n * n), ww, vv;
  if (!mlcc::eig_sym(n, a, ww, vv)) return 0;
  for (int i = 0; i < n; ++i) w[i] = ww[i];
  for (int i = 0; i < n * n; ++i) V[i] = vv[i];
  return 1;
}
"""


@pytest.fixture(scope="module")
def symlib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("eig_sym")
    (d / "shim.cpp").write_text(SYM_SHIM)
    so = d / "libeig_sym_test.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", f"-I{CSRC}", str(d / "shim.cpp"),
                    os.path.join(CSRC, "small_eig.cpp"), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    P = ctypes.POINTER(ctypes.c_double)
    L.t_eig_sym.argtypes = [ctypes.c_int, P, P, P]
    return L


def _eig_sym(lib, A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w, V = np.zeros(n), np.zeros((n, n))
    ok = lib.t_eig_sym(n, _p(A), _p(w), _p(V))
    return bool(ok), w, V


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (17, 3), (64, 4), (201, 5)])
def test_eig_sym_random(symlib, n, seed):
    """Eigenvalues against LAPACK (numpy.linalg.eigvalsh); A V = V diag(w) and V^T V = I."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    A = B + B.T
    ok, w, V = _eig_sym(symlib, A)
    assert ok
    scale = max(1.0, np.abs(A).max())
    assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-12 * scale * n
    assert np.all(np.diff(w) >= 0)
    assert np.abs(A @ V - V * w).max() < 1e-11 * scale * n
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12 * n


def test_eig_sym_degenerate_and_structured(symlib):
    """Repeated eigenvalues (a rotated diagonal with a threefold level), a diagonal matrix (no
    reflections needed) and a tridiagonal one with tiny off-diagonals."""
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.array([1.0, 1.0, 1.0, -2.0, 0.5, 0.5, 3.0, 4.0, -1.0, 0.0, 2.0, 2.0])
    A = Q @ np.diag(lam) @ Q.T
    ok, w, V = _eig_sym(symlib, A)
    assert ok and np.abs(w - np.sort(lam)).max() < 1e-13
    assert np.abs(A @ V - V * w).max() < 1e-13 and np.abs(V.T @ V - np.eye(12)).max() < 1e-13
    D = np.diag([3.0, -1.0, 2.0, 0.0])
    ok, w, V = _eig_sym(symlib, D)
    assert ok and np.array_equal(w, [-1.0, 0.0, 2.0, 3.0]) and np.abs(np.abs(V) - np.abs(V).round()).max() == 0.0
    T = np.diag(np.arange(6.0)) + np.diag(np.full(5, 1e-9), 1) + np.diag(np.full(5, 1e-9), -1)
    ok, w, V = _eig_sym(symlib, T)
    assert ok and np.abs(w - np.linalg.eigvalsh(T)).max() < 1e-14

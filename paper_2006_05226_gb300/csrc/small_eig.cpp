// Small dense linear algebra on the host for the solver control loops: the DIIS
// equations and the Davidson subspace eigenproblem (at most a few hundred unknowns).
//
// Non-symmetric eigenvalues: Householder reduction to upper Hessenberg form followed by
// the complex single-shift QR iteration with Wilkinson shifts and deflation (Golub and
// Van Loan, Matrix Computations, Sec. 7.4-7.5). Eigenvectors: inverse iteration on the
// original matrix with a complex LU factorisation with partial pivoting.
#include "small_eig.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace mlcc {

using cplx = std::complex<double>;

bool solve_linear(int n, std::vector<double> A, std::vector<double> b, std::vector<double>& x) {
  // Gaussian elimination with partial pivoting, A row-major n x n
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(A[r * n + k]) > std::fabs(A[p * n + k])) p = r;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int c = 0; c < n; ++c) std::swap(A[k * n + c], A[p * n + c]);
      std::swap(b[k], b[p]);
    }
    for (int r = k + 1; r < n; ++r) {
      const double f = A[r * n + k] / A[k * n + k];
      if (f == 0.0) continue;
      for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
      b[r] -= f * b[k];
    }
  }
  x.assign(n, 0.0);
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * x[c];
    x[k] = s / A[k * n + k];
  }
  return true;
}

static void hessenberg(int n, std::vector<cplx>& H) {
  for (int k = 0; k + 2 < n + 0 && k < n - 2; ++k) {
    // Householder vector for column k below the subdiagonal
    double alpha = 0.0;
    for (int r = k + 1; r < n; ++r) alpha += std::norm(H[r * n + k]);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    std::vector<cplx> v(n, 0.0);
    const cplx x0 = H[(k + 1) * n + k];
    const cplx phase = (std::abs(x0) > 0.0) ? x0 / std::abs(x0) : cplx(1.0, 0.0);
    for (int r = k + 1; r < n; ++r) v[r] = H[r * n + k];
    v[k + 1] += phase * alpha;
    double vn = 0.0;
    for (int r = k + 1; r < n; ++r) vn += std::norm(v[r]);
    if (vn == 0.0) continue;
    // H = (I - 2 v v^H / vn) H (I - 2 v v^H / vn)
    for (int c = 0; c < n; ++c) {
      cplx s = 0.0;
      for (int r = k + 1; r < n; ++r) s += std::conj(v[r]) * H[r * n + c];
      s *= 2.0 / vn;
      for (int r = k + 1; r < n; ++r) H[r * n + c] -= v[r] * s;
    }
    for (int r = 0; r < n; ++r) {
      cplx s = 0.0;
      for (int c = k + 1; c < n; ++c) s += H[r * n + c] * v[c];
      s *= 2.0 / vn;
      for (int c = k + 1; c < n; ++c) H[r * n + c] -= s * std::conj(v[c]);
    }
    for (int r = k + 2; r < n; ++r) H[r * n + k] = 0.0;
  }
}

static bool hessenberg_qr(int n, std::vector<cplx>& H, std::vector<cplx>& w) {
  const double eps = 2.220446049250313e-16;
  int hi = n - 1;
  int iter = 0, total = 0;
  while (hi >= 0) {
    if (hi == 0) {
      w[0] = H[0];
      break;
    }
    // find the active block [lo, hi]
    int lo = hi;
    while (lo > 0) {
      const double sub = std::abs(H[lo * n + lo - 1]);
      const double dia = std::abs(H[lo * n + lo]) + std::abs(H[(lo - 1) * n + lo - 1]);
      if (sub <= eps * (dia > 0.0 ? dia : 1.0)) {
        H[lo * n + lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      w[hi] = H[hi * n + hi];
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 100 * n) return false;
    ++iter;
    // Wilkinson shift from the trailing 2 x 2 block
    const cplx a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
    const cplx c = H[hi * n + hi - 1], d = H[hi * n + hi];
    const cplx tr = a + d, det = a * d - b * c;
    const cplx disc = std::sqrt(tr * tr - 4.0 * det);
    cplx l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
    cplx mu = (std::abs(l1 - d) < std::abs(l2 - d)) ? l1 : l2;
    if (iter % 11 == 10) mu = d + cplx(0.75 * std::abs(c), 0.0);  // exceptional shift
    // QR step on the block by Givens rotations: H - mu I = Q R, H <- R Q + mu I
    std::vector<cplx> cs(hi - lo), sn(hi - lo);
    for (int k = lo; k <= hi; ++k) H[k * n + k] -= mu;
    for (int k = lo; k < hi; ++k) {
      const cplx x = H[k * n + k], y = H[(k + 1) * n + k];
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      cplx cc = 1.0, ss = 0.0;
      if (r > 0.0) {
        cc = x / r;
        ss = y / r;
      }
      cs[k - lo] = cc;
      sn[k - lo] = ss;
      // rows k, k+1: [conj(c) conj(s); -s c] applied from the left
      for (int col = k; col < n; ++col) {
        const cplx p = H[k * n + col], q = H[(k + 1) * n + col];
        H[k * n + col] = std::conj(cc) * p + std::conj(ss) * q;
        H[(k + 1) * n + col] = -ss * p + cc * q;
      }
    }
    for (int k = lo; k < hi; ++k) {
      const cplx cc = cs[k - lo], ss = sn[k - lo];
      // columns k, k+1: right multiplication by the adjoint rotation
      for (int row = 0; row <= std::min(k + 2, hi); ++row) {
        const cplx p = H[row * n + k], q = H[row * n + k + 1];
        H[row * n + k] = p * cc + q * ss;
        H[row * n + k + 1] = -p * std::conj(ss) + q * std::conj(cc);
      }
    }
    for (int k = lo; k <= hi; ++k) H[k * n + k] += mu;
  }
  return true;
}

// inverse iteration: (A - lambda I) x = b with complex LU, a few sweeps
static void inverse_iteration(int n, const std::vector<double>& A, cplx lambda,
                              std::vector<cplx>& x) {
  std::vector<cplx> M(size_t(n) * n);
  double anorm = 0.0;
  for (int i = 0; i < n * n; ++i) anorm = std::max(anorm, std::fabs(A[i]));
  const double pert = 1e-13 * std::max(anorm, 1.0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) M[r * n + c] = A[r * n + c] - (r == c ? lambda + pert : 0.0);
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (std::abs(M[r * n + k]) > std::abs(M[p * n + k])) p = r;
    piv[k] = p;
    if (p != k)
      for (int c = 0; c < n; ++c) std::swap(M[k * n + c], M[p * n + c]);
    if (std::abs(M[k * n + k]) < 1e-300) M[k * n + k] = 1e-300;
    for (int r = k + 1; r < n; ++r) {
      const cplx f = M[r * n + k] / M[k * n + k];
      M[r * n + k] = f;
      for (int c = k + 1; c < n; ++c) M[r * n + c] -= f * M[k * n + c];
    }
  }
  x.assign(n, cplx(1.0, 0.0));
  for (int i = 0; i < n; ++i) x[i] = cplx(1.0 + 0.01 * std::sin(1.0 + i), 0.0);
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) std::swap(x[k], x[piv[k]]);
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < r; ++c) x[r] -= M[r * n + c] * x[c];
    for (int r = n - 1; r >= 0; --r) {
      for (int c = r + 1; c < n; ++c) x[r] -= M[r * n + c] * x[c];
      x[r] /= M[r * n + r];
    }
    double nrm = 0.0;
    for (auto& v : x) nrm += std::norm(v);
    nrm = std::sqrt(nrm);
    for (auto& v : x) v /= nrm;
  }
}

bool eig_nonsym(int n, const std::vector<double>& A, std::vector<cplx>& w,
                std::vector<std::vector<cplx>>* vecs, int n_vecs) {
  std::vector<cplx> H(A.begin(), A.end());
  hessenberg(n, H);
  w.assign(n, 0.0);
  if (!hessenberg_qr(n, H, w)) return false;
  std::stable_sort(w.begin(), w.end(), [](const cplx& a, const cplx& b) { return a.real() < b.real(); });
  if (vecs) {
    vecs->clear();
    for (int k = 0; k < std::min(n_vecs, n); ++k) {
      std::vector<cplx> x;
      inverse_iteration(n, A, w[k], x);
      // fix the phase: largest component real positive
      int im = 0;
      for (int i = 1; i < n; ++i)
        if (std::abs(x[i]) > std::abs(x[im])) im = i;
      const cplx ph = std::abs(x[im]) > 0 ? std::conj(x[im]) / std::abs(x[im]) : cplx(1.0, 0.0);
      for (auto& v : x) v *= ph;
      vecs->push_back(x);
    }
  }
  return true;
}

}  // namespace mlcc

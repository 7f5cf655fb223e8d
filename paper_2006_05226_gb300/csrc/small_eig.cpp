// Small dense linear algebra on the host for the solver control loops: the DIIS
// equations and the Davidson subspace eigenproblem (at most a few hundred unknowns).
//
// Non-symmetric eigenvalues: Householder reduction to upper Hessenberg form followed by
// the complex single-shift QR iteration with Wilkinson shifts and deflation (Golub and
// Van Loan, Matrix Computations, Sec. 7.4-7.5). Eigenvectors: inverse iteration on the
// original matrix with a complex LU factorisation with partial pivoting.
//
// Symmetric eigenpairs (the orbital rotations that make the Fock matrix diagonal inside
// each level): Householder tridiagonalisation with the reflections accumulated, then the
// implicit QL iteration on the tridiagonal matrix with a shift from its leading 2 x 2 block
// (Golub and Van Loan, Sec. 8.3; Wilkinson and Reinsch's QL variant).
#include "small_eig.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <limits>
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

bool eig_sym(int n, const std::vector<double>& A0, std::vector<double>& w, std::vector<double>& V) {
  if (n < 1 || int64_t(A0.size()) < int64_t(n) * n) return false;
  std::vector<double> a(A0.begin(), A0.begin() + size_t(n) * n);
  V.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
  // 1. tridiagonalisation: column k below the subdiagonal is annihilated by the reflection
  //    H = I - beta v v^T acting on rows and columns k+1..n-1
  std::vector<double> v(n), p(n), q(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;   // length of the reflected part
    double alpha = 0.0;
    for (int i = 0; i < m; ++i) alpha += a[size_t(k + 1 + i) * n + k] * a[size_t(k + 1 + i) * n + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = a[size_t(k + 1) * n + k];
    const double sub = x0 >= 0.0 ? -alpha : alpha;   // the new subdiagonal element
    for (int i = 0; i < m; ++i) v[i] = a[size_t(k + 1 + i) * n + k];
    v[0] -= sub;
    double vv = 0.0;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // trailing block B <- H B H = B - v q^T - q v^T with p = beta B v, q = p - (beta/2)(v^T p) v
    for (int i = 0; i < m; ++i) {
      double sdot = 0.0;
      const double* row = &a[size_t(k + 1 + i) * n + (k + 1)];
      for (int j = 0; j < m; ++j) sdot += row[j] * v[j];
      p[i] = beta * sdot;
    }
    double vp = 0.0;
    for (int i = 0; i < m; ++i) vp += v[i] * p[i];
    const double K = 0.5 * beta * vp;
    for (int i = 0; i < m; ++i) q[i] = p[i] - K * v[i];
    for (int i = 0; i < m; ++i) {
      double* row = &a[size_t(k + 1 + i) * n + (k + 1)];
      for (int j = 0; j < m; ++j) row[j] -= v[i] * q[j] + q[i] * v[j];
    }
    a[size_t(k + 1) * n + k] = a[size_t(k) * n + k + 1] = sub;
    for (int i = 1; i < m; ++i) a[size_t(k + 1 + i) * n + k] = a[size_t(k) * n + k + 1 + i] = 0.0;
    // accumulate: V <- V H on columns k+1..n-1
    for (int r = 0; r < n; ++r) {
      double* row = &V[size_t(r) * n + (k + 1)];
      double sdot = 0.0;
      for (int j = 0; j < m; ++j) sdot += row[j] * v[j];
      sdot *= beta;
      for (int j = 0; j < m; ++j) row[j] -= sdot * v[j];
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = a[size_t(i) * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = a[size_t(i + 1) * n + i];   // couples d[i] and d[i+1]
  // 2. implicit QL: deflate from the top; each sweep chases the bulge from the bottom of
  //    the unreduced block [l, m] up to l with plane rotations, applied to V's columns
  const double eps = std::numeric_limits<double>::epsilon();
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (++iter > 80) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      bool early = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pp;
          e[m] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        for (int k = 0; k < n; ++k) {
          double* row = &V[size_t(k) * n];
          const double t = row[i + 1];
          row[i + 1] = s * row[i] + c * t;
          row[i] = c * row[i] - s * t;
        }
      }
      if (early) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  // 3. ascending order
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
  w.resize(n);
  std::vector<double> Vs(size_t(n) * n);
  for (int k = 0; k < n; ++k) {
    w[k] = d[idx[k]];
    for (int r = 0; r < n; ++r) Vs[size_t(r) * n + k] = V[size_t(r) * n + idx[k]];
  }
  V.swap(Vs);
  for (double x : w)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace mlcc

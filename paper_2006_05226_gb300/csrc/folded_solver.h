// Eigensolver of the folded CC2 Jacobian A_eff(omega) (c1, c_T) = omega (c1, c_T) with
// subspaces kept across omega updates. Plain C++ (header only, no CUDA): the vector space
// and the operator are a template parameter, so the same control logic runs on device
// vectors in the library and on host vectors with a dense operator in the host tests.
//
// Each trial vector b stores A_eff(w_b) b and dA_eff/domega (w_b) b at the omega w_b it was
// applied at; the projected problem at omega uses the first-order model
//   A_eff(omega) b ~ A_eff(w_b) b + (omega - w_b) dA_eff/domega (w_b) b.
// With a column b referred to w_b, the projected model is the linear pencil
// (G0 - G1 W) y + omega G1 y, so its self-consistent pairs are the eigenpairs of
// (I - G1)^-1 (G0 - G1 W): one small eigensolve gives them all.
// Stage 1 (all roots): every vector is applied at one omega_0 (the lowest diagonal element
// of the guesses); the k-th self-consistent eigenvalue of the model is the k-th root;
// new directions are the preconditioned residuals; it stops when every model residual is
// below stage1_tol.
// Stage 2 (each root): a subspace of its own, started from the stage-1 Ritz vector applied
// at omega_k; the Ritz pair of the projected model that overlaps most with the previous one
// is taken; its preconditioned residual, applied at the current omega,
// extends the subspace. Once the model residual is below refresh_tol, omega is known to
// about the square of the residual: vectors applied farther than exact_dw from it are
// dropped and the rest of the Ritz vector is applied exactly at omega, so the model is exact
// (its error is second order in omega - w_b) for the remaining convergence to res_tol. A
// subspace that reaches max_sub collapses onto combinations of its vectors: exact in stage 1
// (one omega); in stage 2 they carry the distance of their sources, and count as inexact.
// A wanted eigenvalue with a non-zero imaginary part (a complex pair of the non-symmetric
// Jacobian) is reported as such (Result::complex_pair) instead of being refined, and two
// roots that settled on the same eigenpair make the solve fail.

#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <vector>

#include "small_eig.h"

namespace mlcc {
namespace fold {

struct Options {
  int n_roots = 3;
  double res_tol = 1e-8;     // model residual norm per root
  double exact_dw = 1e-7;    // |omega - w_b| bound for every subspace vector at convergence
  double stage1_tol = 1e-3;  // model residual norm that ends stage 1
  double refresh_tol = 1e-5; // stage 2: below this model residual an inexact subspace
                             // restarts from the Ritz vector applied exactly at omega
  int max_iter = 200;        // iterations per stage (per root in stage 2)
  int max_sub = 0;           // subspace size limit (0: 8 n_roots, at least 2 n_roots + 4)
  double omega_max = 1e300;  // the lowest P_S denominator: omega must stay below it
};

struct Result {
  std::vector<double> omega;      // ascending
  std::vector<double> residual;   // model residual norm per root at the end
  int n_apply = 0;                // applications of A_eff (each with its derivative)
  int iterations = 0;             // stage 1 plus stage 2 iterations
  bool converged = false;
  bool complex_pair = false;      // a wanted eigenvalue is complex (its real part reported)
  const char* failure = nullptr;  // why not, when not converged
};

// Space requirements (Vec is a value type: copyable, movable):
//   Vec make();                                    zero vector
//   int n_guess();                                 candidate unit start vectors
//   void guess(int k, Vec& v, double& diag);       the k-th lowest-diagonal unit vector
//   double dot(const Vec& x, const Vec& y);
//   void axpy(double a, const Vec& x, Vec& y);     y += a x
//   void scale(double a, Vec& x);
//   void precondition(const Vec& r, double omega, Vec& t);   t = P[(D - omega)^-1 r]
//   void apply(double omega, const Vec& x, Vec& y, Vec& dy); A_eff x and dA_eff/domega x
template <class Space>
class Solver {
 public:
  using Vec = typename Space::Vec;

  Solver(Space& sp, const Options& o) : sp_(sp), o_(o) {
    // stage 1 collapses to 2 n_roots vectors and then adds n_roots, stage 2 restarts on 4:
    // a limit below 3 n_roots (or 2 n_roots + 4) would collapse without progress
    max_sub_ = o.max_sub > 0 ? o.max_sub : 8 * o.n_roots;
    max_sub_ = std::max(max_sub_, std::max(3 * o.n_roots, 2 * o.n_roots + 4));
  }

  // vectors (optional): the folded Ritz vectors of the roots, in the order of res.omega
  Result run(std::vector<Vec>* vectors = nullptr);

 private:
  struct Basis {
    std::vector<Vec> V, S0, S1;
    std::vector<double> w;        // the omega S0 and S1 refer to
    std::vector<double> d;        // 0 if applied exactly at w, else a bound on the distance
                                  // of the first-order combination it came from
    std::vector<double> G0, G1;   // V^T S0, V^T S1, row-major m x m
    int m() const { return int(V.size()); }
  };
  struct Pair {
    double omega = 0.0;
    std::vector<double> y;   // coefficients in the basis
    Vec x, r;
    double rnorm = 0.0;
    double imag = 0.0;       // imaginary part of the model eigenvalue (0 for a real pair)
    bool ok = false;
  };

  Space& sp_;
  Options o_;
  int max_sub_ = 0;
  int n_apply_ = 0;

  // orthonormalises t against the basis (two Gram-Schmidt passes); false if it vanishes
  bool orthonormalise(const Basis& B, Vec& t, double drop) {
    const double n0 = std::sqrt(std::max(0.0, sp_.dot(t, t)));
    if (!(n0 > 0.0)) return false;
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < B.m(); ++i) sp_.axpy(-sp_.dot(B.V[i], t), B.V[i], t);
    const double n1 = std::sqrt(std::max(0.0, sp_.dot(t, t)));
    if (!(n1 > drop * n0)) return false;
    sp_.scale(1.0 / n1, t);
    return true;
  }

  // appends an orthonormal v applied at w, updating the projected matrices
  void append(Basis& B, Vec v, double w) {
    Vec y = sp_.make(), dy = sp_.make();
    sp_.apply(w, v, y, dy);
    ++n_apply_;
    const int m = B.m(), m1 = m + 1;
    std::vector<double> G0(size_t(m1) * m1, 0.0), G1(size_t(m1) * m1, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        G0[size_t(i) * m1 + j] = B.G0[size_t(i) * m + j];
        G1[size_t(i) * m1 + j] = B.G1[size_t(i) * m + j];
      }
    B.V.push_back(std::move(v));
    B.S0.push_back(std::move(y));
    B.S1.push_back(std::move(dy));
    B.w.push_back(w);
    B.d.push_back(0.0);
    for (int i = 0; i < m1; ++i) {
      G0[size_t(i) * m1 + m] = sp_.dot(B.V[i], B.S0[m]);
      G1[size_t(i) * m1 + m] = sp_.dot(B.V[i], B.S1[m]);
      G0[size_t(m) * m1 + i] = sp_.dot(B.V[m], B.S0[i]);
      G1[size_t(m) * m1 + i] = sp_.dot(B.V[m], B.S1[i]);
    }
    B.G0.swap(G0);
    B.G1.swap(G1);
  }

  // a basis of the combinations C (coefficients in B) of B's vectors, all referred to w by
  // the first-order model: v = sum c_b V_b, S0 = sum c_b (S0_b + (w - w_b) S1_b),
  // S1 = sum c_b S1_b; orthonormalised with the same operations on S0 and S1. Exact when
  // every w_b equals w; no applications of the operator
  Basis combine(const Basis& B, const std::vector<std::vector<double>>& C, double w) {
    Basis N;
    for (const auto& c : C) {
      Vec v = sp_.make(), s0 = sp_.make(), s1 = sp_.make();
      double dist = 0.0;
      for (int b = 0; b < B.m() && b < int(c.size()); ++b) {
        if (c[b] == 0.0) continue;
        dist = std::max(dist, std::fabs(w - B.w[b]) + B.d[b]);
        sp_.axpy(c[b], B.V[b], v);
        sp_.axpy(c[b], B.S0[b], s0);
        if (w != B.w[b]) sp_.axpy(c[b] * (w - B.w[b]), B.S1[b], s0);
        sp_.axpy(c[b], B.S1[b], s1);
      }
      const double n0 = std::sqrt(std::max(0.0, sp_.dot(v, v)));
      if (!(n0 > 0.0)) continue;
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < N.m(); ++i) {
          const double a = sp_.dot(N.V[i], v);
          sp_.axpy(-a, N.V[i], v);
          sp_.axpy(-a, N.S0[i], s0);
          sp_.axpy(-a, N.S1[i], s1);
        }
      const double n1 = std::sqrt(std::max(0.0, sp_.dot(v, v)));
      if (!(n1 > 1e-8 * n0)) continue;
      sp_.scale(1.0 / n1, v);
      sp_.scale(1.0 / n1, s0);
      sp_.scale(1.0 / n1, s1);
      N.V.push_back(std::move(v));
      N.S0.push_back(std::move(s0));
      N.S1.push_back(std::move(s1));
      N.w.push_back(w);
      N.d.push_back(dist);   // conservative: the orthonormalisation mixes earlier ones in
    }
    double dmax = 0.0;
    for (double x : N.d) dmax = std::max(dmax, x);
    for (double& x : N.d) x = dmax;
    const int m = N.m();
    N.G0.assign(size_t(m) * m, 0.0);
    N.G1.assign(size_t(m) * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        N.G0[size_t(i) * m + j] = sp_.dot(N.V[i], N.S0[j]);
        N.G1[size_t(i) * m + j] = sp_.dot(N.V[i], N.S1[j]);
      }
    return N;
  }

  // The first-order model of the projected operator is the linear pencil
  //   A(omega) y = (G0 - G1 W) y + omega G1 y,   W = diag(w_b),
  // so its self-consistent pairs A(omega) y = omega y are the eigenpairs of
  //   M = (I - G1)^-1 (G0 - G1 W),
  // found in one small eigensolve (no fixed-point iteration in omega, which can stall on a
  // spurious point where only the real part of a complex pair equals omega). Returns M,
  // or an empty matrix if I - G1 is singular.
  std::vector<double> pencil(const Basis& B) {
    const int m = B.m();
    std::vector<double> IG(size_t(m) * m), R(size_t(m) * m), M(size_t(m) * m);
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        IG[size_t(a) * m + b] = (a == b ? 1.0 : 0.0) - B.G1[size_t(a) * m + b];
        R[size_t(a) * m + b] = B.G0[size_t(a) * m + b] - B.G1[size_t(a) * m + b] * B.w[b];
      }
    std::vector<double> col(m), x;
    for (int b = 0; b < m; ++b) {
      for (int a = 0; a < m; ++a) col[a] = R[size_t(a) * m + b];
      if (!solve_linear(m, IG, col, x)) return {};
      for (int a = 0; a < m; ++a) M[size_t(a) * m + b] = x[a];
    }
    return M;
  }

  // real parts of the model's eigenvectors, ordered by eig_nonsym (ascending real part);
  // empty on failure
  std::vector<std::vector<double>> model_vectors(const Basis& B, std::vector<double>* re) {
    const int m = B.m();
    std::vector<std::vector<double>> out;
    const std::vector<double> M = pencil(B);
    if (M.empty()) return out;
    std::vector<std::complex<double>> lam;
    std::vector<std::vector<std::complex<double>>> Y;
    if (!eig_nonsym(m, M, lam, &Y, m)) return out;
    for (int j = 0; j < m; ++j) {
      std::vector<double> y(m);
      for (int a = 0; a < m; ++a) y[a] = Y[j][a].real();
      out.push_back(std::move(y));
      if (re) re->push_back(lam[j].real());
    }
    return out;
  }

  // the model pair chosen by pick among the self-consistent pairs of the pencil
  Pair model_pair(const Basis& B,
                  const std::function<int(const std::vector<std::complex<double>>&,
                                          const std::vector<std::vector<std::complex<double>>>&)>& pick) {
    Pair p;
    const int m = B.m();
    const std::vector<double> M = pencil(B);
    if (M.empty()) return p;
    std::vector<std::complex<double>> lam;
    std::vector<std::vector<std::complex<double>>> Y;
    if (!eig_nonsym(m, M, lam, &Y, m)) return p;
    const int j = pick(lam, Y);
    if (j < 0) return p;
    const double w = lam[j].real();
    if (!std::isfinite(w) || !(w < o_.omega_max)) return p;
    p.imag = lam[j].imag();
    // Ritz pair (the basis is orthonormal, so |x| = |y|)
    p.y.resize(m);
    double ny = 0.0;
    for (int a = 0; a < m; ++a) {
      p.y[a] = Y[j][a].real();
      ny += p.y[a] * p.y[a];
    }
    ny = std::sqrt(ny);
    if (!(ny > 0.0)) return p;
    for (double& v : p.y) v /= ny;
    p.omega = w;
    p.x = sp_.make();
    p.r = sp_.make();
    for (int a = 0; a < m; ++a) {
      sp_.axpy(p.y[a], B.V[a], p.x);
      sp_.axpy(p.y[a], B.S0[a], p.r);
      sp_.axpy(p.y[a] * (w - B.w[a]), B.S1[a], p.r);
    }
    sp_.axpy(-w, p.x, p.r);
    p.rnorm = std::sqrt(std::max(0.0, sp_.dot(p.r, p.r)));
    p.ok = std::isfinite(p.rnorm);
    return p;
  }
};

template <class Space>
Result Solver<Space>::run(std::vector<Vec>* vectors) {
  Result res;
  const int nr = o_.n_roots;
  const int ng = std::min(2 * nr, sp_.n_guess());
  if (nr < 1 || ng < nr) {
    res.failure = "fewer start vectors than roots";
    res.n_apply = n_apply_;
    return res;
  }
  // stage 1: every vector applied at omega_0
  Basis B;
  double w0 = 0.0;
  for (int k = 0; k < ng; ++k) {
    Vec v = sp_.make();
    double dk = 0.0;
    sp_.guess(k, v, dk);
    if (k == 0) w0 = std::min(dk, 0.5 * o_.omega_max);
    if (orthonormalise(B, v, 1e-10)) append(B, std::move(v), w0);
  }
  std::vector<double> om(nr, w0);
  std::vector<Vec> X(nr);
  bool stage1_done = false;
  for (int it = 0; it < o_.max_iter && !stage1_done; ++it) {
    ++res.iterations;
    std::vector<Pair> P(nr);
    double worst = 0.0;
    for (int k = 0; k < nr; ++k) {
      P[k] = model_pair(B, [k](const std::vector<std::complex<double>>& lam,
                                      const std::vector<std::vector<std::complex<double>>>&) {
        return k < int(lam.size()) ? k : -1;   // eigenvalues come sorted by real part
      });
      if (!P[k].ok) {
        res.failure = "stage 1: no admissible Ritz pair";
        res.n_apply = n_apply_;
        return res;
      }
      om[k] = P[k].omega;
      X[k] = P[k].x;
      worst = std::max(worst, P[k].rnorm);
    }
    if (worst < o_.stage1_tol) {
      stage1_done = true;
      break;
    }
    if (B.m() + nr > max_sub_) {
      // collapse onto the roots' Ritz vectors and the next model eigenvectors (2 n_roots
      // in all); every vector was applied at omega_0, so the combinations are exact
      std::vector<std::vector<double>> C;
      for (int k = 0; k < nr; ++k) C.push_back(P[k].y);
      std::vector<std::vector<double>> extra = model_vectors(B, nullptr);
      for (int j = nr; j < int(extra.size()) && int(C.size()) < 2 * nr; ++j) C.push_back(extra[j]);
      B = combine(B, C, w0);
      continue;
    }
    int added = 0;
    for (int k = 0; k < nr; ++k) {
      Vec t = sp_.make();
      sp_.precondition(P[k].r, om[k], t);
      if (orthonormalise(B, t, 1e-10)) {
        append(B, std::move(t), w0);
        ++added;
      }
    }
    if (added == 0) stage1_done = true;   // invariant subspace: the model pairs are final
  }
  if (!stage1_done) {
    res.failure = "stage 1 did not converge";
    res.n_apply = n_apply_;
    return res;
  }
  // stage 2: one root at a time
  res.omega.assign(nr, 0.0);
  res.residual.assign(nr, 0.0);
  std::vector<Vec> xs;   // the roots' folded Ritz vectors
  bool all = true;
  for (int k = 0; k < nr; ++k) {
    double w = om[k];
    Basis R;
    std::vector<double> yprev;
    auto restart = [&](Vec x, double wr) {
      R = Basis();
      const double nx = std::sqrt(std::max(0.0, sp_.dot(x, x)));
      sp_.scale(1.0 / nx, x);
      append(R, std::move(x), wr);
      yprev.assign(1, 1.0);
    };
    restart(X[k], w);
    bool done = false, cplx = false;
    int n_complex = 0;   // consecutive iterations whose chosen model eigenvalue is complex
    Pair p;
    for (int it = 0; it < o_.max_iter; ++it) {
      ++res.iterations;
      const std::vector<double> prev = yprev;
      p = model_pair(R, [&prev](const std::vector<std::complex<double>>& lam,
                                   const std::vector<std::vector<std::complex<double>>>& Y) {
        // homing: the Ritz vector with the largest overlap with the previous one
        int best = -1;
        double bo = -1.0;
        for (int j = 0; j < int(lam.size()); ++j) {
          double ov = 0.0, nrm = 0.0;
          for (size_t a = 0; a < Y[j].size(); ++a) {
            nrm += std::norm(Y[j][a]);
            if (a < prev.size()) ov += Y[j][a].real() * prev[a];
          }
          const double s = nrm > 0.0 ? std::fabs(ov) / std::sqrt(nrm) : 0.0;
          if (s > bo) {
            bo = s;
            best = j;
          }
        }
        return best;
      });
      if (!p.ok) break;
      w = p.omega;
      // a complex pair of the Jacobian: its real part is a fixed point of the model but no
      // real eigenvector exists there, so the residual cannot fall below |Im|
      n_complex = std::fabs(p.imag) > std::max(o_.res_tol, 1e-6 * std::fabs(w)) ? n_complex + 1 : 0;
      if (n_complex >= 3) {
        cplx = true;
        break;
      }
      if (p.rnorm < std::max(o_.res_tol, o_.refresh_tol)) {
        double dw = 0.0;
        for (int b = 0; b < R.m(); ++b) dw = std::max(dw, std::fabs(w - R.w[b]) + R.d[b]);
        // the first-order model errs by about (omega - w_b)^2 |d2A/domega2|; refer the subspace
        // to omega only when that could matter at the present residual (|omega - w_b| above
        // 0.1 sqrt(|r|)), and exactly (within exact_dw) before accepting convergence, so the
        // subspace is not rebuilt at every small move of omega
        const double allow = p.rnorm < o_.res_tol ? o_.exact_dw
                                                  : std::max(o_.exact_dw, 0.1 * std::sqrt(p.rnorm));
        if (dw >= allow) {
          // omega is now known to about the square of the residual: refer the subspace to
          // it exactly, so that the rest of the convergence uses an exact model. Vectors
          // applied within exact_dw of omega stay; the rest of the Ritz vector is applied
          // exactly at omega
          std::vector<std::vector<double>> C;
          for (int b = 0; b < R.m(); ++b)
            if (std::fabs(w - R.w[b]) + R.d[b] < o_.exact_dw) {
              std::vector<double> e(R.m(), 0.0);
              e[b] = 1.0;
              C.push_back(std::move(e));
            }
          Basis K = combine(R, C, w);
          Vec t = p.x;
          if (orthonormalise(K, t, 1e-10)) append(K, std::move(t), w);
          if (K.m() == 0) {
            restart(p.x, w);
            continue;
          }
          R = std::move(K);
          yprev.assign(R.m(), 0.0);
          for (int b = 0; b < R.m(); ++b) yprev[b] = sp_.dot(R.V[b], p.x);
          continue;
        }
        if (p.rnorm < o_.res_tol) {
          done = true;
          break;
        }
      }
      if (R.m() >= max_sub_) {
        // thick restart: the Ritz vector and the three model eigenvectors whose values lie
        // nearest omega, referred to omega by the first-order model (no applications)
        std::vector<double> re;
        std::vector<std::vector<double>> ev = model_vectors(R, &re);
        std::vector<int> idx(ev.size());
        for (size_t j = 0; j < idx.size(); ++j) idx[j] = int(j);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return std::fabs(re[a] - w) < std::fabs(re[b] - w); });
        std::vector<std::vector<double>> C{p.y};
        for (int j : idx) {
          if (C.size() >= 4) break;
          C.push_back(ev[j]);
        }
        R = combine(R, C, w);
        yprev.assign(R.m(), 0.0);
        yprev[0] = 1.0;
        continue;
      }
      Vec t = sp_.make();
      sp_.precondition(p.r, w, t);
      if (!orthonormalise(R, t, 1e-12)) {
        restart(p.x, w);
        continue;
      }
      append(R, std::move(t), w);
      yprev = p.y;
      yprev.push_back(0.0);
    }
    res.omega[k] = w;
    res.residual[k] = p.ok ? p.rnorm : INFINITY;
    xs.push_back(p.ok ? p.x : sp_.make());
    if (cplx) {
      all = false;
      res.complex_pair = true;
      if (!res.failure) res.failure = "a wanted eigenvalue is complex (a complex pair of the Jacobian)";
    } else if (!done) {
      all = false;
      if (!res.failure) res.failure = p.ok ? "stage 2 did not converge" : "stage 2: no admissible Ritz pair";
    }
  }
  // two roots that settled on the same eigenpair (equal omega, parallel vectors) would
  // hide a root: refuse them
  if (all) {
    for (int a = 0; a < nr && all; ++a)
      for (int b = a + 1; b < nr && all; ++b) {
        if (std::fabs(res.omega[a] - res.omega[b]) > 1e-6 * std::max(1.0, std::fabs(res.omega[a]))) continue;
        const Vec& xa = xs[a];
        const Vec& xb = xs[b];
        const double na = sp_.dot(xa, xa), nb = sp_.dot(xb, xb);
        const double c = na > 0.0 && nb > 0.0 ? std::fabs(sp_.dot(xa, xb)) / std::sqrt(na * nb) : 1.0;
        if (c > 0.99) {
          all = false;
          res.failure = "two roots settled on the same eigenpair";
        }
      }
  }
  // ascending order (vectors alongside)
  std::vector<int> idx(nr);
  for (int k = 0; k < nr; ++k) idx[k] = k;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return res.omega[a] < res.omega[b]; });
  std::vector<double> so(nr), sr(nr);
  for (int k = 0; k < nr; ++k) {
    so[k] = res.omega[idx[k]];
    sr[k] = res.residual[idx[k]];
  }
  res.omega.swap(so);
  res.residual.swap(sr);
  if (vectors) {
    vectors->clear();
    for (int k = 0; k < nr; ++k) vectors->push_back(std::move(xs[idx[k]]));
  }
  res.n_apply = n_apply_;
  res.converged = all;
  return res;
}

}  // namespace fold
}  // namespace mlcc

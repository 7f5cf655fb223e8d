// Host-side small dense solvers used by the DIIS and Davidson control loops.
#pragma once
#include <complex>
#include <vector>

namespace mlcc {
// Solves A x = b (row-major n x n) by Gaussian elimination with partial pivoting.
bool solve_linear(int n, std::vector<double> A, std::vector<double> b, std::vector<double>& x);
// Eigenvalues of a real non-symmetric n x n matrix (row-major), sorted by real part, and
// right eigenvectors of the first n_vecs of them.
bool eig_nonsym(int n, const std::vector<double>& A, std::vector<std::complex<double>>& w,
                std::vector<std::vector<std::complex<double>>>* vecs, int n_vecs);
// Eigenpairs of a real symmetric n x n matrix (row-major): w ascending, V row-major with
// column k the unit eigenvector of w[k]. Householder tridiagonalisation with the
// transformations accumulated, then the implicit QL iteration with Wilkinson-type shifts.
bool eig_sym(int n, const std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);
}  // namespace mlcc

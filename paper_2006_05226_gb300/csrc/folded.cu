// Folded CC2 Jacobian (the CC2 response strategy that Sec. 2.1 points to): in the
// three-level model the P_S doubles rows of the Jacobian have a diagonal doubles block
// (eps_aibj, Appendix A sigma^MLCC2_aibj) and no coupling to P_T, so an eigenvector's P_S
// part is c_S(omega) = (omega - eps_S)^-1 A_S1 c1 and (c1, c_T) solves
//   A_eff(omega) (c1, c_T) = omega (c1, c_T),
//   A_eff(omega) = [[A_11 + A_1S (omega - eps_S)^-1 A_S1, A_1T], [A_T1, A_TT]].
// sigma_eff applies A_eff(omega) with two partial Jacobian transformations: sigma(c1, 0)
// without its doubles-to-singles and CCSD parts gives A_S1 c1 on the P_S rows;
// sigma(c1, c_S(omega) + c_T) without its P_S rows gives the singles and P_T rows. The
// omega-derivative dA_eff/domega (c1, c_T) = (-A_1S (omega - eps_S)^-2 A_S1 c1, 0) is the
// singles part of sigma(0, x_S) with x_S = -(A_S1 c1) / (omega - eps_S)^2, of which only
// the doubles-to-singles part is evaluated. Each part runs one Cholesky-rank GEMM.
#include "system.cuh"

#include <algorithm>

namespace mlcc {
namespace {

inline int nblk(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16384))); }

__device__ __forceinline__ void split4f(int64_t t, int sv, int so, int& a, int& i, int& b, int& j) {
  j = int(t % so);
  t /= so;
  b = int(t % sv);
  t /= sv;
  i = int(t % so);
  a = int(t / so);
}

// doubles of the second transformation and of the derivative direction:
//   P_T: c2 (the caller's P_T amplitudes), derivative direction 0;
//   P_S: r2 / (omega - eps_aibj) and -r2 / (omega - eps_aibj)^2.
__global__ void k_fold_doubles(const double* __restrict__ r2, const double* __restrict__ c2,
                               const double* __restrict__ eps, int no, int sv, int so, int tv, int to,
                               double omega, double* __restrict__ cs, double* __restrict__ xs) {
  const int64_t total = int64_t(sv) * so * sv * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int a, i, b, j;
    split4f(t, sv, so, a, i, b, j);
    if (a < tv && i < to && b < tv && j < to) {
      cs[t] = c2[t];
      xs[t] = 0.0;
    } else {
      const double den = omega - (eps[no + a] - eps[i] + eps[no + b] - eps[j]);
      const double q = r2[t] / den;
      cs[t] = q;
      xs[t] = -q / den;
    }
  }
}

// keeps the P_T rows of the doubles, zeroes the P_S rows
__global__ void k_keep_T(double* __restrict__ s2, int sv, int so, int tv, int to) {
  const int64_t total = int64_t(sv) * so * sv * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int a, i, b, j;
    split4f(t, sv, so, a, i, b, j);
    if (!(a < tv && i < to && b < tv && j < to)) s2[t] = 0.0;
  }
}

}  // namespace

// lowest eps_aibj over the P_S pairs: (ai) outside the CCSD pairs with any (bj), or the
// reverse (eps_aibj = eps_ai + eps_bj); +inf without P_S pairs
double lowest_ps_denominator(const mlcc_system* S) {
  const int no = S->no, so = S->so, sv = S->sv, to = S->to, tv = S->tv;
  double min_all = 1e300, min_out = 1e300;
  for (int a = 0; a < sv; ++a)
    for (int i = 0; i < so; ++i) {
      const double e = S->eps_host[no + a] - S->eps_host[i];
      min_all = std::min(min_all, e);
      if (!(a < tv && i < to)) min_out = std::min(min_out, e);
    }
  if (min_out >= 1e300) return 1e300;
  return min_out + min_all;
}

void sigma_eff_eval(mlcc_system* S, const double* c, double omega, double* out, double* dout, int precision,
                    double* w0, double* w1, double* w2) {
  cudaStream_t s = S->ctx->stream;
  const int no = S->no, nv = S->nv, sv = S->sv, so = S->so, tv = S->tv, to = S->to;
  const int64_t n1 = int64_t(nv) * no, nd = S->nd;
  // w0 = (c1, 0); w1 = sigma(c1, 0)
  MLCC_CUDA(cudaMemcpyAsync(w0, c, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
  if (nd) MLCC_CUDA(cudaMemsetAsync(w0 + n1, 0, size_t(nd) * 8, s));
  sigma_eval(S, w0, w1, precision, SIGMA_CC2_DOUBLES);   // only its P_S rows are read
  // w0 doubles = c_S(omega) + c_T; w2 doubles = derivative direction x_S
  if (nd) {
    k_fold_doubles<<<nblk(nd), 256, 0, s>>>(w1 + n1, c + n1, S->eps, no, sv, so, tv, to, omega, w0 + n1, w2 + n1);
    MLCC_CHECK_LAUNCH();
  }
  sigma_eval(S, w0, out, precision, SIGMA_DOUBLES_TO_SINGLES | SIGMA_CCSD_ROWS);
  if (nd) {
    k_keep_T<<<nblk(nd), 256, 0, s>>>(out + n1, sv, so, tv, to);
    MLCC_CHECK_LAUNCH();
  }
  if (dout) {
    // (0, x_S): its singles are A_1S x_S
    MLCC_CUDA(cudaMemsetAsync(w2, 0, size_t(n1) * 8, s));
    sigma_eval(S, w2, w1, precision, SIGMA_DOUBLES_TO_SINGLES);
    MLCC_CUDA(cudaMemcpyAsync(dout, w1, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace mlcc

// Correlated natural transition orbitals (Sec. 2.2): the orbital rotations that select the
// active spaces of a multilevel calculation from CCS excitation vectors.
//
//  1. CCS states: the Davidson solve of the all-CCS system (at the Hartree-Fock reference
//     its Jacobian is the CIS matrix), singles vectors R normalised to unit 2-norm.
//  2. Approximate doubles (Eqs. approx_double_1 and approx_double_2):
//       A^J_ai  = sum_c L^J_ac R_ci - sum_k R_ak L^J_ki            (batched GEMMs over J)
//       gbar    = sum_J (A^J_ai L^J_bj + L^J_ai A^J_bj)              (rank-N_J GEMM pair)
//       R_aibj  = -gbar_aibj / ((1 + delta_{ai,bj}) (eps_a + eps_b - eps_i - eps_j - omega))
//     A^J is the t1-derivative of the dressed L~_vo along R, so gbar is the matching
//     derivative of g~_aibj.
//  3. Eqs. M and N, summed over the states. With the symmetry R_aibj = R_bjai, every row r
//     of R2 (a pair bk) reshaped to X_r [N_v][N_o] gives
//       M += 1/2 sum_r X_r^T X_r,      N += 1/2 sum_r X_r X_r^T
//     (batched reduce GEMMs), plus the (1 + delta) diagonal terms and R1^T R1, R1 R1^T.
//     R2 is therefore built and consumed in blocks of rows: its N_v N_o x N_v N_o size
//     never has to be held at once.
//  4. Host eigensolver (eig_sym) for M and N; eigenvalues descending.
#include "system.cuh"
#include "small_eig.h"

#include <algorithm>
#include <cmath>

namespace mlcc {
namespace {

inline int nblk_c(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16384))); }

// Lvo[J][a * no + i] = L^J[no + a][i]
__global__ void k_pack_vo(const double* __restrict__ L, int n, int no, int nj, double* __restrict__ Lvo) {
  const int nv = n - no;
  const int64_t d = int64_t(nv) * no, total = d * nj;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t J = t / d, r = t - J * d;
    const int a = int(r / no), i = int(r - int64_t(a) * no);
    Lvo[t] = L[(J * n + no + a) * n + i];
  }
}

// rows [r0, r0 + rows) of R2 = -gbar / ((1 + delta) (eps_r + eps_q - omega)) in place, and
// the squares of the diagonal elements R2[r][r] into diag2[r - r0]
__global__ void k_cnto_doubles(double* __restrict__ G, int64_t r0, int64_t rows, int64_t d, int no,
                               const double* __restrict__ eps, double omega, double* __restrict__ diag2) {
  const int64_t total = rows * d;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t rr = t / d, q = t - rr * d, r = r0 + rr;
    const int a = int(r / no), i = int(r - int64_t(a) * no);
    const int b = int(q / no), j = int(q - int64_t(b) * no);
    const double den = eps[no + a] - eps[i] + eps[no + b] - eps[j] - omega;
    double v = -G[t] / den;
    if (q == r) {
      v *= 0.5;
      diag2[rr] = v * v;
    }
    G[t] = v;
  }
}

// M[i][i] += 1/2 sum_a diag2[a * no + i] and N[a][a] += 1/2 sum_i diag2[a * no + i] over the
// rows of one block (pairs r = a * no + i in [r0, r0 + rows)); one thread per orbital
__global__ void k_cnto_diag(const double* __restrict__ diag2, int64_t r0, int64_t rows, int no, int nv,
                            double* __restrict__ M, double* __restrict__ N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < no) {
    double s = 0.0;
    for (int a = 0; a < nv; ++a) {
      const int64_t r = int64_t(a) * no + t;
      if (r >= r0 && r < r0 + rows) s += diag2[r - r0];
    }
    M[int64_t(t) * no + t] += 0.5 * s;
  } else if (t < no + nv) {
    const int a = t - no;
    double s = 0.0;
    for (int i = 0; i < no; ++i) {
      const int64_t r = int64_t(a) * no + i;
      if (r >= r0 && r < r0 + rows) s += diag2[r - r0];
    }
    N[int64_t(a) * nv + a] += 0.5 * s;
  }
}

}  // namespace

// The whole construction; host outputs in res. precision: mlcc_precision of the large GEMMs.
mlcc_status cnto_build(mlcc_ctx* ctx, int n, int no, int nj, const double* chol, const double* fock,
                       int n_states, int precision, mlcc_cnto_result* res) {
  cudaStream_t s = ctx->stream;
  const int nv = n - no;
  const int64_t d = int64_t(nv) * no, nn = int64_t(n) * n;
  // 1. CCS states
  std::vector<int8_t> lev(static_cast<size_t>(n), static_cast<int8_t>(MLCC_LEVEL_CCS));
  mlcc_problem prob{n, no, nj, lev.data()};
  mlcc_system* S = nullptr;
  mlcc_status st = mlcc_system_create(ctx, &prob, chol, fock, &S);
  if (st != MLCC_OK) return st;
  struct Sys { mlcc_system* s; ~Sys() { mlcc_system_destroy(s); } } sg{S};
  MLCC_REQUIRE(S->rot.empty(), "mlcc_cnto: the Fock matrix must be diagonal (canonical orbitals)");
  for (int k = 0; k < n; ++k) MLCC_REQUIRE(S->perm[k] == k, "mlcc_cnto: internal orbital order differs");
  mlcc_options opt;
  mlcc_default_options(&opt);
  opt.n_roots = n_states;
  opt.es_res_tol = 1e-11;
  Arena work;
  const int64_t rows = res->block_rows > 0
                           ? std::min<int64_t>(d, res->block_rows)
                           : std::max<int64_t>(1, std::min<int64_t>(d, std::max<int64_t>(64, (int64_t(1) << 24) / std::max<int64_t>(d, 1))));
  const size_t scratch = (size_t(256) << 20) + size_t(24) * size_t(rows + d) * size_t(2 * nj + 64) +
                         size_t(64) * size_t(rows) * 256 * 4;
  work.reserve(size_t(n_states + 1) * d * 8 + size_t(2) * nj * d * 8 + size_t(rows) * d * 8 + size_t(rows) * 8 +
               size_t(no) * no * 8 + size_t(nv) * nv * 8 + size_t(n) * 8 + 16 * 256 + scratch);
  double* R = work.get<double>(size_t(n_states) * d);
  {
    mlcc_gs_info gi{};
    double* t1 = work.get<double>(size_t(d));
    double* x2 = work.get<double>(1);
    st = mlcc_ground_state(S, &opt, t1, x2, &gi);
    if (st != MLCC_OK) return st;
    mlcc_es_info ei{};
    st = mlcc_excited_states(S, &opt, res->omega, R, &ei);
    if (st != MLCC_OK) return st;
  }
  // 2.-3. approximate doubles and M, N in row blocks
  double* A = work.get<double>(size_t(nj) * d);
  double* Lvo = work.get<double>(size_t(nj) * d);
  double* G = work.get<double>(size_t(rows) * d);
  double* diag2 = work.get<double>(size_t(rows));
  double* M = work.get<double>(size_t(no) * no);
  double* N = work.get<double>(size_t(nv) * nv);
  fill(M, int64_t(no) * no, 0.0, s);
  fill(N, int64_t(nv) * nv, 0.0, s);
  k_pack_vo<<<nblk_c(d * nj), 256, 0, s>>>(S->L, n, no, nj, Lvo);
  MLCC_CHECK_LAUNCH();
  for (int k = 0; k < n_states; ++k) {
    const double* Rk = R + int64_t(k) * d;
    LowpScope lowp(precision == MLCC_FP64 ? 0 : precision, S->tc_err);
    // A^J = L^J_vv R - R L^J_oo
    Gemm g1;
    g1.M = nv; g1.N = no; g1.K = nv;
    g1.A = S->L + int64_t(no) * n + no; g1.lda = n; g1.sA = nn;
    g1.B = Rk; g1.ldb = no; g1.sB = 0;
    g1.C = A; g1.ldc = no; g1.sC = d;
    g1.batch = nj;
    gemm_f64(g1, work, s, ctx->sm_count);
    Gemm g2;
    g2.M = nv; g2.N = no; g2.K = no;
    g2.alpha = -1.0; g2.beta = 1.0;
    g2.A = Rk; g2.lda = no; g2.sA = 0;
    g2.B = S->L; g2.ldb = n; g2.sB = nn;
    g2.C = A; g2.ldc = no; g2.sC = d;
    g2.batch = nj;
    gemm_f64(g2, work, s, ctx->sm_count);
    // singles parts: M += R1^T R1, N += R1 R1^T
    Gemm m1;
    m1.ta = true; m1.M = no; m1.N = no; m1.K = nv; m1.beta = 1.0;
    m1.A = Rk; m1.lda = no; m1.B = Rk; m1.ldb = no; m1.C = M; m1.ldc = no;
    gemm_f64(m1, work, s, ctx->sm_count);
    Gemm n1;
    n1.tb = true; n1.M = nv; n1.N = nv; n1.K = no; n1.beta = 1.0;
    n1.A = Rk; n1.lda = no; n1.B = Rk; n1.ldb = no; n1.C = N; n1.ldc = nv;
    gemm_f64(n1, work, s, ctx->sm_count);
    for (int64_t r0 = 0; r0 < d; r0 += rows) {
      const int64_t nr = std::min(rows, d - r0);
      // gbar rows: A^T Lvo + Lvo^T A over J
      Gemm ga;
      ga.ta = true; ga.M = nr; ga.N = d; ga.K = nj;
      ga.A = A + r0; ga.lda = d; ga.B = Lvo; ga.ldb = d; ga.C = G; ga.ldc = d;
      ga.b_const = true;
      gemm_f64(ga, work, s, ctx->sm_count);
      Gemm gb = ga;
      gb.A = Lvo + r0; gb.B = A; gb.beta = 1.0;
      gb.b_const = false; gb.a_const = true;
      gemm_f64(gb, work, s, ctx->sm_count);
      k_cnto_doubles<<<nblk_c(nr * d), 256, 0, s>>>(G, r0, nr, d, no, S->eps, res->omega[k], diag2);
      MLCC_CHECK_LAUNCH();
      // M += 1/2 sum_r X_r^T X_r, N += 1/2 sum_r X_r X_r^T, X_r = row r as [nv][no]
      Gemm gm;
      gm.reduce = true; gm.batch = nr;
      gm.ta = true; gm.M = no; gm.N = no; gm.K = nv; gm.alpha = 0.5; gm.beta = 1.0;
      gm.A = G; gm.lda = no; gm.sA = d; gm.B = G; gm.ldb = no; gm.sB = d; gm.C = M; gm.ldc = no;
      gemm_f64(gm, work, s, ctx->sm_count);
      Gemm gn;
      gn.reduce = true; gn.batch = nr;
      gn.tb = true; gn.M = nv; gn.N = nv; gn.K = no; gn.alpha = 0.5; gn.beta = 1.0;
      gn.A = G; gn.lda = no; gn.sA = d; gn.B = G; gn.ldb = no; gn.sB = d; gn.C = N; gn.ldc = nv;
      gemm_f64(gn, work, s, ctx->sm_count);
      k_cnto_diag<<<(no + nv + 255) / 256, 256, 0, s>>>(diag2, r0, nr, no, nv, M, N);
      MLCC_CHECK_LAUNCH();
    }
    if (precision != MLCC_FP64) check_tc_error(S);
  }
  // 4. eigenpairs on the host, descending
  std::vector<double> Mh(size_t(no) * no), Nh(size_t(nv) * nv);
  copy_d2h(Mh.data(), M, int64_t(no) * no, s);
  copy_d2h(Nh.data(), N, int64_t(nv) * nv, s);
  MLCC_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < no; ++i)   // exact symmetry (the two triangles summed in other orders)
    for (int j = 0; j < i; ++j) Mh[size_t(i) * no + j] = Mh[size_t(j) * no + i] = 0.5 * (Mh[size_t(i) * no + j] + Mh[size_t(j) * no + i]);
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < a; ++b) Nh[size_t(a) * nv + b] = Nh[size_t(b) * nv + a] = 0.5 * (Nh[size_t(a) * nv + b] + Nh[size_t(b) * nv + a]);
  if (res->m) std::copy(Mh.begin(), Mh.end(), res->m);
  if (res->n) std::copy(Nh.begin(), Nh.end(), res->n);
  auto eig_desc = [](int m, const std::vector<double>& X, double* vals, double* vecs) {
    std::vector<double> w, V;
    if (!eig_sym(m, X, w, V)) throw Error(MLCC_E_CUDA, "mlcc_cnto: host eigensolver failed");
    for (int k = 0; k < m; ++k) {
      vals[k] = w[size_t(m - 1 - k)];
      if (vecs) {
        // column k of the output: eigenvector m-1-k, largest-magnitude component positive
        int big = 0;
        for (int p = 1; p < m; ++p)
          if (std::fabs(V[size_t(p) * m + (m - 1 - k)]) > std::fabs(V[size_t(big) * m + (m - 1 - k)])) big = p;
        const double sg = V[size_t(big) * m + (m - 1 - k)] < 0.0 ? -1.0 : 1.0;
        for (int p = 0; p < m; ++p) vecs[size_t(p) * m + k] = sg * V[size_t(p) * m + (m - 1 - k)];
      }
    }
  };
  eig_desc(no, Mh, res->occ_values, res->occ_vectors);
  eig_desc(nv, Nh, res->vir_values, res->vir_vectors);
  if (res->n_vir_active <= 0) {
    // Eq. select_CNTOs: n_v^a = (N_v / N_o) n_o^a, rounded to the nearest integer
    const double x = double(nv) / double(no) * double(res->n_occ_active);
    res->n_vir_active = int32_t(std::min<double>(nv, std::max(1.0, std::floor(x + 0.5))));
  }
  return MLCC_OK;
}

}  // namespace mlcc

using namespace mlcc;

extern "C" mlcc_status mlcc_cnto(mlcc_ctx* ctx, int32_t n_mo, int32_t n_occ, int32_t n_chol,
                                 const double* chol_dev, const double* fock_dev, int32_t n_states,
                                 int32_t precision, mlcc_cnto_result* res) {
  return guard([&] {
    MLCC_REQUIRE(ctx && chol_dev && fock_dev && res && res->omega && res->occ_values && res->vir_values,
                 "mlcc_cnto: NULL argument");
    MLCC_REQUIRE(n_mo > 0 && n_occ > 0 && n_occ < n_mo && n_chol > 0, "mlcc_cnto: need 0 < n_occ < n_mo, n_chol > 0");
    MLCC_REQUIRE(n_states >= 1 && 2 * int64_t(n_states) <= int64_t(n_occ) * (n_mo - n_occ),
                 "mlcc_cnto: need 1 <= n_states and 2 n_states <= n_occ n_vir");
    MLCC_REQUIRE(res->n_occ_active >= 1 && res->n_occ_active <= n_occ, "mlcc_cnto: n_occ_active in [1, n_occ]");
    MLCC_REQUIRE(res->n_vir_active <= n_mo - n_occ, "mlcc_cnto: n_vir_active above n_vir");
    MLCC_REQUIRE(res->block_rows >= 0, "mlcc_cnto: block_rows must not be negative");
    MLCC_REQUIRE(precision == MLCC_FP64 || precision == MLCC_FP64E || is_split_precision(precision),
                 "mlcc_cnto: unknown precision");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    return cnto_build(ctx, n_mo, n_occ, n_chol, chol_dev, fock_dev, n_states, precision, res);
  });
}

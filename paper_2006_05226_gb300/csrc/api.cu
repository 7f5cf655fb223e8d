// C ABI of libmlcc (declared in include/mlcc.h): argument validation, system set-up
// (orbital re-ordering, recovery of the one-electron matrix of Sec. 2.3) and the
// exception-to-status boundary.
#include "system.cuh"
#include "small_eig.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

namespace mlcc {
const char* last_error_cstr();
int64_t launch_count();
mlcc_status ground_state(mlcc_system* S, const mlcc_options* opt, double* t1_out, double* x2_out,
                         mlcc_gs_info* info);
mlcc_status excited_states(mlcc_system* S, const mlcc_options* opt, double* omega_host,
                           double* r_out, mlcc_es_info* info, double* residual_host = nullptr,
                           bool left = false);

// the Davidson solve behind mlcc_excited_states and mlcc_solve, with their argument checks
static mlcc_status excited_states_checked(mlcc_system* S, const mlcc_options* opt, double* omega, double* r,
                                          mlcc_es_info* info, double* residual, bool left = false) {
  MLCC_REQUIRE(S && opt && omega, "mlcc_excited_states: NULL argument");
  MLCC_REQUIRE(opt->precision >= MLCC_FP64 && opt->precision <= MLCC_FP64E,
               "mlcc_excited_states: unknown precision");
  MLCC_REQUIRE(opt->refine_precision == MLCC_FP64 || opt->refine_precision == MLCC_FP64E,
               "mlcc_excited_states: refine_precision must be MLCC_FP64 or MLCC_FP64E");
  MLCC_CUDA(cudaSetDevice(S->ctx->device));
  const mlcc_status st = excited_states(S, opt, omega, r, info, residual, left);
  if (st == MLCC_E_ES_NOCONV) set_last_error("excited states did not converge");
  if (st == MLCC_E_COMPLEX_ROOT) set_last_error("a wanted Ritz value is complex");
  return st;
}

namespace {
__global__ void k_reorder(const double* src, const int* perm, int n, int64_t batch, double* dst) {
  const int64_t nn = int64_t(n) * n, total = nn * batch;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t J = t / nn, r = t - J * nn;
    const int p = int(r / n), q = int(r - int64_t(p) * n);
    dst[t] = src[J * nn + int64_t(perm[p]) * n + perm[q]];
  }
}
// max_J,p,q |X[J][p][q] - X[J][q][p]| as an order-preserving integer (values >= 0)
__global__ void k_asym(const double* X, int n, int64_t batch, unsigned long long* out) {
  const int64_t nn = int64_t(n) * n, total = nn * batch;
  double m = 0.0;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t J = t / nn, r = t - J * nn;
    const int p = int(r / n), q = int(r - int64_t(p) * n);
    const double d = fabs(X[t] - X[J * nn + int64_t(q) * n + p]);
    m = (d > m || d != d) ? (d != d ? 1e308 : d) : m;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
__global__ void k_diag(const double* F, int n, double* eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) eps[p] = F[int64_t(p) * n + p];
}
}  // namespace

static void setup_system(mlcc_system* S, const mlcc_problem* P, const double* chol, const double* fock) {
  cudaStream_t s = S->ctx->stream;
  const int n = P->n_mo, no = P->n_occ, nj = P->n_chol;
  S->n = n;
  S->no = no;
  S->nv = n - no;
  S->nj = nj;
  // level-ordered permutation: occupied [CCSD, CC2-only, CCS], then virtual likewise
  S->perm.clear();
  int cnt[2][3] = {{0, 0, 0}, {0, 0, 0}};
  for (int part = 0; part < 2; ++part) {
    const int lo = part == 0 ? 0 : no, hi = part == 0 ? no : n;
    for (int lev = 2; lev >= 0; --lev)
      for (int p = lo; p < hi; ++p)
        if (P->level[p] == lev) {
          S->perm.push_back(p);
          ++cnt[part][lev];
        }
  }
  S->to = cnt[0][2];
  S->tv = cnt[1][2];
  S->so = cnt[0][2] + cnt[0][1];
  S->sv = cnt[1][2] + cnt[1][1];
  S->dS = int64_t(S->sv) * S->so;
  S->nd = S->dS * S->dS;
  const int64_t nn = int64_t(n) * n, dS = S->dS;
  // persistent buffers
  const sizes::Dims dims = sys_dims(S);
  {
    const int64_t need = int64_t(sizes::persist_bytes(dims) + sizes::ws_bytes(dims));
    mlcc_ctx* c = S->ctx;
    if (c->budget > 0 && c->held.load() + need > c->budget)
      throw Error(MLCC_E_OOM, "mlcc_system_create: the system needs " + std::to_string(need) +
                                  " bytes; the context's budget leaves " +
                                  std::to_string(c->budget - c->held.load()));
  }
  S->persist.reserve(sizes::persist_bytes(dims));
  S->L = S->persist.get<double>(size_t(nj) * nn);
  S->Lt = S->persist.get<double>(size_t(nj) * nn);
  S->h = S->persist.get<double>(nn);
  S->ht = S->persist.get<double>(nn);
  S->Ft = S->persist.get<double>(nn);
  S->eps = S->persist.get<double>(n);
  S->Lai = S->persist.get<double>(size_t(nj) * dS);
  S->Lov = S->persist.get<double>(size_t(nj) * dS);
  S->Z = S->persist.get<double>(size_t(nj) * dS);
  S->u = S->persist.get<double>(size_t(S->nd));
  S->x2gs = S->persist.get<double>(size_t(S->nd));
  S->Fov = S->persist.get<double>(size_t(dS));
  S->t1gs = S->persist.get<double>(size_t(S->nv) * no);
  S->Xji = S->persist.get<double>(size_t(no) * S->so + 1);
  S->Yab = S->persist.get<double>(size_t(S->sv) * S->nv + 1);
  S->tc_err = S->persist.get<int>(64);
  S->opcache = operand_cache_new();
  MLCC_CUDA(cudaMemsetAsync(S->tc_err, 0, 256, s));
  // scratch: enough for sigma (dLt, three doubles-sized arrays, two [nj][dS]) plus GEMM
  // partials and the einsum engine's permuted operands
  S->ws.reserve(sizes::ws_bytes(dims));
  S->workspace_bytes = int64_t(S->persist.capacity() + S->ws.capacity());
  // re-ordered copies of L and F
  int* dperm = S->ws.get<int>(size_t(n));
  MLCC_CUDA(cudaMemcpyAsync(dperm, S->perm.data(), size_t(n) * 4, cudaMemcpyHostToDevice, s));
  {
    const int64_t total = nn * nj;
    const int blocks = int(std::min<int64_t>((total + 255) / 256, 16384));
    k_reorder<<<blocks, 256, 0, s>>>(chol, dperm, n, nj, S->L);
    MLCC_CHECK_LAUNCH();
    k_reorder<<<int(std::min<int64_t>((nn + 255) / 256, 16384)), 256, 0, s>>>(fock, dperm, n, 1, S->ht);
    MLCC_CHECK_LAUNCH();
  }
  // checks: symmetric L and F
  unsigned long long* asym = S->ws.get<unsigned long long>(1);
  MLCC_CUDA(cudaMemsetAsync(asym, 0, 8, s));
  k_asym<<<1024, 256, 0, s>>>(S->L, n, nj, asym);
  MLCC_CHECK_LAUNCH();
  unsigned long long ah = 0;
  MLCC_CUDA(cudaMemcpyAsync(&ah, asym, 8, cudaMemcpyDeviceToHost, s));
  std::vector<double> Fh(static_cast<size_t>(nn));
  MLCC_CUDA(cudaMemcpyAsync(Fh.data(), S->ht, size_t(nn) * 8, cudaMemcpyDeviceToHost, s));
  MLCC_CUDA(cudaStreamSynchronize(s));
  double amax;
  std::memcpy(&amax, &ah, 8);
  if (!(amax <= 1e-10)) throw Error(MLCC_E_ARG, "Cholesky vectors are not symmetric in pq (max asymmetry " + std::to_string(amax) + ")");
  double fmax = 0.0;
  for (int p = 0; p < n; ++p) fmax = std::max(fmax, std::fabs(Fh[size_t(p) * n + p]));
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      const double a = Fh[size_t(p) * n + q], b = Fh[size_t(q) * n + p];
      if (!std::isfinite(a)) throw Error(MLCC_E_NAN, "Fock matrix has NaN or Inf");
      if (std::fabs(a - b) > 1e-10 * std::max(1.0, fmax)) throw Error(MLCC_E_ARG, "Fock matrix is not symmetric");
    }
  // Semicanonical basis (Sec. 2.1-2.2): the CC2 doubles equations use only the orbital
  // energies, so the Fock matrix must be diagonal inside each level's occupied and virtual
  // blocks. Blocks that are not are diagonalised here, and the Cholesky vectors and F are
  // rotated with them (an orbital rotation inside a level leaves the model unchanged);
  // couplings between levels stay and enter through F~.
  {
    const int bounds[7] = {0, S->to, S->so, no, no + S->tv, no + S->sv, n};
    std::vector<double> U;
    for (int b = 0; b < 6; ++b) {
      const int lo = bounds[b], hi = bounds[b + 1], m = hi - lo;
      if (m < 2) continue;
      double off = 0.0;
      for (int p = lo; p < hi; ++p)
        for (int q = lo; q < hi; ++q)
          if (p != q) off = std::max(off, std::fabs(Fh[size_t(p) * n + q]));
      if (off <= 1e-12 * std::max(1.0, fmax)) continue;
      std::vector<double> blk(size_t(m) * m), wb, Vb;
      for (int p = 0; p < m; ++p)
        for (int q = 0; q < m; ++q) blk[size_t(p) * m + q] = 0.5 * (Fh[size_t(lo + p) * n + lo + q] + Fh[size_t(lo + q) * n + lo + p]);
      if (!eig_sym(m, blk, wb, Vb)) throw Error(MLCC_E_ARG, "semicanonicalisation: eigensolver failed");
      for (int k = 0; k < m; ++k) {   // sign: largest-magnitude component positive
        int big = 0;
        for (int p = 1; p < m; ++p)
          if (std::fabs(Vb[size_t(p) * m + k]) > std::fabs(Vb[size_t(big) * m + k])) big = p;
        if (Vb[size_t(big) * m + k] < 0.0)
          for (int p = 0; p < m; ++p) Vb[size_t(p) * m + k] = -Vb[size_t(p) * m + k];
      }
      if (U.empty()) {
        U.assign(size_t(nn), 0.0);
        for (int p = 0; p < n; ++p) U[size_t(p) * n + p] = 1.0;
      }
      for (int p = 0; p < m; ++p)
        for (int q = 0; q < m; ++q) U[size_t(lo + p) * n + lo + q] = Vb[size_t(p) * m + q];
    }
    if (!U.empty()) {
      // F <- U^T F U on the host; L^J <- U^T L^J U on the device (binary64), through Lt
      std::vector<double> T(size_t(nn), 0.0), F2(size_t(nn), 0.0);
      for (int p = 0; p < n; ++p)
        for (int r = 0; r < n; ++r) {
          const double f = Fh[size_t(p) * n + r];
          if (f == 0.0) continue;
          for (int q = 0; q < n; ++q) T[size_t(p) * n + q] += f * U[size_t(r) * n + q];
        }
      for (int r = 0; r < n; ++r)
        for (int p = 0; p < n; ++p) {
          const double u = U[size_t(r) * n + p];
          if (u == 0.0) continue;
          for (int q = 0; q < n; ++q) F2[size_t(p) * n + q] += u * T[size_t(r) * n + q];
        }
      for (int p = 0; p < n; ++p)   // exact zeros inside the rotated blocks, symmetric
        for (int q = 0; q < p; ++q) F2[size_t(p) * n + q] = F2[size_t(q) * n + p] = 0.5 * (F2[size_t(p) * n + q] + F2[size_t(q) * n + p]);
      for (int b = 0; b < 6; ++b)
        for (int p = bounds[b]; p < bounds[b + 1]; ++p)
          for (int q = bounds[b]; q < bounds[b + 1]; ++q)
            if (p != q) F2[size_t(p) * n + q] = 0.0;
      Fh.swap(F2);
      Scope sc(S->ws);
      double* dU = S->ws.get<double>(size_t(nn));
      copy_h2d(dU, U.data(), nn, s);
      copy_h2d(S->ht, Fh.data(), nn, s);
      Gemm g1;   // Lt[J] = L[J] U
      g1.M = g1.N = g1.K = n;
      g1.A = S->L; g1.lda = n; g1.sA = nn;
      g1.B = dU; g1.ldb = n; g1.sB = 0;
      g1.C = S->Lt; g1.ldc = n; g1.sC = nn;
      g1.batch = nj;
      gemm_f64(g1, S->ws, s, S->ctx->sm_count);
      Gemm g2;   // L[J] = U^T Lt[J]
      g2.ta = true;
      g2.M = g2.N = g2.K = n;
      g2.A = dU; g2.lda = n; g2.sA = 0;
      g2.B = S->Lt; g2.ldb = n; g2.sB = nn;
      g2.C = S->L; g2.ldc = n; g2.sC = nn;
      g2.batch = nj;
      gemm_f64(g2, S->ws, s, S->ctx->sm_count);
      MLCC_CUDA(cudaStreamSynchronize(s));
      S->rot.swap(U);
    }
  }
  S->eps_host.resize(n);
  for (int p = 0; p < n; ++p) S->eps_host[p] = Fh[size_t(p) * n + p];
  k_diag<<<(n + 255) / 256, 256, 0, s>>>(S->ht, n, S->eps);
  MLCC_CHECK_LAUNCH();
  // h = F - sum_J [2 L^J (sum_i L^J_ii) - L^J[:, i] L^J[i, :]]   (Eq. eff_fock)
  MLCC_CUDA(cudaMemcpyAsync(S->h, S->ht, size_t(nn) * 8, cudaMemcpyDeviceToDevice, s));
  {
    // reuse build_fock with the sign flipped: F(h=0) then h = F - F(h=0)
    Scope sc(S->ws);
    double* zero = S->ws.get<double>(size_t(nn));
    double* G = S->ws.get<double>(size_t(nn));
    fill(zero, nn, 0.0, s);
    build_fock(S, zero, S->L, G);
    axpby(S->h, G, nn, -1.0, 1.0, s);
  }
  MLCC_CUDA(cudaStreamSynchronize(s));
  S->prepared = false;
}

}  // namespace mlcc

using namespace mlcc;

// ground state and excited states of a system built from device inputs; inputs_done runs
// once the system holds its own copies
static mlcc_status solve_from_device(mlcc_ctx* ctx, const mlcc_problem* prob, const double* dL,
                                     const double* dF, std::function<void()> inputs_done,
                                     const mlcc_options* opt, mlcc_result* res, bool host_out);

extern "C" {

void mlcc_default_options(mlcc_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_roots = 3;
  o->max_gs_iter = 200;
  o->max_es_iter = 200;
  o->diis_dim = 8;
  o->max_subspace = 0;
  o->precision = MLCC_FP64;
  o->refine_fp64 = 1;
  o->gs_precision = MLCC_FP64;
  o->gs_tol = 1e-11;
  o->gs_energy_tol = 1e-12;
  o->es_res_tol = 1e-8;
  o->es_omega_tol = 1e-11;
  o->lowp_res_tol = 1e-4;
  o->refine_precision = MLCC_FP64;
}

const char* mlcc_last_error(void) { return last_error_cstr(); }

mlcc_status mlcc_ctx_create(int device, mlcc_ctx** out) { return mlcc_ctx_create_budget(device, 0, out); }

mlcc_status mlcc_ctx_create_budget(int device, int64_t hbm_budget_bytes, mlcc_ctx** out) {
  return guard([&] {
    MLCC_REQUIRE(out != nullptr, "mlcc_ctx_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    MLCC_CUDA(cudaGetDeviceCount(&ndev));
    MLCC_REQUIRE(device >= 0 && device < ndev, "mlcc_ctx_create: no such CUDA device");
    MLCC_CUDA(cudaSetDevice(device));
    auto* c = new mlcc_ctx();
    c->device = device;
    c->budget = std::max<int64_t>(hbm_budget_bytes, 0);
    MLCC_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    MLCC_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    *out = c;
    return MLCC_OK;
  });
}

void mlcc_ctx_destroy(mlcc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->timer.reset();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int64_t mlcc_launch_count(void) { return launch_count(); }

void* mlcc_ctx_stream(mlcc_ctx* ctx) { return ctx ? static_cast<void*>(ctx->stream) : nullptr; }

void mlcc_kernel_timing(mlcc_ctx* ctx, int enable) {
  if (!ctx) return;
  ctx->timer.reset();
  ctx->timer.enabled = enable != 0;
}

mlcc_status mlcc_kernel_time(mlcc_ctx* ctx, const char* family, int64_t* launches,
                             double* total_ms, double* total_flop) {
  return guard([&] {
    MLCC_REQUIRE(ctx && family, "mlcc_kernel_time: NULL argument");
    MLCC_CUDA(cudaStreamSynchronize(ctx->stream));
    int64_t n = 0;
    double ms = 0.0, fl = 0.0;
    auto it = ctx->timer.recs.find(family);
    if (it != ctx->timer.recs.end()) {
      for (auto& r : it->second) {
        float t = 0.f;
        MLCC_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        fl += r.flop;
        ++n;
      }
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    if (total_flop) *total_flop = fl;
    return MLCC_OK;
  });
}

mlcc_status mlcc_system_create(mlcc_ctx* ctx, const mlcc_problem* prob, const double* chol_dev,
                               const double* fock_dev, mlcc_system** out) {
  return guard([&] {
    MLCC_REQUIRE(ctx && prob && out && chol_dev && fock_dev, "mlcc_system_create: NULL argument");
    *out = nullptr;
    MLCC_REQUIRE(prob->level != nullptr, "mlcc_system_create: level is NULL");
    MLCC_REQUIRE(prob->n_mo > 0 && prob->n_occ > 0 && prob->n_occ < prob->n_mo,
                 "mlcc_system_create: need 0 < n_occ < n_mo");
    MLCC_REQUIRE(prob->n_chol > 0, "mlcc_system_create: n_chol must be positive");
    for (int p = 0; p < prob->n_mo; ++p)
      MLCC_REQUIRE(prob->level[p] >= 0 && prob->level[p] <= 2, "mlcc_system_create: level must be 0, 1 or 2");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    auto* S = new mlcc_system();
    S->ctx = ctx;
    try {
      setup_system(S, prob, chol_dev, fock_dev);
    } catch (...) {
      delete S;
      throw;
    }
    ctx->held += S->workspace_bytes;
    *out = S;
    return MLCC_OK;
  });
}

void mlcc_system_destroy(mlcc_system* sys) {
  if (!sys) return;
  sys->ctx->held -= sys->workspace_bytes;
  cudaSetDevice(sys->ctx->device);
  cudaStreamSynchronize(sys->ctx->stream);
  sigma_graphs_free(sys);
  ccsd_cache_free(sys);
  operand_cache_free(sys->opcache);
  delete sys;
}

mlcc_status mlcc_system_info(const mlcc_system* S, mlcc_dims* d) {
  return guard([&] {
    MLCC_REQUIRE(S && d, "mlcc_system_info: NULL argument");
    d->n_occ = S->no;
    d->n_vir = S->nv;
    d->s_occ = S->so;
    d->s_vir = S->sv;
    d->t_occ = S->to;
    d->t_vir = S->tv;
    d->n_singles = int64_t(S->nv) * S->no;
    d->n_doubles = S->nd;
    d->vector_len = d->n_singles + d->n_doubles;
    d->workspace_bytes = S->workspace_bytes;
    return MLCC_OK;
  });
}

mlcc_status mlcc_orbital_order(const mlcc_system* S, int32_t* perm) {
  return guard([&] {
    MLCC_REQUIRE(S && perm, "mlcc_orbital_order: NULL argument");
    std::copy(S->perm.begin(), S->perm.end(), perm);
    return MLCC_OK;
  });
}

mlcc_status mlcc_orbitals(const mlcc_system* S, double* c) {
  return guard([&] {
    MLCC_REQUIRE(S && c, "mlcc_orbitals: NULL argument");
    const int n = S->n;
    std::fill(c, c + size_t(n) * n, 0.0);
    // system orbital k = sum_k' rot[k'][k] (re-ordered orbital k'), re-ordered k' = caller perm[k']
    for (int kp = 0; kp < n; ++kp)
      for (int k = 0; k < n; ++k) {
        const double u = S->rot.empty() ? (kp == k ? 1.0 : 0.0) : S->rot[size_t(kp) * n + k];
        if (u != 0.0) c[size_t(S->perm[kp]) * n + k] = u;
      }
    return MLCC_OK;
  });
}

mlcc_status mlcc_t1_transform(mlcc_system* S, const double* t1, double* lt) {
  return guard([&] {
    MLCC_REQUIRE(S && t1 && lt, "mlcc_t1_transform: NULL argument");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    S->prepared = false;
    sigma_graphs_free(S);
    operand_cache_clear(S->opcache);
    dress(S, t1, lt, nullptr);
    return MLCC_OK;
  });
}

mlcc_status mlcc_fock_t1(mlcc_system* S, const double* t1, double* f) {
  return guard([&] {
    MLCC_REQUIRE(S && t1 && f, "mlcc_fock_t1: NULL argument");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    S->prepared = false;
    sigma_graphs_free(S);
    operand_cache_clear(S->opcache);
    dress(S, t1, S->Lt, S->ht);
    build_fock(S, S->ht, S->Lt, f);
    return MLCC_OK;
  });
}

mlcc_status mlcc_omega(mlcc_system* S, const double* t1, const double* x2, double* om1,
                       double* om2, double* energy) {
  return guard([&] {
    MLCC_REQUIRE(S && t1 && om1, "mlcc_omega: NULL argument");
    MLCC_REQUIRE(S->nd == 0 || (x2 && om2), "mlcc_omega: doubles buffers required");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    omega_eval(S, t1, x2, false, nullptr, nullptr, om1, om2, energy);
    return MLCC_OK;
  });
}

mlcc_status mlcc_ground_state(mlcc_system* S, const mlcc_options* opt, double* t1, double* x2,
                              mlcc_gs_info* info) {
  return guard([&] {
    MLCC_REQUIRE(S && opt && t1, "mlcc_ground_state: NULL argument");
    MLCC_REQUIRE(S->nd == 0 || x2, "mlcc_ground_state: x2 buffer required");
    MLCC_REQUIRE(opt->max_gs_iter >= 1 && opt->diis_dim >= 1, "mlcc_ground_state: bad options");
    MLCC_REQUIRE(opt->gs_precision >= MLCC_FP64 && opt->gs_precision <= MLCC_FP64E,
                 "mlcc_ground_state: unknown gs_precision");
    MLCC_REQUIRE(opt->refine_precision == MLCC_FP64 || opt->refine_precision == MLCC_FP64E,
                 "mlcc_ground_state: refine_precision must be MLCC_FP64 or MLCC_FP64E");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    mlcc_gs_info local{};
    mlcc_status st = ground_state(S, opt, t1, x2, info ? info : &local);
    if (info) {
      double e_hf = 0.0;
      std::vector<double> h(static_cast<size_t>(S->n) * S->n);
      copy_d2h(h.data(), S->h, int64_t(S->n) * S->n, S->ctx->stream);
      for (int i = 0; i < S->no; ++i) e_hf += h[size_t(i) * S->n + i] + S->eps_host[i];
      info->e_hf = e_hf;
    }
    if (st == MLCC_E_GS_NOCONV) set_last_error("ground state did not converge");
    return st;
  });
}

mlcc_status mlcc_jacobian_prepare(mlcc_system* S, const double* t1, const double* x2) {
  return guard([&] {
    MLCC_REQUIRE(S && t1 && (S->nd == 0 || x2), "mlcc_jacobian_prepare: NULL argument");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    jacobian_prepare(S, t1, x2);
    return MLCC_OK;
  });
}

mlcc_status mlcc_sigma(mlcc_system* S, int32_t n_vec, const double* c, double* sigma,
                       int32_t precision) {
  return guard([&] {
    MLCC_REQUIRE(S && c && sigma, "mlcc_sigma: NULL argument");
    MLCC_REQUIRE(n_vec >= 0, "mlcc_sigma: n_vec < 0");
    MLCC_REQUIRE(precision >= MLCC_FP64 && precision <= MLCC_FP64E, "mlcc_sigma: unknown precision");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    const int64_t len = int64_t(S->nv) * S->no + S->nd;
    for (int k = 0; k < n_vec; ++k) sigma_eval(S, c + k * len, sigma + k * len, precision);
    if (precision != MLCC_FP64) check_tc_error(S);
    return MLCC_OK;
  });
}

// Restricts a prepared system to the Cholesky vectors [j0, j1) for the duration of a
// sharded Jacobian transformation: the J-indexed buffers are offset, nj shrinks, and the
// converted-operand caches (which cover every J) are bypassed.
namespace {
struct JWindow {
  mlcc_system* S;
  int nj;
  double *Lt, *Lai, *Lov, *Z;
  OperandCache* oc;
  JWindow(mlcc_system* s, int j0, int j1) : S(s), nj(s->nj), Lt(s->Lt), Lai(s->Lai), Lov(s->Lov), Z(s->Z), oc(s->opcache) {
    const int64_t nn = int64_t(S->n) * S->n;
    S->Lt += int64_t(j0) * nn;
    S->Lai += int64_t(j0) * S->dS;
    S->Lov += int64_t(j0) * S->dS;
    S->Z += int64_t(j0) * S->dS;
    S->nj = j1 - j0;
    S->jwin = true;
    S->jwin0 = j0;
    S->opcache = nullptr;
  }
  ~JWindow() {
    S->Lt = Lt; S->Lai = Lai; S->Lov = Lov; S->Z = Z;
    S->nj = nj;
    S->jwin = false;
    S->jwin0 = 0;
    S->opcache = oc;
  }
};
}  // namespace

mlcc_status mlcc_sigma_partial(mlcc_system* S, int32_t j_begin, int32_t j_end, int32_t with_rest,
                               int32_t n_vec, const double* c, double* sigma, int32_t precision) {
  return guard([&] {
    MLCC_REQUIRE(S && c && sigma, "mlcc_sigma_partial: NULL argument");
    MLCC_REQUIRE(n_vec >= 0, "mlcc_sigma_partial: n_vec < 0");
    MLCC_REQUIRE(0 <= j_begin && j_begin < j_end && j_end <= S->nj,
                 "mlcc_sigma_partial: need 0 <= j_begin < j_end <= n_chol");
    MLCC_REQUIRE(precision >= MLCC_FP64 && precision <= MLCC_FP64E, "mlcc_sigma_partial: unknown precision");
    if (!S->prepared) throw Error(MLCC_E_STATE, "mlcc_sigma_partial: call mlcc_jacobian_prepare first");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    const int64_t len = int64_t(S->nv) * S->no + S->nd;
    {
      JWindow w(S, j_begin, j_end);
      const unsigned parts = SIGMA_ALL | (with_rest ? 0u : unsigned(SIGMA_J_ONLY));
      for (int k = 0; k < n_vec; ++k) sigma_eval(S, c + k * len, sigma + k * len, precision, parts);
    }
    if (precision != MLCC_FP64) check_tc_error(S);
    return MLCC_OK;
  });
}

namespace {
// <x_k, y_k> for k < nv vectors of length n (device), to the host
std::vector<double> pair_dots(mlcc_system* S, const double* x, const double* y, int nv, int64_t n) {
  std::vector<double> out(size_t(std::max(nv, 0)));
  Scope sc(S->ws);
  double* d = S->ws.get<double>(1);
  for (int k = 0; k < nv; ++k) {
    dots(x + int64_t(k) * n, 0, 1, y + int64_t(k) * n, n, d, S->ws, S->ctx->stream);
    copy_d2h(&out[size_t(k)], d, 1, S->ctx->stream);
  }
  return out;
}
}  // namespace

mlcc_status mlcc_sigma_left(mlcc_system* S, int32_t n_vec, const double* l, double* rho, int32_t precision) {
  return guard([&] {
    MLCC_REQUIRE(S && l && rho, "mlcc_sigma_left: NULL argument");
    MLCC_REQUIRE(n_vec >= 0, "mlcc_sigma_left: n_vec < 0");
    MLCC_REQUIRE(precision >= MLCC_FP64 && precision <= MLCC_FP64E, "mlcc_sigma_left: unknown precision");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    const int64_t len = int64_t(S->nv) * S->no + S->nd;
    for (int k = 0; k < n_vec; ++k) sigma_left_eval(S, l + k * len, rho + k * len, precision);
    if (precision != MLCC_FP64) check_tc_error(S);
    return MLCC_OK;
  });
}

mlcc_status mlcc_excited_states_left(mlcc_system* S, const mlcc_options* opt, double* omega, double* l_dev,
                                     const double* r_dev, mlcc_es_info* info) {
  return guard([&] {
    MLCC_REQUIRE(S && opt && omega && l_dev, "mlcc_excited_states_left: NULL argument");
    if (S->to > 0 && S->tv > 0)
      throw Error(MLCC_E_ARG, "mlcc_excited_states_left: systems with a CCSD level are not supported");
    const mlcc_status st = excited_states_checked(S, opt, omega, l_dev, info, nullptr, true);
    if (st != MLCC_OK) return st;
    if (r_dev) {
      // biorthonormal pair: <l_k, r_k> = 1
      const int64_t len = int64_t(S->nv) * S->no + S->nd;
      const std::vector<double> ov = pair_dots(S, l_dev, r_dev, opt->n_roots, len);
      for (int k = 0; k < opt->n_roots; ++k) {
        if (!(std::fabs(ov[size_t(k)]) > 1e-12))
          throw Error(MLCC_E_ES_NOCONV, "mlcc_excited_states_left: a left vector is orthogonal to its right vector");
        axpby(l_dev + k * len, l_dev + k * len, len, 0.0, 1.0 / ov[size_t(k)], S->ctx->stream);
      }
      MLCC_CUDA(cudaStreamSynchronize(S->ctx->stream));
    }
    return MLCC_OK;
  });
}

mlcc_status mlcc_fold_window(const mlcc_system* S, double* omega_max) {
  return guard([&] {
    MLCC_REQUIRE(S && omega_max, "mlcc_fold_window: NULL argument");
    *omega_max = lowest_ps_denominator(S);
    return MLCC_OK;
  });
}

mlcc_status mlcc_sigma_eff(mlcc_system* S, int32_t n_vec, const double* omega, const double* c,
                           double* sigma, double* dsigma, int32_t precision) {
  return guard([&] {
    MLCC_REQUIRE(S && (n_vec == 0 || (omega && c && sigma)), "mlcc_sigma_eff: NULL argument");
    MLCC_REQUIRE(n_vec >= 0, "mlcc_sigma_eff: n_vec < 0");
    MLCC_REQUIRE(precision >= MLCC_FP64 && precision <= MLCC_FP64E, "mlcc_sigma_eff: unknown precision");
    if (!S->prepared) throw Error(MLCC_E_STATE, "mlcc_sigma_eff: call mlcc_jacobian_prepare first");
    const double top = lowest_ps_denominator(S);
    for (int k = 0; k < n_vec; ++k)
      MLCC_REQUIRE(std::isfinite(omega[k]) && omega[k] < top,
                   "mlcc_sigma_eff: omega must lie below the lowest P_S denominator");
    if (n_vec == 0) return MLCC_OK;
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    const int64_t n1 = int64_t(S->nv) * S->no, len = n1 + S->nd;
    Arena w;
    w.reserve(size_t(3) * len * 8 + 3 * 256);
    double* w0 = w.get<double>(len);
    double* w1 = w.get<double>(len);
    double* w2 = w.get<double>(len);
    for (int k = 0; k < n_vec; ++k)
      sigma_eff_eval(S, c + k * len, omega[k], sigma + k * len, dsigma ? dsigma + k * n1 : nullptr, precision,
                     w0, w1, w2);
    if (precision != MLCC_FP64) check_tc_error(S);
    MLCC_CUDA(cudaStreamSynchronize(S->ctx->stream));   // the scratch is freed on return
    return MLCC_OK;
  });
}

mlcc_status mlcc_excited_states_folded(mlcc_system* S, const mlcc_options* opt, double* omega,
                                       double* r, mlcc_es_info* info) {
  return guard([&] {
    MLCC_REQUIRE(S && opt && omega, "mlcc_excited_states_folded: NULL argument");
    MLCC_REQUIRE(opt->precision == MLCC_FP64 || opt->precision == MLCC_FP64E,
                 "mlcc_excited_states_folded: precision must be MLCC_FP64 or MLCC_FP64E");
    MLCC_REQUIRE(opt->max_es_iter >= 1, "mlcc_excited_states_folded: bad options");
    MLCC_CUDA(cudaSetDevice(S->ctx->device));
    return excited_states_folded(S, opt, omega, r, info);
  });
}

mlcc_status mlcc_excited_states(mlcc_system* S, const mlcc_options* opt, double* omega,
                                double* r, mlcc_es_info* info) {
  return guard([&] { return excited_states_checked(S, opt, omega, r, info, nullptr); });
}

mlcc_status mlcc_gemm(mlcc_ctx* ctx, int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K,
                      double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double beta, double* C, int64_t ldc, int32_t precision) {
  return guard([&] {
    MLCC_REQUIRE(ctx != nullptr, "mlcc_gemm: NULL context");
    MLCC_REQUIRE(M >= 0 && N >= 0 && K >= 0, "mlcc_gemm: negative size");
    MLCC_REQUIRE(precision >= MLCC_FP64 && precision <= MLCC_FP64E, "mlcc_gemm: unknown precision");
    if (M == 0 || N == 0) return MLCC_OK;
    MLCC_REQUIRE(C && (K == 0 || (A && B)), "mlcc_gemm: NULL matrix");
    MLCC_REQUIRE(ldc >= N && lda >= (trans_a ? M : K) && ldb >= (trans_b ? K : N) && lda >= 1 && ldb >= 1,
                 "mlcc_gemm: leading dimension too small");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    Gemm g;
    g.ta = trans_a != 0;
    g.tb = trans_b != 0;
    g.M = M; g.N = N; g.K = K;
    g.alpha = alpha; g.beta = beta;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    // scratch for this call: converted operands plus partial sums (split-K, or the
    // emulation's chunk planes, bounded by panelling over the output columns)
    const int64_t Kp = (K + 63) / 64 * 64;
    size_t bytes = (size_t(1) << 30) + (size_t(64) << 20);
    if (precision != MLCC_FP64) bytes += size_t(M + N) * 8 * Kp * 2 + size_t(M + N) * 4;
    Arena ws;
    ws.reserve(bytes);
    Arena flag;
    flag.reserve(256);
    int* err = flag.get<int>(1);
    MLCC_CUDA(cudaMemsetAsync(err, 0, 4, s));
    if (precision == MLCC_FP64) {
      gemm_f64(g, ws, s, ctx->sm_count);
    } else if (precision == MLCC_FP64E) {
      MLCC_REQUIRE(gemm_emu(g, ws, s, ctx->sm_count, err),
                   "mlcc_gemm: shape outside the MLCC_FP64E tensor-core path (M, N >= 16, K <= 2^20)");
    } else {
      MLCC_REQUIRE(K > 0 && gemm_tc(g, precision, ws, s, ctx->sm_count, err),
                   "mlcc_gemm: shape outside the tensor-core path");
    }
    int h = 0;
    MLCC_CUDA(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, s));
    MLCC_CUDA(cudaStreamSynchronize(s));
    if (h != 0) throw Error(MLCC_E_TIMEOUT, "mlcc_gemm: a tensor-core pipeline wait timed out");
    return MLCC_OK;
  });
}

// a whole solve must fit the context's budget next to the systems it already holds
static void check_solve_budget(mlcc_ctx* ctx, const mlcc_problem* prob, const mlcc_options* opt) {
  if (ctx->budget <= 0) return;
  int64_t fp = 0;
  const mlcc_status st = mlcc_solve_footprint(prob, opt, &fp);
  if (st != MLCC_OK) throw Error(st, mlcc_last_error());
  if (ctx->held.load() + fp > ctx->budget)
    throw Error(MLCC_E_OOM, "mlcc_solve: the solve holds up to " + std::to_string(fp) +
                                " bytes; the context's budget leaves " + std::to_string(ctx->budget - ctx->held.load()));
}

mlcc_status mlcc_solve(mlcc_ctx* ctx, const mlcc_problem* prob, const double* chol_host,
                       const double* fock_host, const mlcc_options* opt, mlcc_result* res) {
  return guard([&] {
    MLCC_REQUIRE(ctx && prob && chol_host && fock_host && opt && res && res->omega, "mlcc_solve: NULL argument");
    MLCC_REQUIRE(prob->n_mo > 0 && prob->n_chol > 0, "mlcc_solve: sizes must be positive");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    check_solve_budget(ctx, prob, opt);
    const int64_t nn = int64_t(prob->n_mo) * prob->n_mo;
    double *dL = nullptr, *dF = nullptr;
    struct Free {
      double** a; double** b;
      ~Free() { if (*a) cudaFree(*a); if (*b) cudaFree(*b); }
    } fr{&dL, &dF};
    MLCC_CUDA(cudaMalloc(&dL, size_t(nn) * prob->n_chol * 8));
    MLCC_CUDA(cudaMalloc(&dF, size_t(nn) * 8));
    MLCC_CUDA(cudaMemcpyAsync(dL, chol_host, size_t(nn) * prob->n_chol * 8, cudaMemcpyHostToDevice, ctx->stream));
    MLCC_CUDA(cudaMemcpyAsync(dF, fock_host, size_t(nn) * 8, cudaMemcpyHostToDevice, ctx->stream));
    // the copies go once the system holds its own re-ordered inputs
    auto release = [&] {
      cudaFree(dL); dL = nullptr;
      cudaFree(dF); dF = nullptr;
    };
    return solve_from_device(ctx, prob, dL, dF, release, opt, res, true);
  });
}

mlcc_status mlcc_solve_device(mlcc_ctx* ctx, const mlcc_problem* prob, const double* chol_dev,
                              const double* fock_dev, const mlcc_options* opt, mlcc_result* res) {
  return guard([&] {
    MLCC_REQUIRE(ctx && prob && chol_dev && fock_dev && opt && res && res->omega, "mlcc_solve_device: NULL argument");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    check_solve_budget(ctx, prob, opt);
    return solve_from_device(ctx, prob, chol_dev, fock_dev, nullptr, opt, res, false);
  });
}

int64_t mlcc_vector_len(const mlcc_problem* prob) {
  sizes::Dims d;
  if (!prob || !sizes::dims_from_levels(prob->n_mo, prob->n_occ, prob->n_chol, prob->level, &d)) return -1;
  return d.vector_len();
}

}  // extern "C"

static mlcc_status solve_from_device(mlcc_ctx* ctx, const mlcc_problem* prob, const double* dL,
                                     const double* dF, std::function<void()> inputs_done,
                                     const mlcc_options* opt, mlcc_result* res, bool host_out) {
  mlcc_system* S = nullptr;
  mlcc_status st = mlcc_system_create(ctx, prob, dL, dF, &S);
  if (st != MLCC_OK) return st;
  struct Sys { mlcc_system* s; ~Sys() { mlcc_system_destroy(s); } } sg{S};
  if (inputs_done) inputs_done();
  if (res->perm) std::copy(S->perm.begin(), S->perm.end(), res->perm);
  if (res->orbitals) {
    st = mlcc_orbitals(S, res->orbitals);
    if (st != MLCC_OK) return st;
  }
  const int64_t n1 = int64_t(S->nv) * S->no, dim = n1 + S->nd;
  double *t1 = nullptr, *x2 = nullptr;
  MLCC_CUDA(cudaMalloc(&t1, size_t(n1) * 8 + 8));
  struct Free1 { double* a; ~Free1() { cudaFree(a); } } f1{t1};
  MLCC_CUDA(cudaMalloc(&x2, size_t(S->nd) * 8 + 8));
  struct Free2 { double* a; ~Free2() { cudaFree(a); } } f2{x2};
  mlcc_gs_info gi{};
  const mlcc_status gst = mlcc_ground_state(S, opt, t1, x2, &gi);
  res->gs = gi;
  auto out = [&](double* dst, const double* src, int64_t count) {
    if (!dst || count <= 0) return;
    if (host_out) copy_d2h(dst, src, count, ctx->stream);
    else MLCC_CUDA(cudaMemcpyAsync(dst, src, size_t(count) * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  };
  out(res->t1, t1, n1);
  out(res->x2, x2, S->nd);
  if (gst != MLCC_OK) {
    MLCC_CUDA(cudaStreamSynchronize(ctx->stream));
    return gst;
  }
  // eigenvectors into the caller's device buffer directly, or through a device copy
  double* rdev = nullptr;
  struct Free3 { double* a; ~Free3() { if (a) cudaFree(a); } } f3{nullptr};
  if (res->r) {
    if (host_out) {
      MLCC_CUDA(cudaMalloc(&rdev, size_t(opt->n_roots) * dim * 8));
      f3.a = rdev;
    } else {
      rdev = res->r;
    }
  }
  mlcc_es_info ei{};
  st = excited_states_checked(S, opt, res->omega, rdev, &ei, res->residual);
  res->es = ei;
  if (res->r && host_out) copy_d2h(res->r, rdev, int64_t(opt->n_roots) * dim, ctx->stream);
  MLCC_CUDA(cudaStreamSynchronize(ctx->stream));
  return st;
}

// Excitation energies from the folded CC2 Jacobian on the device: the control logic of
// folded_solver.h on folded vectors (singles [n_vir][n_occ] followed by the CCSD-block
// doubles [t_vir][t_occ][t_vir][t_occ]), with A_eff(omega) and its omega-derivative from
// sigma_eff_eval (folded.cu). The doubles outside the CCSD block never enter the subspace:
// a folded vector holds n_vir n_occ + (t_vir t_occ)^2 elements instead of the full
// n_vir n_occ + (s_vir s_occ)^2.
#include "system.cuh"
#include "folded_solver.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <utility>

namespace mlcc {
namespace {

inline int nblk_f(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16384))); }

// CCSD-block doubles [tv][to][tv][to] <-> full doubles [sv][so][sv][so] (CCSD orbitals lead)
__global__ void k_box_gather(const double* __restrict__ full, int sv, int so, int tv, int to,
                             double* __restrict__ box) {
  const int64_t total = int64_t(tv) * to * tv * to;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int64_t q = t;
    const int j = int(q % to); q /= to;
    const int b = int(q % tv); q /= tv;
    const int i = int(q % to);
    const int a = int(q / to);
    box[t] = full[((int64_t(a) * so + i) * sv + b) * so + j];
  }
}
__global__ void k_box_scatter(const double* __restrict__ box, int sv, int so, int tv, int to,
                              double* __restrict__ full) {
  const int64_t total = int64_t(tv) * to * tv * to;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int64_t q = t;
    const int j = int(q % to); q /= to;
    const int b = int(q % tv); q /= tv;
    const int i = int(q % to);
    const int a = int(q / to);
    full[((int64_t(a) * so + i) * sv + b) * so + j] = box[t];
  }
}

// t = (D - omega)^-1 r on a folded vector, D = eps_a - eps_i on the singles and eps_aibj on
// the CCSD block, whose part is symmetrised under (ai) <-> (bj) first; |D - omega| is kept
// at least 1e-8
__global__ void k_fold_precondition(const double* __restrict__ r, const double* __restrict__ eps, int no,
                                    int nv, int tv, int to, double omega, double* __restrict__ t) {
  const int64_t n1 = int64_t(nv) * no, tl = int64_t(tv) * to * tv * to, total = n1 + tl;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < total;
       k += int64_t(gridDim.x) * blockDim.x) {
    double num, d;
    if (k < n1) {
      const int A = int(k / no), I = int(k - int64_t(A) * no);
      num = r[k];
      d = eps[no + A] - eps[I];
    } else {
      int64_t q = k - n1;
      const int j = int(q % to); q /= to;
      const int b = int(q % tv); q /= tv;
      const int i = int(q % to);
      const int a = int(q / to);
      const int64_t sw = ((int64_t(b) * to + j) * tv + a) * to + i;
      num = 0.5 * (r[k] + r[n1 + sw]);
      d = eps[no + a] - eps[i] + eps[no + b] - eps[j];
    }
    double den = d - omega;
    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
    t[k] = num / den;
  }
}

// largest |x| (first index on ties): candidates per block, then one block
__device__ __forceinline__ void take(double& bv, long long& bi, double v, long long i) {
  if (v > bv || (v == bv && i < bi)) {
    bv = v;
    bi = i;
  }
}
__global__ void k_absmax_blocks(const double* x, int64_t n, double* pv, long long* pi) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double bv = -1.0;
  long long bi = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    take(bv, bi, fabs(x[i]), i);
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double v = sv[threadIdx.x];
      long long ii = si[threadIdx.x];
      take(v, ii, sv[threadIdx.x + w], si[threadIdx.x + w]);
      sv[threadIdx.x] = v;
      si[threadIdx.x] = ii;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}
__global__ void k_absmax_final(const double* x, const double* pv, const long long* pi, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double bv = -1.0;
  long long bi = 0;
  for (int b = 0; b < nb; ++b) take(bv, bi, pv[b], pi[b]);
  out[0] = x[bi];
}

// Device storage of the folded vectors: slabs of 16 vectors taken with cudaMalloc as the
// solver needs them and reused through a free list, so that the vector operations of the
// solve allocate and free nothing (cudaFree synchronises the device); the slabs are
// released together when the solve ends. Slots are reused in stream order (all work of a
// solve is on one stream), so a slot released while kernels still read it is only
// overwritten after them.
struct VecPool {
  int64_t n = 0;
  std::vector<double*> slabs, free_slots;
  explicit VecPool(int64_t n_) : n(std::max<int64_t>(n_, 1)) {}
  VecPool(const VecPool&) = delete;
  VecPool& operator=(const VecPool&) = delete;
  double* acquire() {
    if (free_slots.empty()) {
      constexpr int kSlab = 16;
      // each slot starts on a 256-byte boundary
      const int64_t stride = (n + 31) / 32 * 32;
      double* p = nullptr;
      MLCC_CUDA(cudaMalloc(&p, size_t(stride) * kSlab * 8));
      slabs.push_back(p);
      for (int k = kSlab - 1; k >= 0; --k) free_slots.push_back(p + k * stride);
    }
    double* p = free_slots.back();
    free_slots.pop_back();
    return p;
  }
  void release(double* p) { free_slots.push_back(p); }
  ~VecPool() {
    for (double* p : slabs) cudaFree(p);
  }
};

// a folded vector in device memory (a pool slot), ordered on the context stream
struct DVec {
  double* p = nullptr;
  int64_t n = 0;
  cudaStream_t s = nullptr;
  VecPool* pool = nullptr;
  DVec() = default;
  DVec(VecPool* pool_, cudaStream_t s_) : n(pool_->n), s(s_), pool(pool_) {
    p = pool->acquire();
    MLCC_CUDA(cudaMemsetAsync(p, 0, size_t(n) * 8, s));
  }
  DVec(const DVec& o) : n(o.n), s(o.s), pool(o.pool) {
    if (pool) {
      p = pool->acquire();
      MLCC_CUDA(cudaMemcpyAsync(p, o.p, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
    }
  }
  DVec(DVec&& o) noexcept : p(o.p), n(o.n), s(o.s), pool(o.pool) { o.p = nullptr; }
  DVec& operator=(DVec o) noexcept {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(s, o.s);
    std::swap(pool, o.pool);
    return *this;
  }
  ~DVec() {
    if (p && pool) pool->release(p);
  }
};

// the vector space and operator of folded_solver.h on the device
struct DeviceSpace {
  using Vec = DVec;
  mlcc_system* S;
  int precision;
  cudaStream_t s;
  int64_t n1, tl, nf, dim;
  std::vector<int64_t> order;   // singles by ascending eps_a - eps_i
  Arena work;                   // five full vectors, the derivative singles, a scalar
  double *cf, *of, *w0, *w1, *w2, *dsing, *scal;
  VecPool pool;                 // the folded vectors

  DeviceSpace(mlcc_system* sys, int prec)
      : S(sys), precision(prec), s(sys->ctx->stream),
        pool(int64_t(sys->nv) * sys->no + int64_t(sys->tv) * sys->to * sys->tv * sys->to) {
    const int no = S->no, nv = S->nv;
    n1 = int64_t(nv) * no;
    tl = int64_t(S->tv) * S->to * S->tv * S->to;
    nf = n1 + tl;
    dim = n1 + S->nd;
    order.resize(size_t(n1));
    std::iota(order.begin(), order.end(), int64_t(0));
    const std::vector<double>& e = S->eps_host;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
      return e[no + x / no] - e[x % no] < e[no + y / no] - e[y % no];
    });
    work.reserve(size_t(5 * dim + n1 + 1) * 8 + 8 * 256);
    cf = work.get<double>(size_t(dim));
    of = work.get<double>(size_t(dim));
    w0 = work.get<double>(size_t(dim));
    w1 = work.get<double>(size_t(dim));
    w2 = work.get<double>(size_t(dim));
    dsing = work.get<double>(size_t(std::max<int64_t>(n1, 1)));
    scal = work.get<double>(1);
  }
  Vec make() { return DVec(&pool, s); }
  int n_guess() { return int(std::min<int64_t>(n1, 1 << 20)); }
  void guess(int k, Vec& v, double& diag) {
    v = make();
    const double one = 1.0;
    MLCC_CUDA(cudaMemcpyAsync(v.p + order[k], &one, 8, cudaMemcpyHostToDevice, s));
    MLCC_CUDA(cudaStreamSynchronize(s));   // the host value is a local
    const int no = S->no;
    diag = S->eps_host[no + order[k] / no] - S->eps_host[order[k] % no];
  }
  double dot(const Vec& x, const Vec& y) {
    dots(x.p, 0, 1, y.p, nf, scal, S->ws, s);
    double h = 0.0;
    MLCC_CUDA(cudaMemcpyAsync(&h, scal, 8, cudaMemcpyDeviceToHost, s));
    MLCC_CUDA(cudaStreamSynchronize(s));
    return h;
  }
  void axpy(double a, const Vec& x, Vec& y) { axpby(y.p, x.p, nf, a, 1.0, s); }
  void scale(double a, Vec& x) { axpby(x.p, x.p, nf, 0.0, a, s); }
  void precondition(const Vec& r, double omega, Vec& t) {
    t = make();
    k_fold_precondition<<<nblk_f(nf), 256, 0, s>>>(r.p, S->eps, S->no, S->nv, S->tv, S->to, omega, t.p);
    MLCC_CHECK_LAUNCH();
  }
  // folded x -> full-layout vector cf (P_S doubles zero)
  void unpack(const Vec& x, double* full) {
    MLCC_CUDA(cudaMemcpyAsync(full, x.p, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
    if (S->nd) MLCC_CUDA(cudaMemsetAsync(full + n1, 0, size_t(S->nd) * 8, s));
    if (tl) {
      k_box_scatter<<<nblk_f(tl), 256, 0, s>>>(x.p + n1, S->sv, S->so, S->tv, S->to, full + n1);
      MLCC_CHECK_LAUNCH();
    }
  }
  void apply(double omega, const Vec& x, Vec& y, Vec& dy) {
    unpack(x, cf);
    sigma_eff_eval(S, cf, omega, of, dsing, precision, w0, w1, w2);
    y = make();
    dy = make();
    MLCC_CUDA(cudaMemcpyAsync(y.p, of, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
    if (tl) {
      k_box_gather<<<nblk_f(tl), 256, 0, s>>>(of + n1, S->sv, S->so, S->tv, S->to, y.p + n1);
      MLCC_CHECK_LAUNCH();
    }
    MLCC_CUDA(cudaMemcpyAsync(dy.p, dsing, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
  }
};

}  // namespace

mlcc_status excited_states_folded(mlcc_system* S, const mlcc_options* opt, double* omega_host, double* r_out,
                                  mlcc_es_info* info) {
  if (!S->prepared) throw Error(MLCC_E_STATE, "mlcc_excited_states_folded: no prepared ground state");
  const int nr = opt->n_roots;
  const int64_t n1 = int64_t(S->nv) * S->no;
  MLCC_REQUIRE(nr >= 1 && nr <= n1, "n_roots must be in [1, n_vir * n_occ]");
  MLCC_REQUIRE(2 * int64_t(nr) <= n1, "the folded solver starts from 2 n_roots unit singles");
  cudaStream_t s = S->ctx->stream;
  DeviceSpace sp(S, opt->precision);
  fold::Options fo;
  fo.n_roots = nr;
  fo.res_tol = opt->es_res_tol;
  fo.max_iter = opt->max_es_iter;
  fo.max_sub = opt->max_subspace;
  fo.omega_max = lowest_ps_denominator(S);
  fold::Solver<DeviceSpace> solver(sp, fo);
  std::vector<DVec> X;
  const fold::Result res = solver.run(&X);
  int n_sigma = 3 * res.n_apply;
  const bool have = int(res.omega.size()) == nr && int(X.size()) == nr;
  if (have && r_out) {
    // unfolded eigenvectors: (c1, c_S(omega) + c_T), unit 2-norm, largest-magnitude element positive
    const int64_t dim = sp.dim;
    const int nb = int(std::min<int64_t>((dim + 255) / 256, 1024));
    Scope sc(S->ws);
    double* pv = S->ws.get<double>(size_t(nb));
    long long* pi = S->ws.get<long long>(size_t(nb));
    for (int k = 0; k < nr; ++k) {
      sp.unpack(X[k], sp.cf);
      sigma_eff_eval(S, sp.cf, res.omega[k], sp.of, nullptr, opt->precision, sp.w0, sp.w1, sp.w2);
      n_sigma += 2;
      double* r = r_out + int64_t(k) * dim;
      MLCC_CUDA(cudaMemcpyAsync(r, sp.w0, size_t(dim) * 8, cudaMemcpyDeviceToDevice, s));
      dots(r, 0, 1, r, dim, sp.scal, S->ws, s);
      double nrm2 = 0.0;
      MLCC_CUDA(cudaMemcpyAsync(&nrm2, sp.scal, 8, cudaMemcpyDeviceToHost, s));
      MLCC_CUDA(cudaStreamSynchronize(s));
      k_absmax_blocks<<<nb, 256, 0, s>>>(r, dim, pv, pi);
      MLCC_CHECK_LAUNCH();
      k_absmax_final<<<1, 32, 0, s>>>(r, pv, pi, nb, sp.scal);
      MLCC_CHECK_LAUNCH();
      double big = 0.0;
      MLCC_CUDA(cudaMemcpyAsync(&big, sp.scal, 8, cudaMemcpyDeviceToHost, s));
      MLCC_CUDA(cudaStreamSynchronize(s));
      const double f = (big < 0.0 ? -1.0 : 1.0) / std::sqrt(std::max(nrm2, 1e-300));
      axpby(r, r, dim, 0.0, f, s);
    }
  }
  if (opt->precision != MLCC_FP64) check_tc_error(S);
  MLCC_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < nr; ++k) omega_host[k] = have ? res.omega[k] : 0.0;
  if (info) {
    *info = mlcc_es_info{};
    info->iterations = res.iterations;
    info->n_sigma = n_sigma;
    info->converged = res.converged ? 1 : 0;
    double mr = 0.0;
    for (double r : res.residual) mr = std::max(mr, r);
    info->max_residual = have ? mr : INFINITY;
  }
  if (info) info->complex_pair = res.complex_pair ? 1 : 0;
  if (!res.converged) {
    set_last_error(std::string("mlcc_excited_states_folded: ") + (res.failure ? res.failure : "not converged"));
    return res.complex_pair ? MLCC_E_COMPLEX_ROOT : MLCC_E_ES_NOCONV;
  }
  return MLCC_OK;
}

}  // namespace mlcc

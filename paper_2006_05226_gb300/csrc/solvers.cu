// Control loops on the host, arithmetic on the device: the DIIS-accelerated quasi-Newton
// ground-state solver (Sec. 2.1) and the Davidson solver for the lowest right
// eigenpairs of the non-symmetric Jacobian (Sec. 2.1, excitation energies).
#include "system.cuh"
#include "fp_convert.cuh"
#include "small_eig.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <cstdio>
#include <cstdlib>

namespace mlcc {
int64_t launch_count();

namespace {
inline int nblk(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16384))); }

// quasi-Newton step on (t1, tT): p = x - Omega / eps, e = Omega / eps. The CCSD-block part
// is taken on the symmetric (admissible) amplitudes: x and Omega are averaged with their
// (ai) <-> (bj) transposes. Without that, the rounding of a split-precision phase leaves an
// antisymmetric part in tT on which the residual has no eps-diagonal term, so the
// quasi-Newton step cannot remove it and the refinement stalls on it.
__global__ void k_qn(const double* t1, const double* tT, const double* om1, const double* omT,
                     const double* eps, int no, int nv, int tv, int to, double* p, double* e) {
  const int64_t n1 = int64_t(nv) * no, nt = int64_t(tv) * to * tv * to, total = n1 + nt;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < total;
       k += int64_t(gridDim.x) * blockDim.x) {
    double x, om, den;
    if (k < n1) {
      const int a = int(k / no), i = int(k - int64_t(a) * no);
      x = t1[k];
      om = om1[k];
      den = eps[no + a] - eps[i];
    } else {
      int64_t t = k - n1;
      const int j = int(t % to); t /= to;
      const int b = int(t % tv); t /= tv;
      const int i = int(t % to);
      const int a = int(t / to);
      const int64_t kt = ((int64_t(b) * to + j) * tv + a) * to + i;   // (bj, ai)
      x = 0.5 * (tT[k - n1] + tT[kt]);
      om = 0.5 * (omT[k - n1] + omT[kt]);
      den = eps[no + a] - eps[i] + eps[no + b] - eps[j];
    }
    e[k] = om / den;
    p[k] = x - om / den;
  }
}

// Davidson preconditioner: d = (w - eps_mu)^-1 r, doubles symmetrised over (ai) <-> (bj)
__device__ __forceinline__ void st_out(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_out(float* p, double v) { *p = d2f_bits(v); }
__device__ __forceinline__ void st_out32(double* p, float v) { *p = f2d_bits(v); }
__device__ __forceinline__ void st_out32(float* p, float v) { *p = v; }
template <typename T>
__global__ void k_precond_singles(const double* r, const double* eps, int no, int nv, double w, T* d) {
  const int64_t n1 = int64_t(nv) * no;
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < n1;
       k += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(k / no), i = int(k - int64_t(a) * no);
    double den = w - (eps[no + a] - eps[i]);
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    st_out(d + k, r[k] / den);
  }
}
__device__ __forceinline__ float epsf(const double* eps, int p) { return d2f_bits(eps[p]); }
template <typename T>
__global__ void k_precond_doubles(const double* r, const double* eps, int no, int sv, int so, double w, T* d) {
  __shared__ double tile[32][33];
  const float wf = float(w);
  const int64_t dS = int64_t(sv) * so;
  const int64_t r0 = int64_t(blockIdx.y) * 32, c0 = int64_t(blockIdx.x) * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t rr = c0 + y, cc = r0 + threadIdx.x;
    tile[y][threadIdx.x] = (rr < dS && cc < dS) ? r[rr * dS + cc] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t row = r0 + y, col = c0 + threadIdx.x;
    if (row >= dS || col >= dS) continue;
    const int a = int(row / so), i = int(row - int64_t(a) * so);
    const int b = int(col / so), j = int(col - int64_t(b) * so);
    // binary32 arithmetic: the preconditioner only steers the expansion direction
    float den = wf - ((epsf(eps, no + a) - epsf(eps, i)) + (epsf(eps, no + b) - epsf(eps, j)));
    if (fabsf(den) < 1e-8f) den = den < 0.0f ? -1e-8f : 1e-8f;
    const float v = 0.5f * (d2f_bits(r[row * dS + col]) + d2f_bits(tile[threadIdx.x][y]));
    st_out32(d + row * dS + col, __fdividef(v, den));
  }
}
// R_k -= w_k X_k
__global__ void k_resid(double* R, const double* X, int64_t dim, double w) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < dim;
       i += int64_t(gridDim.x) * blockDim.x)
    R[i] -= w * X[i];
}
__global__ void k_scale(double* x, int64_t n, double a) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= a;
}
__global__ void k_set(double* x, int64_t i, double v) { x[i] = v; }
// largest |x| with its index (first on ties): per-block candidates, then one block
__device__ __forceinline__ void better(double& bv, long long& bi, double v, long long i) {
  if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}
__global__ void k_argmax_stage1(const double* x, int64_t n, double* pv, long long* pi) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double bv = -1.0;
  long long bi = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    better(bv, bi, fabs(x[i]), i);
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double v = sv[threadIdx.x];
      long long ii = si[threadIdx.x];
      better(v, ii, sv[threadIdx.x + w], si[threadIdx.x + w]);
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
__global__ void k_argmax_stage2(const double* x, const double* pv, const long long* pi, int nb,
                                double* out_val) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double bv = -1.0;
  long long bi = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) better(bv, bi, pv[b], pi[b]);
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double v = sv[threadIdx.x];
      long long ii = si[threadIdx.x];
      better(v, ii, sv[threadIdx.x + w], si[threadIdx.x + w]);
      sv[threadIdx.x] = v;
      si[threadIdx.x] = ii;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out_val[0] = x[si[0]];
}
}  // namespace

// MLCC_VERBOSE=1 in the environment: one line per iteration on stderr
static bool verbose() {
  static const bool v = [] {
    const char* e = std::getenv("MLCC_VERBOSE");
    return e && e[0] && e[0] != '0';
  }();
  return v;
}

static double host_scalar(mlcc_system* S, const double* d) {
  double h;
  copy_d2h(&h, d, 1, S->ctx->stream);
  return h;
}

// =================================================================================
// Ground state
mlcc_status ground_state(mlcc_system* S, const mlcc_options* opt, double* t1_out,
                         double* x2_out, mlcc_gs_info* info) {
  cudaStream_t s = S->ctx->stream;
  const int no = S->no, nv = S->nv, to = S->to, tv = S->tv;
  const int64_t n1 = int64_t(nv) * no;
  const int64_t tl = (to > 0 && tv > 0) ? int64_t(tv) * to * tv * to : 0;
  const int64_t len = n1 + tl;
  const int dd = std::max(1, opt->diis_dim);
  Scope sc(S->ws);
  double* t1 = S->ws.get<double>(n1);
  double* tT = S->ws.get<double>(std::max<int64_t>(tl, 1));
  double* om1 = S->ws.get<double>(n1);
  double* omT = S->ws.get<double>(std::max<int64_t>(tl, 1));
  double* x2 = S->nd ? x2_out : nullptr;
  double* energy = S->ws.get<double>(1);
  double* nrm = S->ws.get<double>(2);
  double* P = S->ws.get<double>(size_t(dd) * len);
  double* Er = S->ws.get<double>(size_t(dd) * len);
  double* pn = S->ws.get<double>(len);
  double* en = S->ws.get<double>(len);
  double* dv = S->ws.get<double>(dd);
  double* cdev = S->ws.get<double>(dd);
  fill(t1, n1, 0.0, s);
  if (tl) fill(tT, tl, 0.0, s);
  std::vector<double> Bm(size_t(dd) * dd, 0.0);
  std::vector<int> order;   // ring slots, oldest first
  double e_old = 0.0, e = 0.0, norm = 0.0;
  int it = 0;
  bool conv = false;
  // low-precision phase (gs_precision), then refine_precision when refine_fp64 is set
  int phase_prec = opt->gs_precision;
  // the ladder term's undressed integrals, built once in the most accurate precision the
  // iterations use and freed with the ground state
  struct LadderGuard {
    mlcc_system* S;
    ~LadderGuard() { gs_ladder_free(S); }
  } ladder_guard{S};
  {
    const int bprec = (is_split_precision(phase_prec) && opt->refine_fp64) ? opt->refine_precision : phase_prec;
    LowpScope lowp(bprec, S->tc_err);
    timed(S, "gs_ladder_build", 0.0, [&] { gs_ladder_build(S); });
    if (bprec != MLCC_FP64) check_tc_error(S);
  }
  const double lowp_switch = std::max(opt->gs_tol, 1e-7);
  std::vector<double> lowp_norms;   // residual norms of the low-precision phase
  for (it = 1; it <= opt->max_gs_iter; ++it) {
    {
      LowpScope lowp(phase_prec, S->tc_err, S->gsl_cache);
      timed(S, "gs_omega", 0.0, [&] {
        omega_eval(S, t1, nullptr, true, tl ? tT : nullptr, x2, om1, tl ? omT : nullptr, energy);
      });
    }
    if (phase_prec != MLCC_FP64) check_tc_error(S);
    const bool split_phase = is_split_precision(phase_prec);
    dots(om1, 0, 1, om1, n1, nrm, S->ws, s);
    if (tl) dots(omT, 0, 1, omT, tl, nrm + 1, S->ws, s);
    else fill(nrm + 1, 1, 0.0, s);
    double h[3];
    copy_d2h(h, energy, 1, s);
    copy_d2h(h + 1, nrm, 2, s);
    e = h[0];
    norm = std::sqrt(h[1] + h[2]);
    if (!std::isfinite(e) || !std::isfinite(norm))
      throw Error(MLCC_E_NAN, "ground state: NaN or Inf in the residual at iteration " + std::to_string(it));
    if (verbose())
      std::fprintf(stderr, "[mlcc] GS it %3d prec %d E %.14f |Omega| %.3e\n", it, phase_prec, e, norm);
    bool stalled = false;
    if (split_phase) {
      lowp_norms.push_back(norm);
      const size_t q = lowp_norms.size();
      if (q >= 6) {
        const double before = *std::min_element(lowp_norms.begin(), lowp_norms.end() - 3);
        const double recent = *std::min_element(lowp_norms.end() - 3, lowp_norms.end());
        stalled = recent > 0.5 * before;   // no halving in three iterations: the noise floor
      }
      // within a decade of the split-precision noise floor (about 1e-6), one iteration that
      // does not halve the residual already marks it: the binary64-class phase takes over
      if (q >= 2 && norm < 1e-5 && norm > 0.5 * lowp_norms[q - 2]) stalled = true;
    }
    if (split_phase && (norm < lowp_switch || stalled)) {
      if (!opt->refine_fp64) {
        conv = true;
        break;
      }
      phase_prec = opt->refine_precision;   // the next iterations refine these amplitudes
      operand_cache_clear(S->gsl_cache);    // converted in the split precision: not needed now
      order.clear();            // the low-precision residuals do not belong in DIIS
      std::fill(Bm.begin(), Bm.end(), 0.0);
      e_old = e;
      continue;                 // re-evaluate the residual in binary64 before stepping
    } else if (!split_phase && norm < opt->gs_tol &&
               std::fabs(e - e_old) < opt->gs_energy_tol) {
      conv = true;
      break;
    }
    e_old = e;
    k_qn<<<nblk(len), 256, 0, s>>>(t1, tT, om1, omT, S->eps, no, nv, tv, to, pn, en);
    MLCC_CHECK_LAUNCH();
    // ring buffer of (p, e)
    int slot;
    if (int(order.size()) < dd) {
      slot = int(order.size());
    } else {
      slot = order.front();
      order.erase(order.begin());
    }
    order.push_back(slot);
    MLCC_CUDA(cudaMemcpyAsync(P + int64_t(slot) * len, pn, size_t(len) * 8, cudaMemcpyDeviceToDevice, s));
    MLCC_CUDA(cudaMemcpyAsync(Er + int64_t(slot) * len, en, size_t(len) * 8, cudaMemcpyDeviceToDevice, s));
    dots(Er, len, dd, en, len, dv, S->ws, s);
    std::vector<double> dh(dd);
    copy_d2h(dh.data(), dv, dd, s);
    for (int k : order) {
      Bm[size_t(slot) * dd + k] = dh[k];
      Bm[size_t(k) * dd + slot] = dh[k];
    }
    const int m = int(order.size());
    std::vector<double> coef(dd, 0.0);
    bool ok = false;
    if (m > 1) {
      double scale = 0.0;
      for (int k : order) scale = std::max(scale, std::fabs(Bm[size_t(k) * dd + k]));
      if (scale <= 0.0) scale = 1.0;
      std::vector<double> A(size_t(m + 1) * (m + 1), 0.0), b(m + 1, 0.0), x;
      for (int r = 0; r < m; ++r) {
        for (int c = 0; c < m; ++c) A[r * (m + 1) + c] = Bm[size_t(order[r]) * dd + order[c]] / scale;
        A[r * (m + 1) + m] = -1.0;
        A[m * (m + 1) + r] = -1.0;
      }
      b[m] = -1.0;
      if (solve_linear(m + 1, A, b, x)) {
        for (int r = 0; r < m; ++r) coef[order[r]] = x[r];
        ok = true;
      }
    }
    if (!ok) {
      std::fill(coef.begin(), coef.end(), 0.0);
      coef[slot] = 1.0;
    }
    copy_h2d(cdev, coef.data(), dd, s);
    Gemm g;  // pn = sum_k coef_k P_k
    g.M = 1; g.N = len; g.K = dd;
    g.A = cdev; g.lda = dd; g.B = P; g.ldb = len; g.C = pn; g.ldc = len;
    gemm_f64(g, S->ws, s, S->ctx->sm_count);
    MLCC_CUDA(cudaMemcpyAsync(t1, pn, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
    if (tl) MLCC_CUDA(cudaMemcpyAsync(tT, pn + n1, size_t(tl) * 8, cudaMemcpyDeviceToDevice, s));
  }
  if (!conv) it = opt->max_gs_iter;
  MLCC_CUDA(cudaMemcpyAsync(t1_out, t1, size_t(n1) * 8, cudaMemcpyDeviceToDevice, s));
  if (info) {
    info->e_corr = e;
    info->omega_norm = norm;
    info->iterations = it;
    info->converged = conv ? 1 : 0;
  }
  // the Jacobian is taken at the returned amplitudes, in the binary64-class precision of
  // the last phase (the refinement precision after a split-precision phase)
  const int prep = is_split_precision(phase_prec) ? opt->refine_precision : phase_prec;
  {
    LowpScope lowp(prep == MLCC_FP64 ? 0 : prep, S->tc_err);
    timed(S, "jacobian_prepare", 0.0, [&] { jacobian_prepare(S, t1_out, x2_out); });
  }
  if (prep != MLCC_FP64) check_tc_error(S);
  MLCC_CUDA(cudaStreamSynchronize(s));
  return conv ? MLCC_OK : MLCC_E_GS_NOCONV;
}

// =================================================================================
// Davidson
namespace {
// Basis and sigma-vectors of the Davidson solver. In a split-precision phase they are
// stored in binary32 (es = 4: half the HBM traffic of every subspace pass; their
// sigma-vectors carry ~1e-7 relative errors anyway); in a binary64 phase in binary64.
struct DavState {
  mlcc_system* S;
  int64_t dim;
  int maxsub;
  char* Bp;    // basis [maxsub][dim]
  char* Sp;    // sigma-vectors [maxsub][dim]
  int es = 8;  // bytes per stored element
  int m = 0;
  bool left = false;   // the operator is A^T (left eigenvectors)
  std::vector<double> G;  // [maxsub][maxsub] host, G[i][j] = B_i . S_j
  void* B(int64_t k) const { return Bp + k * dim * es; }
  void* Sg(int64_t k) const { return Sp + k * dim * es; }
  bool f32() const { return es == 4; }
};

__global__ void k_set_f(float* v, int64_t i, float x) { v[i] = x; }

// out[k * ny + j] = x_k . y_j for stored vectors x_k, y_j (k < nx, j < ny <= 4)
void vdots_block(DavState& D, const void* x, int nx, const void* y, int ny, double* out) {
  mlcc_system* S = D.S;
  if (D.f32())
    dots_block_f32(static_cast<const float*>(x), D.dim, nx, static_cast<const float*>(y), D.dim, ny, D.dim, out,
                   S->ws, S->ctx->stream);
  else
    dots_block(static_cast<const double*>(x), D.dim, nx, static_cast<const double*>(y), D.dim, ny, D.dim, out,
               S->ws, S->ctx->stream);
}
// out[k] = x_k . y
void vdots(DavState& D, const void* x, int nx, const void* y, double* out) {
  mlcc_system* S = D.S;
  if (D.f32())
    dots_f32(static_cast<const float*>(x), D.dim, nx, static_cast<const float*>(y), D.dim, out, S->ws,
             S->ctx->stream);
  else
    dots(static_cast<const double*>(x), D.dim, nx, static_cast<const double*>(y), D.dim, out, S->ws, S->ctx->stream);
}
// C_i = alpha sum_k op(A)[i][k] V_k + beta C_i (i < M, k < K) with V stored vectors and C
// stored vectors (c_store) or binary64 vectors; A [M][K] (or [K][M] if ta), lda its row length
void vcombine(DavState& D, int M, int K, const double* A, int lda, bool ta, const void* V, void* C, bool c_store,
              double alpha, double beta) {
  mlcc_system* S = D.S;
  cudaStream_t s = S->ctx->stream;
  if (!D.f32()) {
    Gemm g;
    g.ta = ta;
    g.M = M; g.N = D.dim; g.K = K;
    g.A = A; g.lda = lda; g.B = static_cast<const double*>(V); g.ldb = D.dim;
    g.C = static_cast<double*>(C); g.ldc = D.dim;
    g.alpha = alpha; g.beta = beta;
    gemm_f64(g, S->ws, s, S->ctx->sm_count);
    return;
  }
  const size_t ces = c_store ? 4 : 8;
  for (int i0 = 0; i0 < M; i0 += 16) {
    const int mi = std::min(16, M - i0);
    for (int k0 = 0; k0 < K || k0 == 0; k0 += 64) {
      const int kk = std::min(64, K - k0);
      const double* Ab = ta ? A + int64_t(k0) * lda + i0 : A + int64_t(i0) * lda + k0;
      combine_f32(mi, D.dim, std::max(kk, 0), Ab, lda, ta, static_cast<const float*>(V) + int64_t(k0) * D.dim, D.dim,
                  static_cast<char*>(C) + size_t(i0) * D.dim * ces, c_store, D.dim, alpha, k0 == 0 ? beta : 1.0, s);
      if (K <= 0) break;
    }
  }
}
void vscale(DavState& D, void* v, double a) {
  if (D.f32()) {
    scale_f32(static_cast<float*>(v), D.dim, a, D.S->ctx->stream);
  } else {
    k_scale<<<nblk(D.dim), 256, 0, D.S->ctx->stream>>>(static_cast<double*>(v), D.dim, a);
    MLCC_CHECK_LAUNCH();
  }
}
void vcopy(DavState& D, void* dst, const void* src, int64_t count) {
  if (dst == src || count <= 0) return;
  MLCC_CUDA(cudaMemcpyAsync(dst, src, size_t(count) * D.dim * D.es, cudaMemcpyDeviceToDevice, D.S->ctx->stream));
}
}  // namespace

// Captured Jacobian transformations: sigma_eval(in -> out) in one precision as a CUDA graph.
// A graph's kernels read their scratch from S->ws above the mark it was captured at, so it is
// replayed only while the workspace mark is at or below that one (nothing live there).
struct SigmaGraphs {
  struct Entry {
    int prec;
    bool v32;           // captured with binary32 vector arithmetic on (Vec32Scope)
    const double* in;
    double* out;
    size_t mark;
    int64_t kernels;
    cudaGraphExec_t exec;
  };
  std::vector<Entry> entries;
  std::vector<int> warmed;   // (precision, binary32 state) evaluated eagerly since the last prepare
  ~SigmaGraphs() {
    for (auto& e : entries) cudaGraphExecDestroy(e.exec);
  }
};

void sigma_graphs_free(mlcc_system* S) {
  delete S->graphs;
  S->graphs = nullptr;
}

// sigma of `in` into `out`: eagerly, or through a graph captured on the second call of a
// precision and binary32 vector-arithmetic state (the first, eager one fills the operand
// caches, so the capture allocates nothing; the state decides the arithmetic of the skinny
// GEMMs inside sigma, so each state has a graph of its own)
static void sigma_one(mlcc_system* S, const double* in, double* out, int prec, bool graph) {
  cudaStream_t s = S->ctx->stream;
  if (!graph || S->ctx->timer.enabled) {
    timed(S, "sigma", 0.0, [&] { sigma_eval(S, in, out, prec); });
    return;
  }
  if (!S->graphs) S->graphs = new SigmaGraphs();
  SigmaGraphs& G = *S->graphs;
  const bool v32 = vec32_active();
  for (auto& e : G.entries)
    if (e.prec == prec && e.v32 == v32 && e.in == in && e.out == out && S->ws.mark() <= e.mark) {
      MLCC_CUDA(cudaGraphLaunch(e.exec, s));
      count_launches(e.kernels);
      return;
    }
  const int key = 2 * prec + (v32 ? 1 : 0);
  if (std::find(G.warmed.begin(), G.warmed.end(), key) == G.warmed.end()) {
    sigma_eval(S, in, out, prec);
    G.warmed.push_back(key);
    return;
  }
  SigmaGraphs::Entry e{prec, v32, in, out, S->ws.mark(), 0, nullptr};
  const int64_t l0 = launch_count();
  cudaGraph_t g = nullptr;
  MLCC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    sigma_eval(S, in, out, prec);
  } catch (...) {
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  MLCC_CUDA(cudaStreamEndCapture(s, &g));
  e.kernels = launch_count() - l0;
  const cudaError_t st = cudaGraphInstantiate(&e.exec, g, 0);
  cudaGraphDestroy(g);
  MLCC_CUDA(st);
  G.entries.push_back(e);
  MLCC_CUDA(cudaGraphLaunch(e.exec, s));
}

static void sigma_batch(mlcc_system* S, const double* C, double* Sg, int nvec, int64_t dim, int prec) {
  for (int k = 0; k < nvec; ++k)
    timed(S, "sigma", 0.0, [&] { sigma_eval(S, C + int64_t(k) * dim, Sg + int64_t(k) * dim, prec); });
  if (prec != MLCC_FP64) check_tc_error(S);
}
// sigma-vectors of the stored vectors [k0, k0 + nvec); binary32 storage, and every storage
// when sigma runs through a graph, goes through the binary64 buffers tc (trial vector) and
// ts (sigma-vector)
static void sigma_stored(DavState& D, int k0, int nvec, int prec, double* tc, double* ts, bool graph) {
  mlcc_system* S = D.S;
  if (D.left) {
    // A^T: eager, through the binary64 buffers
    cudaStream_t s = S->ctx->stream;
    for (int k = 0; k < nvec; ++k) {
      if (D.f32()) cvt_f2d(static_cast<const float*>(D.B(k0 + k)), tc, D.dim, s);
      else MLCC_CUDA(cudaMemcpyAsync(tc, D.B(k0 + k), size_t(D.dim) * 8, cudaMemcpyDeviceToDevice, s));
      timed(S, "sigma", 0.0, [&] { sigma_left_eval(S, tc, ts, prec); });
      if (D.f32()) cvt_d2f(ts, static_cast<float*>(D.Sg(k0 + k)), D.dim, s);
      else MLCC_CUDA(cudaMemcpyAsync(D.Sg(k0 + k), ts, size_t(D.dim) * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (prec != MLCC_FP64) check_tc_error(S);
    return;
  }
  if (!D.f32() && !graph) {
    sigma_batch(S, static_cast<const double*>(D.B(k0)), static_cast<double*>(D.Sg(k0)), nvec, D.dim, prec);
    return;
  }
  cudaStream_t s = S->ctx->stream;
  for (int k = 0; k < nvec; ++k) {
    if (D.f32()) cvt_f2d(static_cast<const float*>(D.B(k0 + k)), tc, D.dim, s);
    else MLCC_CUDA(cudaMemcpyAsync(tc, D.B(k0 + k), size_t(D.dim) * 8, cudaMemcpyDeviceToDevice, s));
    sigma_one(S, tc, ts, prec, graph);
    if (D.f32()) cvt_d2f(ts, static_cast<float*>(D.Sg(k0 + k)), D.dim, s);
    else MLCC_CUDA(cudaMemcpyAsync(D.Sg(k0 + k), ts, size_t(D.dim) * 8, cudaMemcpyDeviceToDevice, s));
  }
  if (prec != MLCC_FP64) check_tc_error(S);
}

// add the new columns [m0, m) to G: G[i][k] = B_i . S_k and G[k][j] = B_k . S_j, with the
// basis read once per block of up to four new vectors
static void update_G_body(DavState& D, int m0);
static void update_G(DavState& D, int m0) {
  timed(D.S, "dav_update_G", 0.0, [&] { update_G_body(D, m0); });
}
static void update_G_body(DavState& D, int m0) {
  mlcc_system* S = D.S;
  cudaStream_t s = S->ctx->stream;
  Scope sc(S->ws);
  double* out = S->ws.get<double>(size_t(D.maxsub) * 4);
  std::vector<double> h(size_t(D.maxsub) * 4);
  for (int k0 = m0; k0 < D.m; k0 += 4) {
    const int nk = std::min(4, D.m - k0);
    // B_i . S_k for i < m
    vdots_block(D, D.B(0), D.m, D.Sg(k0), nk, out);
    copy_d2h(h.data(), out, int64_t(D.m) * nk, s);
    for (int i = 0; i < D.m; ++i)
      for (int j = 0; j < nk; ++j) D.G[size_t(i) * D.maxsub + k0 + j] = h[size_t(i) * nk + j];
    // B_k . S_j for j < m0
    if (m0 > 0) {
      vdots_block(D, D.Sg(0), m0, D.B(k0), nk, out);
      copy_d2h(h.data(), out, int64_t(m0) * nk, s);
      for (int j = 0; j < m0; ++j)
        for (int q = 0; q < nk; ++q) D.G[size_t(k0 + q) * D.maxsub + j] = h[size_t(j) * nk + q];
    }
  }
}

// orthogonalise the block V = B[m .. m+nv) against B[0..m): two passes of
// V -= B (B^T V), reading the basis once per pass
static void block_project_body(DavState& D, int nv);
static void block_project(DavState& D, int nv) {
  timed(D.S, "dav_orthonormalise", 0.0, [&] { block_project_body(D, nv); });
}
static void block_project_body(DavState& D, int nv) {
  mlcc_system* S = D.S;
  if (D.m == 0 || nv == 0) return;
  Scope sc(S->ws);
  double* coef = S->ws.get<double>(size_t(D.m) * 4);
  for (int pass = 0; pass < 2; ++pass) {
    vdots_block(D, D.B(0), D.m, D.B(D.m), nv, coef);   // coef[k][j]
    // V_j -= sum_k coef[k][j] B_k
    vcombine(D, nv, D.m, coef, nv, true, D.B(0), D.B(D.m), true, -1.0, 1.0);
  }
}

// orthonormalise v against B[from..m) (two passes); returns false if v collapses
// ref_norm > 0: the norm of v before an earlier projection, for the drop test
static bool orthonormalise_body(DavState& D, void* v, int from, double ref_norm);
static bool orthonormalise(DavState& D, void* v, int from = 0, double ref_norm = 0.0) {
  bool ok = false;
  timed(D.S, "dav_orthonormalise", 0.0, [&] { ok = orthonormalise_body(D, v, from, ref_norm); });
  return ok;
}
static bool orthonormalise_body(DavState& D, void* v, int from, double ref_norm) {
  mlcc_system* S = D.S;
  Scope sc(S->ws);
  const int cnt = D.m - from;
  double* coef = S->ws.get<double>(std::max(cnt, 1));
  double* nr = S->ws.get<double>(1);
  vdots(D, v, 1, v, nr);
  const double n0 = ref_norm > 0.0 ? ref_norm : std::sqrt(host_scalar(S, nr));
  if (!(n0 > 0.0) || !std::isfinite(n0)) return false;
  for (int pass = 0; pass < 2 && cnt > 0; ++pass) {
    vdots(D, D.B(from), cnt, v, coef);
    vcombine(D, 1, cnt, coef, cnt, false, D.B(from), v, true, -1.0, 1.0);
  }
  vdots(D, v, 1, v, nr);
  const double n1 = std::sqrt(host_scalar(S, nr));
  // what is left of a direction inside the span is rounding noise: near 1e-16 of its norm
  // in binary64, near 1e-7 with binary32 storage or arithmetic
  if (!(n1 > (D.f32() || vec32_active() ? 1e-5 : 1e-10) * n0)) return false;
  vscale(D, v, 1.0 / n1);
  return true;
}

// X = Y^T B, R = Y^T S - w X for the wanted Ritz pairs (X, R binary64)
static void ritz_body(DavState& D, const std::vector<double>& Yt, int nr, const std::vector<double>& w,
                      double* X, double* R);
static void ritz(DavState& D, const std::vector<double>& Yt, int nr, const std::vector<double>& w,
                 double* X, double* R) {
  timed(D.S, "dav_ritz", 0.0, [&] { ritz_body(D, Yt, nr, w, X, R); });
}
static void ritz_body(DavState& D, const std::vector<double>& Yt, int nr, const std::vector<double>& w,
                      double* X, double* R) {
  mlcc_system* S = D.S;
  cudaStream_t s = S->ctx->stream;
  Scope sc(S->ws);
  double* y = S->ws.get<double>(size_t(nr) * D.m);
  copy_h2d(y, Yt.data(), int64_t(nr) * D.m, s);
  vcombine(D, nr, D.m, y, D.m, false, D.B(0), X, false, 1.0, 0.0);
  vcombine(D, nr, D.m, y, D.m, false, D.Sg(0), R, false, 1.0, 0.0);
  for (int k = 0; k < nr; ++k) {
    k_resid<<<nblk(D.dim), 256, 0, s>>>(R + int64_t(k) * D.dim, X + int64_t(k) * D.dim, D.dim, w[k]);
    MLCC_CHECK_LAUNCH();
  }
}

mlcc_status excited_states(mlcc_system* S, const mlcc_options* opt, double* omega_host,
                           double* r_out, mlcc_es_info* info, double* residual_host, bool left) {
  if (!S->prepared) throw Error(MLCC_E_STATE, "mlcc_excited_states: no prepared ground state");
  cudaStream_t s = S->ctx->stream;
  const int no = S->no, nv = S->nv, nreq = opt->n_roots;
  const int64_t n1 = int64_t(nv) * no, dim = n1 + S->nd;
  MLCC_REQUIRE(nreq >= 1 && nreq <= n1, "n_roots must be in [1, n_vir * n_occ]");
  const int nr = nreq;
  const int maxsub = sizes::davidson_max_subspace(opt->max_subspace, nr);
  const int collapse = 2 * nr;
  // Davidson memory: basis and sigma vectors, Ritz vectors, residuals, collapse scratch
  Arena dav;
  dav.reserve(sizes::davidson_bytes(dim, maxsub, nr));
  DavState D{S, dim, maxsub, static_cast<char*>(dav.alloc(size_t(maxsub) * dim * 8)),
             static_cast<char*>(dav.alloc(size_t(maxsub) * dim * 8))};
  D.G.assign(size_t(maxsub) * maxsub, 0.0);
  D.left = left;
  double* X = dav.get<double>(size_t(nr) * dim);
  double* R = dav.get<double>(size_t(nr) * dim);
  char* CB = static_cast<char*>(dav.alloc(size_t(collapse) * dim * 8));   // collapse scratch (stored type)
  char* CS = static_cast<char*>(dav.alloc(size_t(collapse) * dim * 8));
  double* tmpv = dav.get<double>(size_t(dim));   // binary64 trial vector / refinement restart
  double* tmps = dav.get<double>(size_t(dim));   // binary64 sigma-vector of a binary32 basis

  // start vectors: 2 n_roots unit singles with the lowest eps_a - eps_i
  std::vector<double> eh(S->n);
  copy_d2h(eh.data(), S->eps, S->n, s);
  std::vector<int64_t> idx(n1);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
    const double ex = eh[no + x / no] - eh[x % no], ey = eh[no + y / no] - eh[y % no];
    return ex < ey;
  });
  const int nguess = int(std::min<int64_t>(2 * nr, n1));
  int prec = opt->precision;
  const bool lowp = is_split_precision(prec);
  D.es = lowp ? 4 : 8;
  MLCC_CUDA(cudaMemsetAsync(D.B(0), 0, size_t(nguess) * dim * D.es, s));
  for (int k = 0; k < nguess; ++k) {
    if (D.f32()) k_set_f<<<1, 1, 0, s>>>(static_cast<float*>(D.B(k)), idx[k], 1.0f);
    else k_set<<<1, 1, 0, s>>>(static_cast<double*>(D.B(k)), idx[k], 1.0);
  }
  MLCC_CHECK_LAUNCH();
  D.m = nguess;

  const bool two_phase = lowp && opt->refine_fp64 > 0;
  int fp64_sweeps = 0;
  int n_sigma = 0, n_sigma_lowp = 0;
  auto count_sigma = [&](int k) {
    n_sigma += k;
    if (is_split_precision(prec)) n_sigma_lowp += k;
  };
  sigma_stored(D, 0, D.m, prec, tmpv, tmps, opt->sigma_graph != 0);
  count_sigma(D.m);
  {
    Vec32Scope v32(lowp);
    update_G(D, 0);
  }

  std::vector<double> w_old(nr, 1e300), w(nr), rn(nr);
  bool conv = false, complex_pair = false;
  int it = 0;
  const int max_it = std::max(1, opt->max_es_iter);
  for (it = 1; it <= max_it; ++it) {
    // vector arithmetic in binary32 while the sigma-vectors are split-precision
    Vec32Scope v32(is_split_precision(prec));
    // subspace eigenproblem (host, binary64)
    std::vector<double> Gm(size_t(D.m) * D.m);
    for (int i = 0; i < D.m; ++i)
      for (int j = 0; j < D.m; ++j) Gm[size_t(i) * D.m + j] = D.G[size_t(i) * maxsub + j];
    std::vector<std::complex<double>> ev;
    std::vector<std::vector<std::complex<double>>> vecs;
    const int nwant = std::min(std::max(nr, collapse), D.m);
    if (!eig_nonsym(D.m, Gm, ev, &vecs, nwant))
      throw Error(MLCC_E_ES_NOCONV, "Davidson: subspace eigenproblem failed");
    complex_pair = false;
    for (int k = 0; k < nr; ++k) {
      w[k] = ev[k].real();
      if (k < nreq && std::fabs(ev[k].imag()) > 1e-10 * std::max(1.0, std::fabs(ev[k].real())))
        complex_pair = true;
    }
    std::vector<double> Yt(size_t(nr) * D.m);
    for (int k = 0; k < nr; ++k)
      for (int i = 0; i < D.m; ++i) Yt[size_t(k) * D.m + i] = vecs[k][i].real();
    ritz(D, Yt, nr, w, X, R);
    // normalise X_k (and R_k with it), residual norms
    {
      Scope sc2(S->ws);
      double* nx = S->ws.get<double>(1);
      double* nrr = S->ws.get<double>(1);
      for (int k = 0; k < nr; ++k) {
        dots(X + int64_t(k) * dim, 0, 1, X + int64_t(k) * dim, dim, nx, S->ws, s);
        const double xn = std::sqrt(host_scalar(S, nx));
        k_scale<<<nblk(dim), 256, 0, s>>>(X + int64_t(k) * dim, dim, 1.0 / xn);
        k_scale<<<nblk(dim), 256, 0, s>>>(R + int64_t(k) * dim, dim, 1.0 / xn);
        MLCC_CHECK_LAUNCH();
        dots(R + int64_t(k) * dim, 0, 1, R + int64_t(k) * dim, dim, nrr, S->ws, s);
        rn[k] = std::sqrt(host_scalar(S, nrr));
        if (!std::isfinite(rn[k])) throw Error(MLCC_E_NAN, "Davidson: NaN in a residual");
      }
    }
    const bool in_lowp = is_split_precision(prec);
    if (verbose()) {
      std::fprintf(stderr, "[mlcc] ES it %3d prec %d dim %3d", it, prec, D.m);
      for (int k = 0; k < nr; ++k) std::fprintf(stderr, "  w %.10f r %.2e", w[k], rn[k]);
      std::fprintf(stderr, "\n");
    }
    if (two_phase && !in_lowp) ++fp64_sweeps;
    const double rtol = in_lowp ? opt->lowp_res_tol : opt->es_res_tol;
    std::vector<int> todo;
    bool req_done = true;
    for (int k = 0; k < nr; ++k) {
      const bool ok = (rn[k] < rtol) && (in_lowp ? true : std::fabs(w[k] - w_old[k]) < opt->es_omega_tol);
      if (!ok) todo.push_back(k);
      if (!ok && k < nreq) req_done = false;
    }
    w_old = w;
    if (req_done) todo.clear();
    if (todo.empty()) {
      if (two_phase && in_lowp) {
        // refinement: restart from the low-precision Ritz vectors with refine_precision sigma
        prec = opt->refine_precision;
        v32.set(false);
        D.es = 8;   // binary64 storage from here on
        const int keep = std::min(nr, D.m);   // all tracked Ritz vectors (binary64)
        MLCC_CUDA(cudaMemcpyAsync(CB, X, size_t(keep) * dim * 8, cudaMemcpyDeviceToDevice, s));
        D.m = 0;
        int added = 0;
        for (int k = 0; k < keep; ++k) {
          MLCC_CUDA(cudaMemcpyAsync(D.B(D.m), CB + size_t(k) * dim * 8, size_t(dim) * 8,
                                    cudaMemcpyDeviceToDevice, s));
          if (orthonormalise(D, D.B(D.m))) {
            ++D.m;
            ++added;
          }
        }
        sigma_stored(D, 0, D.m, prec, tmpv, tmps, opt->sigma_graph != 0);
        count_sigma(D.m);
        std::fill(D.G.begin(), D.G.end(), 0.0);
        update_G(D, 0);
        std::fill(w_old.begin(), w_old.end(), 1e300);
        continue;
      }
      conv = true;
      break;
    }
    if (two_phase && !in_lowp && fp64_sweeps >= opt->refine_fp64) {
      conv = true;   // the binary64 refinement budget is spent; max_residual tells how far
      break;
    }
    // new directions
    std::vector<int> newk;
    if (D.m + int(todo.size()) > maxsub) {
      // collapse onto the lowest `collapse` Ritz vectors
      const int c = std::min(collapse, D.m);
      std::vector<double> Yc(size_t(c) * D.m);
      for (int k = 0; k < c; ++k)
        for (int i = 0; i < D.m; ++i) Yc[size_t(k) * D.m + i] = vecs[k][i].real();
      {
        Scope sc3(S->ws);
        double* y = S->ws.get<double>(size_t(c) * D.m);
        copy_h2d(y, Yc.data(), int64_t(c) * D.m, s);
        vcombine(D, c, D.m, y, D.m, false, D.B(0), CB, true, 1.0, 0.0);
        vcombine(D, c, D.m, y, D.m, false, D.Sg(0), CS, true, 1.0, 0.0);
        // Gram-Schmidt on CB with the same combinations on CS
        double* coef = S->ws.get<double>(size_t(c));
        double* nx = S->ws.get<double>(1);
        const size_t vb = size_t(dim) * D.es;
        for (int k = 0; k < c; ++k) {
          void* bk = CB + k * vb;
          void* sk = CS + k * vb;
          for (int pass = 0; pass < 2 && k > 0; ++pass) {
            vdots(D, CB, k, bk, coef);
            vcombine(D, 1, k, coef, k, false, CB, bk, true, -1.0, 1.0);
            vcombine(D, 1, k, coef, k, false, CS, sk, true, -1.0, 1.0);
          }
          vdots(D, bk, 1, bk, nx);
          const double nk = std::sqrt(host_scalar(S, nx));
          vscale(D, bk, 1.0 / nk);
          vscale(D, sk, 1.0 / nk);
        }
      }
      vcopy(D, D.B(0), CB, c);
      vcopy(D, D.Sg(0), CS, c);
      D.m = c;
      std::fill(D.G.begin(), D.G.end(), 0.0);
      update_G(D, 0);
    }
    const int m0 = D.m;
    int nnew = 0;
    for (int k : todo) {
      if (D.m + nnew >= maxsub || nnew == 4) break;
      void* v = D.B(D.m + nnew);
      dim3 blk(32, 8), grd(unsigned((S->dS + 31) / 32), unsigned((S->dS + 31) / 32));
      if (D.f32()) {
        float* vf = static_cast<float*>(v);
        k_precond_singles<<<nblk(n1), 256, 0, s>>>(R + int64_t(k) * dim, S->eps, no, nv, w[k], vf);
        if (S->nd)
          k_precond_doubles<<<grd, blk, 0, s>>>(R + int64_t(k) * dim + n1, S->eps, no, S->sv, S->so, w[k], vf + n1);
      } else {
        double* vd = static_cast<double*>(v);
        k_precond_singles<<<nblk(n1), 256, 0, s>>>(R + int64_t(k) * dim, S->eps, no, nv, w[k], vd);
        if (S->nd)
          k_precond_doubles<<<grd, blk, 0, s>>>(R + int64_t(k) * dim + n1, S->eps, no, S->sv, S->so, w[k], vd + n1);
      }
      MLCC_CHECK_LAUNCH();
      ++nnew;
    }
    // the old basis is projected out of the whole block first; the vectors of the block are
    // then orthonormalised one by one (against the basis and the accepted block members),
    // dropped when less than 1e-10 of their norm before the projection remains
    std::vector<double> pre(nnew, 0.0);
    {
      Scope sp(S->ws);
      double* nrm = S->ws.get<double>(4);
      for (int q = 0; q < nnew; ++q) vdots(D, D.B(D.m + q), 1, D.B(D.m + q), nrm + q);
      double hn[4] = {0, 0, 0, 0};
      if (nnew) copy_d2h(hn, nrm, nnew, s);
      for (int q = 0; q < nnew; ++q) pre[q] = std::sqrt(hn[q]);
    }
    block_project(D, nnew);
    for (int q = 0; q < nnew; ++q) {
      void* v = D.B(D.m);
      if (D.m != m0 + q) vcopy(D, v, D.B(m0 + q), 1);
      if (pre[q] > 0.0 && std::isfinite(pre[q]) && orthonormalise(D, v, m0, pre[q])) ++D.m;
    }
    if (D.m == m0) {
      // no new direction: the basis spans an invariant subspace
      conv = true;
      for (int k = 0; k < nreq; ++k) conv = conv && rn[k] < opt->es_res_tol;
      break;
    }
    sigma_stored(D, m0, D.m - m0, prec, tmpv, tmps, opt->sigma_graph != 0);
    count_sigma(D.m - m0);
    update_G(D, m0);
  }
  // sign convention: largest-magnitude element positive
  {
    Scope sc4(S->ws);
    double* mv = S->ws.get<double>(1);
    for (int k = 0; k < nr; ++k) {
      const int nb = int(std::min<int64_t>((dim + 255) / 256, 1024));
      double* pv = S->ws.get<double>(size_t(nb));
      long long* pi = S->ws.get<long long>(size_t(nb));
      k_argmax_stage1<<<nb, 256, 0, s>>>(X + int64_t(k) * dim, dim, pv, pi);
      MLCC_CHECK_LAUNCH();
      k_argmax_stage2<<<1, 256, 0, s>>>(X + int64_t(k) * dim, pv, pi, nb, mv);
      MLCC_CHECK_LAUNCH();
      if (host_scalar(S, mv) < 0.0) {
        k_scale<<<nblk(dim), 256, 0, s>>>(X + int64_t(k) * dim, dim, -1.0);
        MLCC_CHECK_LAUNCH();
      }
    }
  }
  for (int k = 0; k < nreq; ++k) omega_host[k] = w[k];
  if (residual_host)
    for (int k = 0; k < nreq; ++k) residual_host[k] = rn[k];
  if (r_out) MLCC_CUDA(cudaMemcpyAsync(r_out, X, size_t(nreq) * dim * 8, cudaMemcpyDeviceToDevice, s));
  MLCC_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->iterations = it;
    info->n_sigma = n_sigma;
    info->n_sigma_lowp = n_sigma_lowp;
    info->converged = conv ? 1 : 0;
    info->complex_pair = complex_pair ? 1 : 0;
    info->fp64_sweeps = fp64_sweeps;
    double mr = 0.0;
    for (int k = 0; k < nr; ++k) mr = std::max(mr, rn[k]);
    info->max_residual = mr;
  }
  if (!conv) return MLCC_E_ES_NOCONV;
  if (complex_pair) return MLCC_E_COMPLEX_ROOT;
  return MLCC_OK;
}

}  // namespace mlcc

// The MLCC residual and Jacobian transformation on the device (arXiv 2006.05226,
// Sec. 2.1 and Appendix A). The residual pipeline is written once; the Jacobian
// transformation sigma = A c is its forward-mode derivative along c, evaluated by the
// product rule contraction by contraction around the cached ground-state values.
#include "system.cuh"

#include <algorithm>

namespace mlcc {

static inline cudaStream_t stm(mlcc_system* S) { return S->ctx->stream; }
static inline int smc(mlcc_system* S) { return S->ctx->sm_count; }
static inline int nblk(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16384))); }

// ---------------------------------------------------------------------------------
// kernels
namespace {
// D[J] = sum_{I < no} X[J][I][I]
__global__ void k_trace_occ(const double* X, int nj, int n, int no, double* D) {
  const int J = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (J >= nj) return;
  const double* x = X + int64_t(J) * n * n;
  double s = 0.0;
  for (int I = lane; I < no; I += 32) s += x[int64_t(I) * n + I];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) D[J] = s;
}
// out[J][a*so + i] = X[J][no + a][i]   (virtual-occupied block, CC2-active)
__global__ void k_gather_vo(const double* X, int nj, int n, int no, int sv, int so, double* out) {
  const int64_t dS = int64_t(sv) * so, total = dS * nj;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t J = t / dS, r = t - J * dS;
    const int a = int(r / so), i = int(r - int64_t(a) * so);
    out[t] = X[J * n * n + int64_t(no + a) * n + i];
  }
}
// out[J][c*so + j] = X[J][j][no + c]   (occupied-virtual block, CC2-active)
__global__ void k_gather_ov(const double* X, int nj, int n, int no, int sv, int so, double* out) {
  const int64_t dS = int64_t(sv) * so, total = dS * nj;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t J = t / dS, r = t - J * dS;
    const int c = int(r / so), j = int(r - int64_t(c) * so);
    out[t] = X[J * n * n + int64_t(j) * n + no + c];
  }
}
__device__ __forceinline__ void split4(int64_t t, int sv, int so, int& a, int& i, int& b, int& j) {
  j = int(t % so);
  t /= so;
  b = int(t % sv);
  t /= sv;
  i = int(t % so);
  a = int(t / so);
}
// u[a,i,b,j] = 2 x[a,i,b,j] - x[a,j,b,i]: block (a, b) of u is 2 X - X^T for the so x so
// block X at rows a so, columns b so of x; one CTA per block through shared memory (so <= 64)
__global__ void k_make_u_blocks(const double* x, int sv, int so, double* u) {
  __shared__ double tile[64][65];
  const int64_t dS = int64_t(sv) * so;
  const double* xb = x + (int64_t(blockIdx.y) * so) * dS + int64_t(blockIdx.x) * so;
  double* ub = u + (int64_t(blockIdx.y) * so) * dS + int64_t(blockIdx.x) * so;
  for (int t = threadIdx.x; t < so * so; t += blockDim.x) {
    const int i = t / so, j = t - i * so;
    tile[i][j] = xb[int64_t(i) * dS + j];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < so * so; t += blockDim.x) {
    const int i = t / so, j = t - i * so;
    ub[int64_t(i) * dS + j] = fma(2.0, tile[i][j], -tile[j][i]);
  }
}
// the same for any so, element by element
__global__ void k_make_u(const double* x, int sv, int so, double* u) {
  const int64_t total = int64_t(sv) * so * sv * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int a, i, b, j;
    split4(t, sv, so, a, i, b, j);
    const int64_t tx = ((int64_t(a) * so + j) * sv + b) * so + i;
    u[t] = 2.0 * x[t] - x[tx];
  }
}
__device__ __forceinline__ bool in_T(int a, int i, int b, int j, int tv, int to) {
  return a < tv && i < to && b < tv && j < to;
}
__device__ __forceinline__ double eps4(const double* eps, int no, int a, int i, int b, int j) {
  return eps[no + a] - eps[i] + eps[no + b] - eps[j];
}
// GS: CC2 doubles s = -g~/eps on P_S (Appendix A), P_T amplitudes from tT (or 0)
__global__ void k_cc2_amp(const double* g, const double* eps, int no, int sv, int so, int tv,
                          int to, const double* tT, double* x2) {
  const int64_t total = int64_t(sv) * so * sv * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int a, i, b, j;
    split4(t, sv, so, a, i, b, j);
    if (in_T(a, i, b, j, tv, to)) {
      x2[t] = tT ? tT[((int64_t(a) * to + i) * tv + b) * to + j] : 0.0;
    } else {
      x2[t] = -g[t] / eps4(eps, no, a, i, b, j);
    }
  }
}
// Omega on P_S: g~ + eps x (Eq. mlcc2_omega2 in the semicanonical basis); P_T rows 0
__global__ void k_omega2_cc2(const double* g, const double* x2, const double* eps, int no, int sv,
                             int so, int tv, int to, double* om2) {
  const int64_t total = int64_t(sv) * so * sv * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int a, i, b, j;
    split4(t, sv, so, a, i, b, j);
    om2[t] = in_T(a, i, b, j, tv, to) ? 0.0 : g[t] + eps4(eps, no, a, i, b, j) * x2[t];
  }
}
// sigma on P_S: W_(ai)(bj) + W_(bj)(ai) + eps c; P_T rows 0. 32 x 32 tiles through shared
// memory so that both the direct and the transposed read are coalesced.
// The orbital-energy part eps_scale (e_a - e_i + e_b - e_j) is split into a row and a column
// share taken once per row and per thread: three binary64 operations per element remain
// (the binary64 pipe, not HBM, bounded the straightforward form on GB300).
__global__ void k_sigma2_cc2(const double* W, const double* c, const double* eps, int no, int sv,
                             int so, int tv, int to, double eps_scale, double* s2) {
  __shared__ double tile[32][33];
  const int dS = sv * so;   // dS^2 doubles fit the device: dS < 2^31
  const int r0 = int(blockIdx.y) * 32, c0 = int(blockIdx.x) * 32;
  // transposed block W[c0.., r0..] -> tile[col][row]
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int rr = c0 + y, cc = r0 + threadIdx.x;
    tile[y][threadIdx.x] = (rr < dS && cc < dS) ? W[int64_t(rr) * dS + cc] : 0.0;
  }
  __syncthreads();
  const int col = c0 + threadIdx.x;
  if (col >= dS) return;
  const int b = col / so, j = col - b * so;
  const double ec = eps_scale * (eps[no + b] - eps[j]);
  const bool tcol = b < tv && j < to;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int row = r0 + y;
    if (row >= dS) break;
    const int a = row / so, i = row - a * so;
    const double er = eps_scale * (eps[no + a] - eps[i]);
    const int64_t t = int64_t(row) * dS + col;
    s2[t] = (tcol && a < tv && i < to) ? 0.0 : fma(er + ec, c[t], W[t] + tile[threadIdx.x][y]);
  }
}
// om1[a*no + i] += alpha * tmp[a*so + i]
__global__ void k_scatter_add_ai(const double* tmp, int sv, int so, int no, double alpha,
                                 double* om1) {
  const int64_t total = int64_t(sv) * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(t / so), i = int(t - int64_t(a) * so);
    om1[int64_t(a) * no + i] += alpha * tmp[t];
  }
}
// fv[b*so + j] = F[j][no + b]
__global__ void k_fov(const double* F, int n, int no, int sv, int so, double* fv) {
  const int64_t total = int64_t(sv) * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(t / so), j = int(t - int64_t(b) * so);
    fv[t] = F[int64_t(j) * n + no + b];
  }
}
// part[J] = 2 tr(M_J)^2 - sum_IK M_J[I][K] M_J[K][I]   (Eq. mlcc_energy, singles term)
__global__ void k_energy1(const double* M, int no, double* part) {
  __shared__ double r1[256], r2[256];
  const double* m = M + int64_t(blockIdx.x) * no * no;
  double tr = 0.0, q = 0.0;
  for (int t = threadIdx.x; t < no * no; t += blockDim.x) {
    const int I = t / no, K = t - I * no;
    if (I == K) tr += m[t];
    q += m[t] * m[int64_t(K) * no + I];
  }
  r1[threadIdx.x] = tr;
  r2[threadIdx.x] = q;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = 2.0 * r1[0] * r1[0] - r2[0];
}
// out = sum_k part[k] + extra[0]  (one block, fixed order)
__global__ void k_sum_plus(const double* part, int n, const double* extra, double* out) {
  __shared__ double r[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) r[threadIdx.x] += r[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = r[0] + (extra ? extra[0] : 0.0);
}
}  // namespace

// ---------------------------------------------------------------------------------
// strided 2-D block copy / accumulate: dst[r*ldd + c] = alpha src[r*lds + c] + beta dst
static void block2d(mlcc_system* S, int64_t rows, int64_t cols, const double* src, int64_t lds,
                    double* dst, int64_t ldd, double alpha, double beta) {
  int64_t dims[2] = {rows, cols}, ss[2] = {lds, 1}, ds[2] = {ldd, 1};
  permute_f64(2, dims, src, ss, dst, ds, alpha, beta, stm(S));
}

void gather_vo(mlcc_system* S, const double* X, double* out) {
  if (S->dS == 0) return;
  k_gather_vo<<<nblk(S->dS * S->nj), 256, 0, stm(S)>>>(X, S->nj, S->n, S->no, S->sv, S->so, out);
  MLCC_CHECK_LAUNCH();
}
void gather_ov(mlcc_system* S, const double* X, double* out) {
  if (S->dS == 0) return;
  k_gather_ov<<<nblk(S->dS * S->nj), 256, 0, stm(S)>>>(X, S->nj, S->n, S->no, S->sv, S->so, out);
  MLCC_CHECK_LAUNCH();
}
void make_u(mlcc_system* S, const double* x2, double* u) {
  if (S->nd == 0) return;
  if (S->so <= 64 && S->sv < 65536) {
    k_make_u_blocks<<<dim3(unsigned(S->sv), unsigned(S->sv), 1), 256, 0, stm(S)>>>(x2, S->sv, S->so, u);
  } else {
    k_make_u<<<nblk(S->nd), 256, 0, stm(S)>>>(x2, S->sv, S->so, u);
  }
  MLCC_CHECK_LAUNCH();
}

// T1-dressing (Sec. 2.1, Appendix A): Lt = (1 - t) L (1 + t), t in the vir-occ block.
// (1 - t) L changes the virtual rows: Lt[v,:] = L[v,:] - t L[o,:]; the right factor
// changes the occupied columns: Lt[:,o] += Lt[:,v] t.
void dress(mlcc_system* S, const double* t1, double* Lt, double* ht) {
  const int n = S->n, no = S->no, nv = S->nv, nj = S->nj;
  const int64_t nn = int64_t(n) * n;
  cudaStream_t s = stm(S);
  auto one = [&](const double* X, double* Y, int64_t batch) {
    MLCC_CUDA(cudaMemcpyAsync(Y, X, size_t(batch * nn) * 8, cudaMemcpyDeviceToDevice, s));
    if (no == 0 || nv == 0) return;
    Gemm g1;
    g1.M = nv; g1.N = n; g1.K = no;
    g1.A = t1; g1.lda = no; g1.sA = 0;
    g1.B = X; g1.ldb = n; g1.sB = nn;
    g1.C = Y + int64_t(no) * n; g1.ldc = n; g1.sC = nn;
    g1.alpha = -1.0; g1.beta = 1.0; g1.batch = batch;
    gemm_f64(g1, S->ws, s, smc(S));
    Gemm g2;
    g2.M = n; g2.N = no; g2.K = nv;
    g2.A = Y + no; g2.lda = n; g2.sA = nn;
    g2.B = t1; g2.ldb = no; g2.sB = 0;
    g2.C = Y; g2.ldc = n; g2.sC = nn;
    g2.alpha = 1.0; g2.beta = 1.0; g2.batch = batch;
    gemm_f64(g2, S->ws, s, smc(S));
  };
  one(S->L, Lt, nj);
  if (ht) one(S->h, ht, 1);
}

// Tangent of the dressing along c1: d Lt = Lt C - C Lt with C the vir-occ matrix of c1
// (exp(-T) M exp(T) differentiated; C T = T C = 0).
void dress_tangent(mlcc_system* S, const double* c1, double* dLt, double* dht) {
  const int n = S->n, no = S->no, nv = S->nv, nj = S->nj;
  const int64_t nn = int64_t(n) * n;
  cudaStream_t s = stm(S);
  auto one = [&](const double* X, double* Y, int64_t batch) {
    MLCC_CUDA(cudaMemsetAsync(Y, 0, size_t(batch * nn) * 8, s));
    if (no == 0 || nv == 0) return;
    Gemm g1;  // Y[:, o] = X[:, v] c1
    g1.M = n; g1.N = no; g1.K = nv;
    g1.A = X + no; g1.lda = n; g1.sA = nn;
    g1.B = c1; g1.ldb = no; g1.sB = 0;
    g1.C = Y; g1.ldc = n; g1.sC = nn;
    g1.alpha = 1.0; g1.beta = 0.0; g1.batch = batch;
    gemm_f64(g1, S->ws, s, smc(S));
    Gemm g2;  // Y[v, :] -= c1 X[o, :]
    g2.M = nv; g2.N = n; g2.K = no;
    g2.A = c1; g2.lda = no; g2.sA = 0;
    g2.B = X; g2.ldb = n; g2.sB = nn;
    g2.C = Y + int64_t(no) * n; g2.ldc = n; g2.sC = nn;
    g2.alpha = -1.0; g2.beta = 1.0; g2.batch = batch;
    gemm_f64(g2, S->ws, s, smc(S));
  };
  one(S->Lt, dLt, nj);
  one(S->ht, dht, 1);
}

static void trace_occ(mlcc_system* S, const double* X, double* D) {
  const int warps = 8;
  k_trace_occ<<<(S->nj + warps - 1) / warps, 32 * warps, 0, stm(S)>>>(X, S->nj, S->n, S->no, D);
  MLCC_CHECK_LAUNCH();
}

// F += alpha_c * 2 sum_J D_J X^J  and  F -= alpha_x * sum_J X^J[:, o] Y^J[o, :]
static void fock_terms(mlcc_system* S, const double* D, const double* X, const double* XL,
                       const double* YR, double* F, double sgn) {
  const int n = S->n, no = S->no, nj = S->nj;
  const int64_t nn = int64_t(n) * n;
  cudaStream_t s = stm(S);
  if (D) {
    Gemm c;
    c.M = 1; c.N = nn; c.K = nj;
    c.A = D; c.lda = nj; c.B = X; c.ldb = nn; c.C = F; c.ldc = nn;
    c.alpha = 2.0 * sgn; c.beta = 1.0;
    gemm_f64(c, S->ws, s, smc(S));
  }
  if (XL && no > 0) {
    Gemm x;
    x.M = n; x.N = n; x.K = no;
    x.A = XL; x.lda = n; x.sA = nn;
    x.B = YR; x.ldb = n; x.sB = nn;
    x.C = F; x.ldc = n;
    x.alpha = -sgn; x.beta = 1.0; x.batch = nj; x.reduce = true;
    gemm_f64(x, S->ws, s, smc(S));
  }
}

// F~ = h~ + sum_J [2 Lt^J (sum_I Lt^J_II) - Lt^J[:, I] Lt^J[I, :]]   (Appendix A, F~_PQ)
void build_fock(mlcc_system* S, const double* ht, const double* Lt, double* Ft) {
  Scope sc(S->ws);
  const int64_t nn = int64_t(S->n) * S->n;
  double* D = S->ws.get<double>(S->nj);
  trace_occ(S, Lt, D);
  MLCC_CUDA(cudaMemcpyAsync(Ft, ht, size_t(nn) * 8, cudaMemcpyDeviceToDevice, stm(S)));
  fock_terms(S, D, Lt, Lt, Lt, Ft, 1.0);
}

void build_fock_tangent(mlcc_system* S, const double* dht, const double* dLt, double* dFt) {
  Scope sc(S->ws);
  const int64_t nn = int64_t(S->n) * S->n;
  double* D = S->ws.get<double>(S->nj);
  double* dD = S->ws.get<double>(S->nj);
  trace_occ(S, S->Lt, D);
  trace_occ(S, dLt, dD);
  MLCC_CUDA(cudaMemcpyAsync(dFt, dht, size_t(nn) * 8, cudaMemcpyDeviceToDevice, stm(S)));
  fock_terms(S, D, dLt, dLt, S->Lt, dFt, 1.0);
  fock_terms(S, dD, S->Lt, S->Lt, dLt, dFt, 1.0);
}

// ---------------------------------------------------------------------------------
// The Cholesky-rank doubles GEMMs (the dominant work): C[dS x dS] = A^T B with A, B
// [nj][dS], or C[nj x dS] = A[nj x dS] B[dS x dS]. Binary64 (FMA units, or MLCC_FP64E on
// the tensor cores) here; the split-bfloat16 precisions go through rank_gemm_lowp.
void rank_gemm_f64(mlcc_system* S, bool outer, const double* A, const double* B, double* C,
                   double alpha, double beta);

void rank_gemm_f64(mlcc_system* S, bool outer, const double* A, const double* B, double* C,
                   double alpha, double beta) {
  const int64_t dS = S->dS, nj = S->nj;
  Gemm g;
  if (outer) {  // C[dS][dS] = A^T B, K = nj
    g.ta = true; g.M = dS; g.N = dS; g.K = nj;
    g.A = A; g.lda = dS; g.B = B; g.ldb = dS; g.C = C; g.ldc = dS;
  } else {      // C[nj][dS] = A[nj][dS] B[dS][dS]
    g.M = nj; g.N = dS; g.K = dS;
    g.A = A; g.lda = dS; g.B = B; g.ldb = dS; g.C = C; g.ldc = dS;
  }
  g.alpha = alpha;
  g.beta = beta;
  const int lp = lowp_precision();
  const double flop = 2.0 * double(g.M) * double(g.N) * double(g.K);
  if (lp == MLCC_FP64E && gemm_emu_fits(g, S->ws)) {
    timed(S, "rank_gemm_f64e", flop, [&] { gemm_emu(g, S->ws, stm(S), smc(S), lowp_error_flag()); });
    return;
  }
  // binary64 FMA units (also MLCC_FP64E when the workspace cannot hold the emulation)
  LowpScope scope(lp == MLCC_FP64E ? 0 : lp, lowp_error_flag(), lowp_cache());
  timed(S, lp && lp != MLCC_FP64E ? "rank_gemm_tc" : "rank_gemm_f64", flop,
        [&] { gemm_f64(g, S->ws, stm(S), smc(S)); });
}

static void rank_gemm(mlcc_system* S, int precision, bool outer, const double* A, const double* B,
                      double* C, double alpha, double beta) {
  if (is_split_precision(precision) && !S->jwin) {   // the cached pieces cover every J
    if (S->lowp_prec != precision) lowp_prepare(S, precision);
    rank_gemm_lowp(S, outer, A, B, C, alpha, beta, precision, false);
  } else {
    rank_gemm_f64(S, outer, A, B, C, alpha, beta);
  }
}

// ---------------------------------------------------------------------------------
// CCSD-active block extraction helpers (the CCSD orbitals lead each range)
struct Box {
  Dual Lai, Lac, Lki, Lkc, Fvv, Foo, t;
};

static DT box_view(mlcc_system* S, int64_t a, int64_t b, int64_t c) {
  DT x;
  x.d = {a, b, c};
  x.p = S->ws.get<double>(size_t(a * b * c));
  return x;
}

// copy the [nj] x rows x cols sub-block at (r0, c0) of X[nj][n][n]
static void take_block(mlcc_system* S, const double* X, int64_t batch, int r0, int rows, int c0,
                       int cols, DT& out) {
  const int64_t n = S->n, nn = n * n;
  int64_t dims[3] = {batch, rows, cols}, ss[3] = {nn, n, 1}, ds[3] = {int64_t(rows) * cols, cols, 1};
  permute_f64(3, dims, X + r0 * n + c0, ss, out.p, ds, 1.0, 0.0, stm(S));
}

static void take_tbox(mlcc_system* S, const double* x2, DT& out) {
  const int so = S->so, sv = S->sv, to = S->to, tv = S->tv;
  int64_t dims[4] = {tv, to, tv, to};
  int64_t ss[4] = {int64_t(so) * sv * so, int64_t(sv) * so, so, 1};
  int64_t ds[4] = {int64_t(to) * tv * to, int64_t(tv) * to, to, 1};
  permute_f64(4, dims, x2, ss, out.p, ds, 1.0, 0.0, stm(S));
}
static void put_tbox(mlcc_system* S, const double* om, double* x2) {
  const int so = S->so, sv = S->sv, to = S->to, tv = S->tv;
  int64_t dims[4] = {tv, to, tv, to};
  int64_t ss[4] = {int64_t(to) * tv * to, int64_t(tv) * to, to, 1};
  int64_t ds[4] = {int64_t(so) * sv * so, int64_t(sv) * so, so, 1};
  permute_f64(4, dims, om, ss, x2, ds, 1.0, 0.0, stm(S));
}

// Values (or tangents) of the CCSD-block inputs from full Lt / Ft-like buffers.
static void extract_box(mlcc_system* S, const double* Lt, const double* Ft, const double* x2,
                        DT& Lai, DT& Lac, DT& Lki, DT& Lkc, DT& Fvv, DT& Foo, DT& t) {
  const int no = S->no, to = S->to, tv = S->tv, nj = S->nj;
  Lai = box_view(S, nj, tv, to);
  Lac = box_view(S, nj, tv, tv);
  Lki = box_view(S, nj, to, to);
  Lkc = box_view(S, nj, to, tv);
  take_block(S, Lt, nj, no, tv, 0, to, Lai);
  take_block(S, Lt, nj, no, tv, no, tv, Lac);
  take_block(S, Lt, nj, 0, to, 0, to, Lki);
  take_block(S, Lt, nj, 0, to, no, tv, Lkc);
  Fvv.d = {tv, tv};
  Fvv.p = S->ws.get<double>(size_t(tv) * tv);
  Foo.d = {to, to};
  Foo.p = S->ws.get<double>(size_t(to) * to);
  take_block(S, Ft, 1, no, tv, no, tv, Fvv);
  take_block(S, Ft, 1, 0, to, 0, to, Foo);
  t.d = {tv, to, tv, to};
  t.p = S->ws.get<double>(size_t(tv) * to * tv * to);
  take_tbox(S, x2, t);
}

// ---------------------------------------------------------------------------------
// Residual. gs_mode: the P_S doubles are the analytic CC2 amplitudes of the current t1
// (written to x2_out, with the P_T part from tT); otherwise x2 is an independent input.
// om2 (full doubles, may be NULL) receives the P_S rows and, if om2 != NULL, the P_T rows;
// in gs_mode the compact P_T residual is written to om2 as [tv][to][tv][to] instead.
void omega_eval(mlcc_system* S, const double* t1, const double* x2, bool gs_mode,
                const double* tT, double* x2_out, double* om1, double* om2, double* energy) {
  cudaStream_t s = stm(S);
  const int n = S->n, no = S->no, nv = S->nv, nj = S->nj, so = S->so, sv = S->sv;
  const int64_t nn = int64_t(n) * n, dS = S->dS;
  S->prepared = false;
  sigma_graphs_free(S);
  operand_cache_clear(S->opcache);
  Scope sc(S->ws);
  dress(S, t1, S->Lt, S->ht);
  build_fock(S, S->ht, S->Lt, S->Ft);
  gather_vo(S, S->Lt, S->Lai);
  gather_ov(S, S->Lt, S->Lov);
  const double* xuse = x2;
  if (dS > 0) {
    double* g = S->ws.get<double>(size_t(S->nd));
    rank_gemm_f64(S, true, S->Lai, S->Lai, g, 1.0, 0.0);   // g~_aibj = Lt_ai Lt_bj
    if (gs_mode) {
      k_cc2_amp<<<nblk(S->nd), 256, 0, s>>>(g, S->eps, no, sv, so, S->tv, S->to, tT, x2_out);
      MLCC_CHECK_LAUNCH();
      xuse = x2_out;
    } else if (om2) {
      k_omega2_cc2<<<nblk(S->nd), 256, 0, s>>>(g, x2, S->eps, no, sv, so, S->tv, S->to, om2);
      MLCC_CHECK_LAUNCH();
    }
  }
  // CCSD doubles residual on P_T
  if (S->to > 0 && S->tv > 0 && om2) {
    Scope sb(S->ws);
    Dual Lai, Lac, Lki, Lkc, Fvv, Foo, t;
    extract_box(S, S->Lt, S->Ft, xuse, Lai.v, Lac.v, Lki.v, Lkc.v, Fvv.v, Foo.v, t.v);
    const int64_t tl = int64_t(S->tv) * S->to * S->tv * S->to;
    double* omT = gs_mode ? om2 : S->ws.get<double>(size_t(tl));
    ccsd_block(S, Mode::Value, Lai, Lac, Lki, Lkc, Fvv, Foo, t, omT, false, t1);
    if (!gs_mode) put_tbox(S, omT, om2);
  }
  // singles (Eq. mlcc2_omega_codable) with u from all doubles
  block2d(S, nv, no, S->Ft + int64_t(no) * n, n, om1, no, 1.0, 0.0);
  if (dS > 0) {
    make_u(S, xuse, S->u);
    rank_gemm_f64(S, false, S->Lov, S->u, S->Z, 1.0, 0.0);  // Z^J_(bi) = Lov^J_(cj) u_(cj)(bi)
    Gemm a;  // om1[A][i] += sum_J Lt^J[A][b] Z^J[b][i]
    a.M = nv; a.N = so; a.K = sv;
    a.A = S->Lt + int64_t(no) * n + no; a.lda = n; a.sA = nn;
    a.B = S->Z; a.ldb = so; a.sB = dS;
    a.C = om1; a.ldc = no; a.alpha = 1.0; a.beta = 1.0; a.batch = nj; a.reduce = true;
    gemm_f64(a, S->ws, s, smc(S));
    Gemm b;  // om1[a][I] -= sum_J Z^J[a][j] Lt^J[j][I]
    b.M = sv; b.N = no; b.K = so;
    b.A = S->Z; b.lda = so; b.sA = dS;
    b.B = S->Lt; b.ldb = n; b.sB = nn;
    b.C = om1; b.ldc = no; b.alpha = -1.0; b.beta = 1.0; b.batch = nj; b.reduce = true;
    gemm_f64(b, S->ws, s, smc(S));
    k_fov<<<nblk(dS), 256, 0, s>>>(S->Ft, n, no, sv, so, S->Fov);
    MLCC_CHECK_LAUNCH();
    double* tmp = S->ws.get<double>(size_t(dS));
    Gemm c;  // tmp_(ai) = u_(ai)(bj) F~_jb
    c.M = dS; c.N = 1; c.K = dS;
    c.A = S->u; c.lda = dS; c.B = S->Fov; c.ldb = 1; c.C = tmp; c.ldc = 1;
    gemm_f64(c, S->ws, s, smc(S));
    k_scatter_add_ai<<<nblk(dS), 256, 0, s>>>(tmp, sv, so, no, 1.0, om1);
    MLCC_CHECK_LAUNCH();
  }
  // energy (Eq. mlcc_energy)
  if (energy) {
    double* M = S->ws.get<double>(size_t(nj) * no * no);
    double* part = S->ws.get<double>(size_t(nj));
    double* e2 = S->ws.get<double>(1);
    Gemm m;  // M^J[I][K] = sum_B L^J_IB t_BK  (L~_ov = L_ov)
    m.M = no; m.N = no; m.K = nv;
    m.A = S->Lt + no; m.lda = n; m.sA = nn;
    m.B = t1; m.ldb = no; m.sB = 0;
    m.C = M; m.ldc = no; m.sC = int64_t(no) * no; m.batch = nj;
    gemm_f64(m, S->ws, s, smc(S));
    k_energy1<<<nj, 256, 0, s>>>(M, no, part);
    MLCC_CHECK_LAUNCH();
    if (dS > 0) {
      // sum_aibj u_aibj g_iajb = sum_J sum_(ai) Lov^J_(ai) Z^J_(ai)
      dots(S->Lov, 0, 1, S->Z, int64_t(nj) * dS, e2, S->ws, s);
    } else {
      fill(e2, 1, 0.0, s);
    }
    k_sum_plus<<<1, 256, 0, s>>>(part, nj, e2, energy);
    MLCC_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------------------------------
static void jacobian_intermediates(mlcc_system* S);

void jacobian_prepare(mlcc_system* S, const double* t1, const double* x2) {
  cudaStream_t s = stm(S);
  const int n = S->n, no = S->no, nv = S->nv, so = S->so, sv = S->sv;
  const int64_t dS = S->dS;
  S->prepared = false;
  S->lowp_prec = -1;
  sigma_graphs_free(S);   // their kernels point into the caches cleared here
  operand_cache_clear(S->opcache);
  ccsd_cache_free(S);
  Scope sc(S->ws);
  MLCC_CUDA(cudaMemcpyAsync(S->t1gs, t1, size_t(nv) * no * 8, cudaMemcpyDeviceToDevice, s));
  if (S->nd)
    MLCC_CUDA(cudaMemcpyAsync(S->x2gs, x2, size_t(S->nd) * 8, cudaMemcpyDeviceToDevice, s));
  dress(S, S->t1gs, S->Lt, S->ht);
  build_fock(S, S->ht, S->Lt, S->Ft);
  gather_vo(S, S->Lt, S->Lai);
  gather_ov(S, S->Lt, S->Lov);
  if (dS > 0) {
    make_u(S, S->x2gs, S->u);
    rank_gemm_f64(S, false, S->Lov, S->u, S->Z, 1.0, 0.0);
    k_fov<<<nblk(dS), 256, 0, s>>>(S->Ft, n, no, sv, so, S->Fov);
    MLCC_CHECK_LAUNCH();
    jacobian_intermediates(S);
  }
  if (S->to > 0 && S->tv > 0) {
    Scope sb(S->ws);
    Dual Lai, Lac, Lki, Lkc, Fvv, Foo, t;
    extract_box(S, S->Lt, S->Ft, S->x2gs, Lai.v, Lac.v, Lki.v, Lkc.v, Fvv.v, Foo.v, t.v);
    const int64_t tl = int64_t(S->tv) * S->to * S->tv * S->to;
    double* omT = S->ws.get<double>(size_t(tl));
    ccsd_block(S, Mode::Value, Lai, Lac, Lki, Lkc, Fvv, Foo, t, omT, true, nullptr);
  }
  S->prepared = true;
}

// out[A][I] += alpha * sum_J d[J] X[J][r0 + A][c0 + I] over a rows x cols block
namespace {
// out[A][I] += alpha sum_J d[J] X^J[r0 + A][c0 + I]. blockIdx.y takes J in [y jc, (y + 1) jc)
// and writes its partial sums to part[y][rows * cols]; k_sum_over_J_add adds them in order
__global__ void k_sum_over_J(const double* d, const double* X, int nj, int n, int r0, int c0,
                             int rows, int cols, int jc, double* part) {
  const int64_t total = int64_t(rows) * cols, nn = int64_t(n) * n;
  const int j0 = int(blockIdx.y) * jc, j1 = min(nj, j0 + jc);
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int A = int(t / cols), I = int(t - int64_t(A) * cols);
    const double* x = X + int64_t(r0 + A) * n + c0 + I;
    double acc = 0.0;
    for (int J = j0; J < j1; ++J) acc = fma(d[J], x[J * nn], acc);
    part[int64_t(blockIdx.y) * total + t] = acc;
  }
}
__global__ void k_sum_over_J_add(const double* part, int nch, int rows, int cols, double alpha, double* out,
                                 int ldo) {
  const int64_t total = int64_t(rows) * cols;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nch; ++c) acc += part[int64_t(c) * total + t];
    const int A = int(t / cols), I = int(t - int64_t(A) * cols);
    out[int64_t(A) * ldo + I] += alpha * acc;
  }
}
// out[b*so + k] = F[k][b] for a [so][sv] block F
__global__ void k_to_fv(const double* F, int so, int sv, double* fv) {
  const int64_t total = int64_t(sv) * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int b = int(t / so), k = int(t - int64_t(b) * so);
    fv[t] = F[int64_t(k) * sv + b];
  }
}
// out[B][J] += alpha sum_K d[K] X^K[J][no + B] for B < nv, J < no (out [nv][no]); threads run
// along B so that the reads of X are contiguous
__global__ void k_sum_over_J_ov_tr(const double* d, const double* X, int nj, int n, int no, double alpha,
                                   double* out) {
  const int nv = n - no;
  const int64_t total = int64_t(nv) * no, nn = int64_t(n) * n;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int J = int(t / nv), B = int(t - int64_t(J) * nv);
    const double* x = X + int64_t(J) * n + no + B;
    double acc = 0.0;
    for (int K = 0; K < nj; ++K) acc = fma(d[K], x[K * nn], acc);
    out[int64_t(B) * no + J] += alpha * acc;
  }
}
// e[K] = sum_{A,I} X^K[no + A][I] l[A][I] (the virtual-occupied block); one block per K
__global__ void k_vo_dot(const double* X, int n, int no, const double* l, double* e) {
  __shared__ double red[256];
  const int K = blockIdx.x, nv = n - no;
  const double* x = X + int64_t(K) * n * n + int64_t(no) * n;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < int64_t(nv) * no; t += blockDim.x) {
    const int A = int(t / no), I = int(t - int64_t(A) * no);
    acc = fma(x[int64_t(A) * n + I], l[t], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) e[K] = red[0];
}
// out[a*so + i] = l[a*no + i] (the CC2-active singles)
__global__ void k_gather_act(const double* l, int sv, int so, int no, double* out) {
  const int64_t total = int64_t(sv) * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(t / so), i = int(t - int64_t(a) * so);
    out[t] = l[int64_t(a) * no + i];
  }
}
// out[k*sv + c] = fv[c*so + k]
__global__ void k_fv_to_kc(const double* fv, int so, int sv, double* out) {
  const int64_t total = int64_t(sv) * so;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int k = int(t / sv), c = int(t - int64_t(k) * sv);
    out[t] = fv[int64_t(c) * so + k];
  }
}
// G[p][q] += alpha x[p] y[q] (p, q < m)
__global__ void k_outer_add(const double* x, const double* y, int64_t m, double alpha, double* G) {
  const int64_t total = m * m;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = t / m, q = t - p * m;
    G[t] += alpha * x[p] * y[q];
  }
}
}  // namespace

static void sum_over_J(mlcc_system* S, const double* d, const double* X, int r0, int c0, int rows,
                       int cols, double alpha, double* out, int ldo) {
  if (rows <= 0 || cols <= 0) return;
  // the sum over J runs in chunks on blockIdx.y, enough blocks to fill the GPU
  const int64_t total = int64_t(rows) * cols;
  const int64_t eb = std::min<int64_t>((total + 255) / 256, 65535);
  const int nch = int(std::max<int64_t>(1, std::min<int64_t>({(4LL * smc(S) + eb - 1) / eb, S->nj, 64})));
  const int jc = (S->nj + nch - 1) / nch;
  const int ny = (S->nj + jc - 1) / jc;
  Scope sc(S->ws);
  double* part = S->ws.get<double>(size_t(ny) * total);
  k_sum_over_J<<<dim3(unsigned(eb), unsigned(ny), 1), 256, 0, stm(S)>>>(d, X, S->nj, S->n, r0, c0, rows, cols, jc,
                                                                       part);
  MLCC_CHECK_LAUNCH();
  k_sum_over_J_add<<<nblk(total), 256, 0, stm(S)>>>(part, ny, rows, cols, alpha, out, ldo);
  MLCC_CHECK_LAUNCH();
}

// batched over J: C^J (M x N) = alpha A^J B^J + beta C^J, with per-J strides (0: shared)
static void bgemm(mlcc_system* S, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                  int64_t lda, int64_t sA, bool ta, const double* B, int64_t ldb, int64_t sB, bool tb,
                  double beta, double* C, int64_t ldc, int64_t sC, bool reduce) {
  if (M <= 0 || N <= 0) return;
  Gemm g;
  g.ta = ta; g.tb = tb;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.sA = sA;
  g.B = B; g.ldb = ldb; g.sB = sB;
  g.C = C; g.ldc = ldc; g.sC = sC;
  g.alpha = alpha; g.beta = beta;
  g.batch = S->nj;
  g.reduce = reduce;
  gemm_f64(g, S->ws, stm(S), smc(S));
}
static void gemm1(mlcc_system* S, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                  int64_t lda, bool ta, const double* B, int64_t ldb, bool tb, double beta, double* C,
                  int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  Gemm g;
  g.ta = ta; g.tb = tb;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta;
  gemm_f64(g, S->ws, stm(S), smc(S));
}

// Intermediates of the Jacobian transformation that do not depend on the trial vector
// (Appendix A, MLCC2 Jacobian): X_Ji = g~_Jbkc u^{cb}_{ki} = sum_K Lt^K_Jb Z^K_bi and
// Y_aB = g~_kcjB u^{ac}_{jk} = sum_K Z^K_aj Lt^K_jB.
static void jacobian_intermediates(mlcc_system* S) {
  const int n = S->n, no = S->no, nv = S->nv, so = S->so, sv = S->sv;
  const int64_t nn = int64_t(n) * n, dS = S->dS;
  if (dS == 0) return;
  // X[J][i]: M = no, N = so, K = sv per Cholesky vector, summed
  bgemm(S, no, so, sv, 1.0, S->Lt + no, n, nn, false, S->Z, so, dS, false, 0.0, S->Xji, so, 0, true);
  // Y[a][B]: M = sv, N = nv, K = so
  bgemm(S, sv, nv, so, 1.0, S->Z, so, dS, false, S->Lt + no, n, nn, false, 0.0, S->Yab, nv, 0, true);
}

// sigma = dOmega/dh (x_gs + h c) for one trial vector c = (c1, c2), evaluated with the
// terms of Appendix A: the CCS terms of Eq. mlcc_A_, the MLCC2 singles terms with the
// intermediates X and Y, the doubles-to-singles terms, the CC2 doubles
// (L~_bC c_Cj - c_bK L~_Kj) L~_ai symmetrised plus eps c, and the CCSD rows as the tangent
// of the MLCCSD doubles residual.
void sigma_eval(mlcc_system* S, const double* c, double* sigma, int precision, unsigned parts) {
  if (!S->prepared) throw Error(MLCC_E_STATE, "mlcc_sigma: call mlcc_jacobian_prepare first");
  cudaStream_t s = stm(S);
  if (precision != MLCC_FP64 && S->opcache) {
    std::vector<std::pair<const char*, size_t>> r = {{S->persist.base(), S->persist.capacity()}};
    if (S->ccsd) r.push_back({S->ccsd->arena_base(), S->ccsd->arena_size()});
    operand_cache_set_ranges(S->opcache, r);
  }
  LowpScope lowp(precision == MLCC_FP64 ? 0 : precision, S->tc_err, S->opcache);
  // rest: the terms that do not sum over the Cholesky vectors (all but SIGMA_J_ONLY)
  const bool rest = !(parts & SIGMA_J_ONLY);
  const int n = S->n, no = S->no, nv = S->nv, nj = S->nj, so = S->so, sv = S->sv;
  const int to = S->to, tv = S->tv;
  const int64_t nn = int64_t(n) * n, dS = S->dS, vo = int64_t(nv) * no;
  const double* c1 = c;
  const double* c2 = c + vo;
  double* s1 = sigma;
  double* s2 = sigma + vo;
  const double* Lvv = S->Lt + int64_t(no) * n + no;   // Lt^J[no+A][no+B]
  const double* Lvo = S->Lt + int64_t(no) * n;        // Lt^J[no+A][I]
  const double* Lov = S->Lt + no;                     // Lt^J[I][no+A]
  const double* Loo = S->Lt;                          // Lt^J[I][K]
  Scope sc(S->ws);
  PhaseMarks phase(S);
  phase.mark("sigma_singles");
  // Xc^J = Lt^J_AB c_BI (the steepest CCS contraction) and the tangent of the
  // virtual-occupied block dLt^J_AI = Xc^J_AI - c_AK Lt^J_KI
  double* Xc = S->ws.get<double>(size_t(nj) * vo);
  bgemm(S, nv, no, nv, 1.0, Lvv, n, nn, false, c1, no, 0, false, 0.0, Xc, no, vo, false);
  double* dvo = S->ws.get<double>(size_t(nj) * vo);
  MLCC_CUDA(cudaMemcpyAsync(dvo, Xc, size_t(nj) * vo * 8, cudaMemcpyDeviceToDevice, s));
  bgemm(S, nv, no, no, -1.0, c1, no, 0, false, Loo, n, nn, false, 1.0, dvo, no, vo, false);
  // Q^J_IK = Lt^J_IB c_BK; d_J = tr Q^J is the tangent of sum_I Lt^J_II
  double* dJ = S->ws.get<double>(size_t(nj));
  {
    double* Q = S->ws.get<double>(size_t(nj) * no * no);
    bgemm(S, no, no, nv, 1.0, Lov, n, nn, false, c1, no, 0, false, 0.0, Q, no, int64_t(no) * no, false);
    const int warps = 8;
    k_trace_occ<<<(nj + warps - 1) / warps, 32 * warps, 0, s>>>(Q, nj, no, no, dJ);
    MLCC_CHECK_LAUNCH();
    // CCS: s1 = F~_AB c_BI - c_AJ F~_JI + 2 d_J Lt^J_AI - (Lt^J_AB c_BJ) Lt^J_JI
    if (rest) {
      gemm1(S, nv, no, nv, 1.0, S->Ft + int64_t(no) * n + no, n, false, c1, no, false, 0.0, s1, no);
      gemm1(S, nv, no, no, -1.0, c1, no, false, S->Ft, n, false, 1.0, s1, no);
    } else {
      fill(s1, vo, 0.0, s);
    }
    sum_over_J(S, dJ, S->Lt, no, 0, nv, no, 2.0, s1, no);
    bgemm(S, nv, no, no, -1.0, Xc, no, vo, false, Loo, n, nn, false, 1.0, s1, no, 0, true);
    if (dS > 0) {
      // MLCC2 singles: - c_AJ X_Ji - Y_aB c_BI
      if (rest) {
        gemm1(S, nv, so, no, -1.0, c1, no, false, S->Xji, so, false, 1.0, s1, no);
        gemm1(S, sv, no, nv, -1.0, S->Yab, nv, false, c1, no, false, 1.0, s1, no);
      }
      // tangent of F~_kc (k, c active): 2 d_J Lt^J_kc - (Lt^J_kB c_BJ) Lt^J_Jc
      double* dF = S->ws.get<double>(size_t(so) * sv);
      fill(dF, int64_t(so) * sv, 0.0, s);
      sum_over_J(S, dJ, S->Lt, 0, no, so, sv, 2.0, dF, sv);
      // Q^J[k][J'] for k < so is the leading block of Q: (Q^J)[k][J'] Lt^J[J'][no+c]
      bgemm(S, so, sv, no, -1.0, Q, no, int64_t(no) * no, false, Lov, n, nn, false, 1.0, dF, sv, 0, true);
      double* dfv = S->ws.get<double>(size_t(dS));
      k_to_fv<<<nblk(dS), 256, 0, s>>>(dF, so, sv, dfv);
      MLCC_CHECK_LAUNCH();
      phase.mark("sigma_doubles_to_singles");
      if (parts & SIGMA_DOUBLES_TO_SINGLES) {
        // doubles -> singles
        double* uc = S->ws.get<double>(size_t(S->nd));
        make_u(S, c2, uc);
        double* Zc = S->ws.get<double>(size_t(nj) * dS);
        rank_gemm(S, precision, false, S->Lov, uc, Zc, 1.0, 0.0);
        double* tmp = S->ws.get<double>(size_t(dS));
        gemm1(S, dS, 1, dS, 1.0, S->u, dS, false, dfv, 1, false, 0.0, tmp, 1);
        if (rest) gemm1(S, dS, 1, dS, 1.0, uc, dS, false, S->Fov, 1, false, 1.0, tmp, 1);
        k_scatter_add_ai<<<nblk(dS), 256, 0, s>>>(tmp, sv, so, no, 1.0, s1);
        MLCC_CHECK_LAUNCH();
        // (u(c)^{bc}_{ij} Lt^K_jc) Lt^K_Ab  and  - (u(c)^{ab}_{jk} Lt^K_kb) Lt^K_jI
        bgemm(S, nv, so, sv, 1.0, Lvv, n, nn, false, Zc, so, dS, false, 1.0, s1, no, 0, true);
        bgemm(S, sv, no, so, -1.0, Zc, so, dS, false, Loo, n, nn, false, 1.0, s1, no, 0, true);
      }
      phase.mark("sigma_cc2_doubles");
      if (parts & SIGMA_CC2_DOUBLES) {
        // CC2 doubles on P_S
        double* V = S->ws.get<double>(size_t(nj) * dS);
        {
          int64_t dims[3] = {nj, sv, so}, ss[3] = {vo, no, 1}, ds[3] = {dS, so, 1};
          permute_f64(3, dims, dvo, ss, V, ds, 1.0, 0.0, s);
        }
        double* W = S->ws.get<double>(size_t(S->nd));
        rank_gemm(S, precision, true, S->Lai, V, W, 1.0, 0.0);
        dim3 blk(32, 8), grd(unsigned((dS + 31) / 32), unsigned((dS + 31) / 32));
        k_sigma2_cc2<<<grd, blk, 0, s>>>(W, c2, S->eps, no, sv, so, tv, to, rest ? 1.0 : 0.0, s2);
        MLCC_CHECK_LAUNCH();
      }
    }
    phase.mark("sigma_ccsd_rows");
    // CCSD rows: tangent of the CCSD residual around the cached values
    if ((parts & SIGMA_CCSD_ROWS) && to > 0 && tv > 0) {
      Scope sb(S->ws);
      const int64_t oo = int64_t(no) * no;
      Dual Lai, Lac, Lki, Lkc, Fvv, Foo, t;
      Lai.d = box_view(S, nj, tv, to);
      {
        int64_t dims[3] = {nj, tv, to}, ss[3] = {vo, no, 1}, ds[3] = {int64_t(tv) * to, to, 1};
        permute_f64(3, dims, dvo, ss, Lai.d.p, ds, 1.0, 0.0, s);
      }
      // dLt_ac = - c_aK Lt_Kc ; dLt_ki = Lt_kA c_Ai ; dLt_kc = 0
      Lac.d = box_view(S, nj, tv, tv);
      bgemm(S, tv, tv, no, -1.0, c1, no, 0, false, Lov, n, nn, false, 0.0, Lac.d.p, tv, int64_t(tv) * tv, false);
      Lki.d = box_view(S, nj, to, to);
      {
        // the leading to x to block of Q^J = Lt^J_ov c1
        int64_t dims[3] = {nj, to, to}, ss[3] = {oo, no, 1}, ds[3] = {int64_t(to) * to, to, 1};
        permute_f64(3, dims, Q, ss, Lki.d.p, ds, 1.0, 0.0, s);
      }
      // dF~_bc = dh~_bc + 2 (dLt^J_bc D_J + Lt^J_bc d_J) - dLt^J_bI Lt^J_Ic, dh~_bc = - c_bK h~_Kc
      Fvv.d.d = {tv, tv};
      Fvv.d.p = S->ws.get<double>(size_t(tv) * tv);
      double* D = S->ws.get<double>(size_t(nj));
      trace_occ(S, S->Lt, D);
      if (rest) gemm1(S, tv, tv, no, -1.0, c1, no, false, S->ht + no, n, false, 0.0, Fvv.d.p, tv);
      else fill(Fvv.d.p, int64_t(tv) * tv, 0.0, s);
      {
        Gemm g;  // + 2 sum_J D_J dLac^J  (M = 1 over the flattened tv*tv block)
        g.M = 1; g.N = int64_t(tv) * tv; g.K = nj;
        g.A = D; g.lda = nj; g.B = Lac.d.p; g.ldb = int64_t(tv) * tv; g.C = Fvv.d.p; g.ldc = int64_t(tv) * tv;
        g.alpha = 2.0; g.beta = 1.0;
        gemm_f64(g, S->ws, s, smc(S));
      }
      sum_over_J(S, dJ, S->Lt, no, no, tv, tv, 2.0, Fvv.d.p, tv);
      bgemm(S, tv, tv, no, -1.0, dvo, no, vo, false, Lov, n, nn, false, 1.0, Fvv.d.p, tv, 0, true);
      // dF~_kj = dh~_kj + 2 (dLt^J_kj D_J + Lt^J_kj d_J) - dLt^J_kI Lt^J_Ij - Lt^J_kI dLt^J_Ij
      //   with dh~_kj = h~_kA c_Aj and dLt^J_kI = Q^J[k][I]
      Foo.d.d = {to, to};
      Foo.d.p = S->ws.get<double>(size_t(to) * to);
      if (rest) gemm1(S, to, to, nv, 1.0, S->ht + no, n, false, c1, no, false, 0.0, Foo.d.p, to);
      else fill(Foo.d.p, int64_t(to) * to, 0.0, s);
      {
        Gemm g;
        g.M = 1; g.N = int64_t(to) * to; g.K = nj;
        g.A = D; g.lda = nj; g.B = Lki.d.p; g.ldb = int64_t(to) * to; g.C = Foo.d.p; g.ldc = int64_t(to) * to;
        g.alpha = 2.0; g.beta = 1.0;
        gemm_f64(g, S->ws, s, smc(S));
      }
      sum_over_J(S, dJ, S->Lt, 0, 0, to, to, 2.0, Foo.d.p, to);
      bgemm(S, to, to, no, -1.0, Q, no, oo, false, Loo, n, nn, false, 1.0, Foo.d.p, to, 0, true);
      bgemm(S, to, to, no, -1.0, Loo, n, nn, false, Q, no, oo, false, 1.0, Foo.d.p, to, 0, true);
      t.d.d = {tv, to, tv, to};
      t.d.p = S->ws.get<double>(size_t(tv) * to * tv * to);
      if (rest) take_tbox(S, c2, t.d);
      else fill(t.d.p, t.d.size(), 0.0, s);   // the trial doubles enter only with the cached values
      Lkc.d.d = {nj, to, tv};   // zero tangent (occupied-virtual block is unchanged)
      const int64_t tl = int64_t(tv) * to * tv * to;
      double* omT = S->ws.get<double>(size_t(tl));
      ccsd_block(S, Mode::Tangent, Lai, Lac, Lki, Lkc, Fvv, Foo, t, omT, false, c1, rest);
      put_tbox(S, omT, s2);
    }
  }
}

// Left transformation rho = A^T l for a system without a CCSD level: the adjoint of the
// Jacobian transformation above in the plain inner product of the vector storage, on
// symmetric doubles (the doubles of rho are symmetrised). Each term of sigma_eval has its
// transpose here, in the same notation (K the Cholesky index; A, B, I, J all virtual /
// occupied orbitals; a, b, i, j CC2-active ones):
//   CCS:    F~_vv^T l - l F~_oo^T + 2 sum_K (e_K + gamma_K) Lt^K[J][B]^T
//           - sum_K Lt^K_vv^T (l Lt^K_oo^T),        e_K = <Lt^K_vo, l>
//   MLCC2:  the F~_kc tangent through lambda = u l_act (gamma_K = <Lt^K_ov, lambda>, Phi^K),
//           - l X^T, - Y^T l
//   doubles -> singles: Psi^K_bj = Lt^K_vv^T l - l Lt^K_oo^T (active), Gamma = Lov^T Psi
//           + l_act F~_ov^T, the doubles of rho = make_u(Gamma) symmetrised + eps l2
//   singles -> doubles: M = 2 Lai l2, rho1 += Lt_vv^T M - M Lt_oo^T (active)
void sigma_left_eval(mlcc_system* S, const double* l, double* rho, int precision) {
  if (!S->prepared) throw Error(MLCC_E_STATE, "left transformation: call mlcc_jacobian_prepare first");
  if (S->to > 0 && S->tv > 0)
    throw Error(MLCC_E_ARG, "left transformation: systems with a CCSD level are not supported");
  cudaStream_t s = stm(S);
  if (precision != MLCC_FP64 && S->opcache) {
    std::vector<std::pair<const char*, size_t>> r = {{S->persist.base(), S->persist.capacity()}};
    operand_cache_set_ranges(S->opcache, r);
  }
  LowpScope lowp(precision == MLCC_FP64 ? 0 : precision, S->tc_err, S->opcache);
  const int n = S->n, no = S->no, nv = S->nv, nj = S->nj, so = S->so, sv = S->sv;
  const int64_t nn = int64_t(n) * n, dS = S->dS, vo = int64_t(nv) * no;
  const double* l1 = l;
  const double* l2 = l + vo;
  double* r1 = rho;
  double* r2 = rho + vo;
  const double* Lvv = S->Lt + int64_t(no) * n + no;   // Lt^K[no+A][no+B]
  const double* Lov = S->Lt + no;                     // Lt^K[I][no+A]
  const double* Loo = S->Lt;                          // Lt^K[I][J]
  Scope sc(S->ws);
  // CCS: F~_vv^T l - l F~_oo^T
  gemm1(S, nv, no, nv, 1.0, S->Ft + int64_t(no) * n + no, n, true, l1, no, false, 0.0, r1, no);
  gemm1(S, nv, no, no, -1.0, l1, no, false, S->Ft, n, true, 1.0, r1, no);
  double* e = S->ws.get<double>(size_t(nj));
  k_vo_dot<<<nj, 256, 0, s>>>(S->Lt, n, no, l1, e);
  MLCC_CHECK_LAUNCH();
  double* lact = nullptr;
  double* lam = nullptr;
  if (dS > 0) {
    lact = S->ws.get<double>(size_t(dS));
    k_gather_act<<<nblk(dS), 256, 0, s>>>(l1, sv, so, no, lact);
    MLCC_CHECK_LAUNCH();
    lam = S->ws.get<double>(size_t(dS));
    gemm1(S, dS, 1, dS, 1.0, S->u, dS, false, lact, 1, false, 0.0, lam, 1);
    gemm1(S, nj, 1, dS, 1.0, S->Lov, dS, false, lam, 1, false, 1.0, e, 1);   // + gamma_K
  }
  k_sum_over_J_ov_tr<<<nblk(vo), 256, 0, s>>>(e, S->Lt, nj, n, no, 2.0, r1);
  MLCC_CHECK_LAUNCH();
  {
    Scope st(S->ws);
    double* T = S->ws.get<double>(size_t(nj) * vo);
    bgemm(S, nv, no, no, 1.0, l1, no, 0, false, Loo, n, nn, true, 0.0, T, no, vo, false);
    bgemm(S, nv, no, nv, -1.0, Lvv, n, nn, true, T, no, vo, false, 1.0, r1, no, 0, true);
  }
  if (dS == 0) return;
  {
    // the F~_kc tangent: Phi^K[k][J] = sum_c Lam[k][c] Lt^K[J][no+c]
    Scope st(S->ws);
    double* Lam = S->ws.get<double>(size_t(so) * sv);
    k_fv_to_kc<<<nblk(dS), 256, 0, s>>>(lam, so, sv, Lam);
    MLCC_CHECK_LAUNCH();
    double* Phi = S->ws.get<double>(size_t(nj) * so * no);
    bgemm(S, so, no, sv, 1.0, Lam, sv, 0, false, Lov, n, nn, true, 0.0, Phi, no, int64_t(so) * no, false);
    bgemm(S, nv, no, so, -1.0, Lov, n, nn, true, Phi, no, int64_t(so) * no, false, 1.0, r1, no, 0, true);
  }
  // - l X^T, - Y^T l
  gemm1(S, nv, no, so, -1.0, l1, no, false, S->Xji, so, true, 1.0, r1, no);
  gemm1(S, nv, no, sv, -1.0, S->Yab, nv, true, l1, no, false, 1.0, r1, no);
  // doubles <- singles (the transpose of the doubles-to-singles terms)
  {
    Scope st(S->ws);
    double* Psi = S->ws.get<double>(size_t(nj) * dS);
    bgemm(S, sv, so, nv, 1.0, Lvv, n, nn, true, l1, no, 0, false, 0.0, Psi, so, dS, false);
    bgemm(S, sv, so, no, -1.0, l1, no, 0, false, Loo, n, nn, true, 1.0, Psi, so, dS, false);
    double* Gam = S->ws.get<double>(size_t(S->nd));
    rank_gemm(S, precision, true, S->Lov, Psi, Gam, 1.0, 0.0);
    k_outer_add<<<nblk(S->nd), 256, 0, s>>>(lact, S->Fov, dS, 1.0, Gam);
    MLCC_CHECK_LAUNCH();
    double* G = S->ws.get<double>(size_t(S->nd));
    make_u(S, Gam, G);
    axpby(G, G, S->nd, 0.0, 0.5, s);
    dim3 blk(32, 8), grd(unsigned((dS + 31) / 32), unsigned((dS + 31) / 32));
    k_sigma2_cc2<<<grd, blk, 0, s>>>(G, l2, S->eps, no, sv, so, 0, 0, 1.0, r2);   // G + G^T + eps l2
    MLCC_CHECK_LAUNCH();
  }
  // singles <- doubles (the transpose of the CC2 doubles rows): M = 2 Lai l2
  {
    Scope st(S->ws);
    double* M = S->ws.get<double>(size_t(nj) * dS);
    rank_gemm(S, precision, false, S->Lai, l2, M, 2.0, 0.0);
    bgemm(S, nv, so, sv, 1.0, Lvv, n, nn, true, M, so, dS, false, 1.0, r1, no, 0, true);
    bgemm(S, sv, no, so, -1.0, M, so, dS, false, Loo, n, nn, true, 1.0, r1, no, 0, true);
  }
}

}  // namespace mlcc

// MO-screened pivoted Cholesky decomposition of the AO two-electron integral matrix and the
// MO Cholesky vectors built from its basis (Sec. 2.4).
//
// Decomposition: the rows and columns of g are AO pairs (ab); D is the updated diagonal,
// D~ = w D the screened one (w = nu_a nu_b, Eq. cd_screening, or 1). Each step takes the pair
// K with the largest D~ (a two-stage device argmax; the host reads the winner to decide the
// stop, Eq. standard_cholesky on D~), forms the new vector
//   L[:, J] = (g[:, K] - L[:, :J] L[K, :J]^T) / sqrt(D[K])
// (a matrix-vector product on the device) and updates D -= L[:, J]^2, D[K] = 0.
// MO vectors (Algorithm 1, the RI expression): S = g[B, B] = Q Q^T (host Cholesky and
// triangular inverse of the small basis block), X[K] = C^T g_K C for each basis pair K
// (batched GEMMs on the gathered rows g[K, :]), L^J = sum_K [Q^-1]_JK X[K] (one GEMM).
#include "internal.cuh"
#include "system.cuh"

#include <algorithm>
#include <cmath>

namespace mlcc {
namespace {

inline int nb_c(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096))); }

// w[ab] = nu_a nu_b, nu_a = max_p C[a][p]^2 (Eq. mo_screening, Eq. cd_screening)
__global__ void k_mo_screen(const double* __restrict__ C, int n_ao, int n_act, double* __restrict__ w) {
  const int64_t total = int64_t(n_ao) * n_ao;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(t / n_ao), b = int(t - int64_t(a) * n_ao);
    double na = 0.0, nb = 0.0;
    for (int p = 0; p < n_act; ++p) {
      const double x = C[int64_t(a) * n_act + p], y = C[int64_t(b) * n_act + p];
      na = fmax(na, x * x);
      nb = fmax(nb, y * y);
    }
    w[t] = na * nb;
  }
}

__global__ void k_diag_of(const double* __restrict__ g, int64_t m, double* __restrict__ D) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m; t += int64_t(gridDim.x) * blockDim.x)
    D[t] = g[t * m + t];
}

// stage 1: per block the largest w[t] D[t] (lowest index on ties)
__global__ void k_amax1(const double* __restrict__ D, const double* __restrict__ w, int64_t m, double* pv,
                        long long* pi) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double bv = -1.0;
  long long bi = -1;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m; t += int64_t(gridDim.x) * blockDim.x) {
    const double v = (w ? w[t] : 1.0) * D[t];
    if (v > bv) {
      bv = v;
      bi = t;
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double v = sv[threadIdx.x + s];
      const long long i = si[threadIdx.x + s];
      if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && i >= 0 && (si[threadIdx.x] < 0 || i < si[threadIdx.x]))) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}
// stage 2: out = {w D at the winner, D at the winner, winner index}
__global__ void k_amax2(const double* pv, const long long* pi, int nb, const double* __restrict__ D, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double bv = -1.0;
  long long bi = -1;
  for (int b = 0; b < nb; ++b)
    if (pi[b] >= 0 && (pv[b] > bv || (pv[b] == bv && pi[b] < bi))) {
      bv = pv[b];
      bi = pi[b];
    }
  out[0] = bv;
  out[1] = bi >= 0 ? D[bi] : 0.0;
  out[2] = double(bi);
}

// L[:, J] = col / sqrt(dK); D -= L[:, J]^2; D[K] = 0
__global__ void k_chol_step(const double* __restrict__ col, int64_t m, int64_t ldl, int J, int64_t K, double dK,
                            double* __restrict__ L, double* __restrict__ D) {
  const double f = 1.0 / sqrt(dK);
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < m; t += int64_t(gridDim.x) * blockDim.x) {
    const double l = col[t] * f;
    L[t * ldl + J] = l;
    D[t] = t == K ? 0.0 : D[t] - l * l;
  }
}

// rows[k][:] = g[piv[k]][:]
__global__ void k_gather_rows(const double* __restrict__ g, int64_t m, const int* __restrict__ piv, int nk,
                              double* __restrict__ rows) {
  const int64_t total = int64_t(nk) * m;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = t / m, c = t - k * m;
    rows[t] = g[int64_t(piv[k]) * m + c];
  }
}

}  // namespace
}  // namespace mlcc

using namespace mlcc;

extern "C" {

mlcc_status mlcc_mo_screening(mlcc_ctx* ctx, int32_t n_ao, int32_t n_active, const double* c_active_dev,
                              double* w_dev) {
  return guard([&] {
    MLCC_REQUIRE(ctx && c_active_dev && w_dev, "mlcc_mo_screening: NULL argument");
    MLCC_REQUIRE(n_ao > 0 && n_active > 0, "mlcc_mo_screening: sizes must be positive");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    k_mo_screen<<<nb_c(int64_t(n_ao) * n_ao), 256, 0, ctx->stream>>>(c_active_dev, n_ao, n_active, w_dev);
    MLCC_CHECK_LAUNCH();
    return MLCC_OK;
  });
}

mlcc_status mlcc_cholesky_decompose(mlcc_ctx* ctx, int64_t n_pairs, const double* g_dev, const double* w_dev,
                                    double tau, int32_t max_vectors, int32_t* pivots_host, double* l_dev,
                                    double* diag_dev, int32_t* n_vectors) {
  return guard([&] {
    MLCC_REQUIRE(ctx && g_dev && pivots_host && l_dev && n_vectors, "mlcc_cholesky_decompose: NULL argument");
    MLCC_REQUIRE(n_pairs > 0 && max_vectors > 0 && max_vectors <= n_pairs,
                 "mlcc_cholesky_decompose: need n_pairs > 0 and 0 < max_vectors <= n_pairs");
    MLCC_REQUIRE(tau >= 0.0, "mlcc_cholesky_decompose: tau must not be negative");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int64_t m = n_pairs, ldl = max_vectors;
    const int nb = nb_c(m);
    Arena ws;
    ws.reserve(size_t(m) * 8 * 2 + size_t(nb) * 16 + 64 + 8 * 256 + (size_t(1) << 24));
    double* D = ws.get<double>(size_t(m));
    double* col = ws.get<double>(size_t(m));
    double* pv = ws.get<double>(size_t(nb));
    long long* pi = ws.get<long long>(size_t(nb));
    double* out = ws.get<double>(4);
    k_diag_of<<<nb, 256, 0, s>>>(g_dev, m, D);
    MLCC_CHECK_LAUNCH();
    int J = 0;
    for (; J < max_vectors; ++J) {
      k_amax1<<<nb, 256, 0, s>>>(D, w_dev, m, pv, pi);
      MLCC_CHECK_LAUNCH();
      k_amax2<<<1, 32, 0, s>>>(pv, pi, nb, D, out);
      MLCC_CHECK_LAUNCH();
      double h[3];
      copy_d2h(h, out, 3, s);
      if (!(h[0] >= tau) || !(h[1] > 0.0) || h[2] < 0.0) break;   // Eq. standard_cholesky on D~
      const int64_t K = int64_t(h[2]);
      pivots_host[J] = int32_t(K);
      // col = g[K, :] - L[:, :J] L[K, :J]^T (g symmetric)
      MLCC_CUDA(cudaMemcpyAsync(col, g_dev + K * m, size_t(m) * 8, cudaMemcpyDeviceToDevice, s));
      if (J > 0) {
        Gemm gv;
        gv.M = m; gv.N = 1; gv.K = J;
        gv.A = l_dev; gv.lda = ldl;
        gv.B = l_dev + K * ldl; gv.ldb = 1;
        gv.C = col; gv.ldc = 1;
        gv.alpha = -1.0; gv.beta = 1.0;
        gemm_f64(gv, ws, s, ctx->sm_count);
      }
      k_chol_step<<<nb, 256, 0, s>>>(col, m, ldl, J, K, h[1], l_dev, D);
      MLCC_CHECK_LAUNCH();
    }
    if (diag_dev) MLCC_CUDA(cudaMemcpyAsync(diag_dev, D, size_t(m) * 8, cudaMemcpyDeviceToDevice, s));
    MLCC_CUDA(cudaStreamSynchronize(s));
    *n_vectors = J;
    return MLCC_OK;
  });
}

mlcc_status mlcc_cholesky_mo_vectors(mlcc_ctx* ctx, int32_t n_ao, int32_t n_mo, const double* g_dev,
                                     const int32_t* pivots_host, int32_t n_vectors, const double* c_dev,
                                     double* lmo_dev) {
  return guard([&] {
    MLCC_REQUIRE(ctx && g_dev && pivots_host && c_dev && lmo_dev, "mlcc_cholesky_mo_vectors: NULL argument");
    MLCC_REQUIRE(n_ao > 0 && n_mo > 0 && n_vectors > 0, "mlcc_cholesky_mo_vectors: sizes must be positive");
    const int64_t m = int64_t(n_ao) * n_ao, J = n_vectors, nmo2 = int64_t(n_mo) * n_mo;
    for (int k = 0; k < n_vectors; ++k)
      MLCC_REQUIRE(pivots_host[k] >= 0 && pivots_host[k] < m, "mlcc_cholesky_mo_vectors: pivot out of range");
    MLCC_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    Arena ws;
    ws.reserve(size_t(J) * 4 + size_t(J) * m * 8 + size_t(J) * n_ao * n_mo * 8 + size_t(J) * nmo2 * 8 +
               size_t(J) * J * 8 + 16 * 256 + (size_t(1) << 26));
    int* dpiv = ws.get<int>(size_t(J));
    MLCC_CUDA(cudaMemcpyAsync(dpiv, pivots_host, size_t(J) * 4, cudaMemcpyHostToDevice, s));
    double* rows = ws.get<double>(size_t(J) * m);
    k_gather_rows<<<nb_c(J * m), 256, 0, s>>>(g_dev, m, dpiv, int(J), rows);
    MLCC_CHECK_LAUNCH();
    // S = g[B, B] (host), S = Q Q^T, Qi = Q^-1
    std::vector<double> Sh(size_t(J) * J), rowh(size_t(m));
    {
      std::vector<double> all(size_t(J) * m);
      copy_d2h(all.data(), rows, J * m, s);
      for (int64_t a = 0; a < J; ++a)
        for (int64_t b = 0; b < J; ++b) Sh[size_t(a * J + b)] = all[size_t(a * m + pivots_host[b])];
    }
    std::vector<double> Q(size_t(J) * J, 0.0), Qi(size_t(J) * J, 0.0);
    for (int64_t j = 0; j < J; ++j) {
      double d = Sh[size_t(j * J + j)];
      for (int64_t k = 0; k < j; ++k) d -= Q[size_t(j * J + k)] * Q[size_t(j * J + k)];
      if (!(d > 0.0)) throw Error(MLCC_E_ARG, "mlcc_cholesky_mo_vectors: the basis block is not positive definite");
      const double q = std::sqrt(d);
      Q[size_t(j * J + j)] = q;
      for (int64_t i = j + 1; i < J; ++i) {
        double v = Sh[size_t(i * J + j)];
        for (int64_t k = 0; k < j; ++k) v -= Q[size_t(i * J + k)] * Q[size_t(j * J + k)];
        Q[size_t(i * J + j)] = v / q;
      }
    }
    for (int64_t c = 0; c < J; ++c) {   // forward substitution, column c of Q^-1
      for (int64_t i = c; i < J; ++i) {
        double v = i == c ? 1.0 : 0.0;
        for (int64_t k = c; k < i; ++k) v -= Q[size_t(i * J + k)] * Qi[size_t(k * J + c)];
        Qi[size_t(i * J + c)] = v / Q[size_t(i * J + i)];
      }
    }
    double* dQi = ws.get<double>(size_t(J) * J);
    copy_h2d(dQi, Qi.data(), J * J, s);
    // X[K] = C^T g_K C: T[K] = g_K C, X[K] = C^T T[K]
    double* T = ws.get<double>(size_t(J) * n_ao * n_mo);
    double* X = ws.get<double>(size_t(J) * nmo2);
    Gemm g1;
    g1.M = n_ao; g1.N = n_mo; g1.K = n_ao;
    g1.A = rows; g1.lda = n_ao; g1.sA = m;
    g1.B = c_dev; g1.ldb = n_mo; g1.sB = 0;
    g1.C = T; g1.ldc = n_mo; g1.sC = int64_t(n_ao) * n_mo;
    g1.batch = J;
    gemm_f64(g1, ws, s, ctx->sm_count);
    Gemm g2;
    g2.ta = true;
    g2.M = n_mo; g2.N = n_mo; g2.K = n_ao;
    g2.A = c_dev; g2.lda = n_mo; g2.sA = 0;
    g2.B = T; g2.ldb = n_mo; g2.sB = int64_t(n_ao) * n_mo;
    g2.C = X; g2.ldc = n_mo; g2.sC = nmo2;
    g2.batch = J;
    gemm_f64(g2, ws, s, ctx->sm_count);
    // L^J = sum_K [Q^-1]_JK X[K]
    Gemm g3;
    g3.M = J; g3.N = nmo2; g3.K = J;
    g3.A = dQi; g3.lda = J;
    g3.B = X; g3.ldb = nmo2;
    g3.C = lmo_dev; g3.ldc = nmo2;
    gemm_f64(g3, ws, s, ctx->sm_count);
    MLCC_CUDA(cudaStreamSynchronize(s));
    return MLCC_OK;
  });
}

}  // extern "C"

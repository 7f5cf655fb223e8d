// mlcc_fock_t1_noalloc: the X1-basis Fock matrix and dressed Cholesky vectors without any
// device allocation. Its only scratch (the occupied traces of L^J and Lt^J, two doubles per
// Cholesky vector) lives in a file-scope device array; the caller owns every other buffer.
//
// Why: some callers cannot let a library allocate device memory. A host program that
// reserves the device memory for its own pool leaves nothing for cudaMalloc, or must keep
// every allocation under its accounting; and cudaMalloc / cudaFree can synchronise the
// device, which a caller interleaving its own work on other streams may not accept.
#include "internal.cuh"

namespace mlcc {

namespace {
constexpr int kMaxChol = MLCC_NOALLOC_MAX_CHOL;
// [0, kMaxChol): D_J = sum_I L^J_II;  [kMaxChol, 2 kMaxChol): the same for Lt^J
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxChol];

// Address of the scratch array on the current device. It is looked up on every call (a
// cheap query) rather than cached, so it stays valid after the caller resets the device
// or makes another context current.
double* scratch_for_current_device() {
  void* p = nullptr;
  MLCC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  return static_cast<double*>(p);
}

inline int blocks_for(int64_t n) {
  return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16384)));
}

// D[J] = sum_{I < no} X[J][I][I]; one warp per Cholesky vector
__global__ void k_na_trace(const double* X, int nj, int n, int no, double* D) {
  const int J = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (J >= nj) return;
  const double* x = X + int64_t(J) * n * n;
  double s = 0.0;
  for (int I = lane; I < no; I += 32) s += x[int64_t(I) * n + I];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) D[J] = s;
}
// left factor (1 - t): Y[p][q] = X[p][q] - [p vir] sum_i t[p-no][i] X[i][q]   (batched)
__global__ void k_na_left(const double* X, const double* t1, int batch, int n, int no, double* Y) {
  const int64_t nn = int64_t(n) * n, total = nn * batch;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t J = e / nn, r = e - J * nn;
    const int p = int(r / n), q = int(r - int64_t(p) * n);
    const double* x = X + J * nn;
    double v = x[r];
    if (p >= no) {
      const double* tp = t1 + int64_t(p - no) * no;
      for (int i = 0; i < no; ++i) v -= tp[i] * x[int64_t(i) * n + q];
    }
    Y[e] = v;
  }
}
// right factor (1 + t), in place: Y[p][q] += [q occ] sum_a Y[p][no+a] t[a][q]
// (reads only virtual columns, writes only occupied columns)
__global__ void k_na_right(double* Y, const double* t1, int batch, int n, int no) {
  const int nv = n - no;
  const int64_t total = int64_t(batch) * n * no;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = e / no;   // J * n + p
    const int q = int(e - row * no);
    double* y = Y + row * n;
    double acc = 0.0;
    for (int a = 0; a < nv; ++a) acc += y[no + a] * t1[int64_t(a) * no + q];
    y[q] += acc;
  }
}
// F[p][q] += sgn * (2 sum_J X[J][p][q] D[J] - sum_J sum_I X[J][p][I] X[J][I][q])
__global__ void k_na_two_electron(const double* X, const double* D, int nj, int n, int no, double sgn,
                                  double* F) {
  const int64_t nn = int64_t(n) * n;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nn;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int p = int(e / n), q = int(e - int64_t(p) * n);
    double coul = 0.0, exch = 0.0;
    for (int J = 0; J < nj; ++J) {
      const double* x = X + int64_t(J) * nn;
      coul += x[e] * D[J];
      for (int I = 0; I < no; ++I) exch += x[int64_t(p) * n + I] * x[int64_t(I) * n + q];
    }
    F[e] += sgn * (2.0 * coul - exch);
  }
}
}  // namespace

}  // namespace mlcc

using namespace mlcc;

extern "C" mlcc_status mlcc_fock_t1_noalloc(int32_t n_mo, int32_t n_occ, int32_t n_chol,
                                           const double* chol_dev, const double* fock_dev,
                                           const double* t1_dev, double* lt_dev, double* ft_dev,
                                           void* stream) {
  try {
    MLCC_REQUIRE(chol_dev && fock_dev && t1_dev && lt_dev && ft_dev,
                 "mlcc_fock_t1_noalloc: NULL argument");
    MLCC_REQUIRE(n_mo > 0 && n_occ > 0 && n_occ < n_mo, "mlcc_fock_t1_noalloc: need 0 < n_occ < n_mo");
    MLCC_REQUIRE(n_chol > 0, "mlcc_fock_t1_noalloc: n_chol must be positive");
    if (n_chol > kMaxChol)
      throw Error(MLCC_E_ARG, "mlcc_fock_t1_noalloc: n_chol " + std::to_string(n_chol) +
                                  " exceeds the scratch limit MLCC_NOALLOC_MAX_CHOL = " +
                                  std::to_string(kMaxChol));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = scratch_for_current_device();
    double* D = scratch;              // occupied traces of L^J
    double* Dt = scratch + kMaxChol;  // occupied traces of Lt^J
    const int n = n_mo, no = n_occ, nj = n_chol;
    const int64_t nn = int64_t(n) * n;
    const int warps = 8;
    // Lt = (1 - t) L (1 + t) into the caller's buffer
    k_na_left<<<blocks_for(nn * nj), 256, 0, s>>>(chol_dev, t1_dev, nj, n, no, lt_dev);
    MLCC_CHECK_LAUNCH();
    k_na_right<<<blocks_for(int64_t(nj) * n * no), 256, 0, s>>>(lt_dev, t1_dev, nj, n, no);
    MLCC_CHECK_LAUNCH();
    k_na_trace<<<(nj + warps - 1) / warps, 32 * warps, 0, s>>>(chol_dev, nj, n, no, D);
    MLCC_CHECK_LAUNCH();
    k_na_trace<<<(nj + warps - 1) / warps, 32 * warps, 0, s>>>(lt_dev, nj, n, no, Dt);
    MLCC_CHECK_LAUNCH();
    // h = F - G(L) (Eq. eff_fock), dressed in place, then + G(Lt)
    MLCC_CUDA(cudaMemcpyAsync(ft_dev, fock_dev, size_t(nn) * 8, cudaMemcpyDeviceToDevice, s));
    k_na_two_electron<<<blocks_for(nn), 256, 0, s>>>(chol_dev, D, nj, n, no, -1.0, ft_dev);
    MLCC_CHECK_LAUNCH();
    k_na_left<<<blocks_for(nn), 256, 0, s>>>(ft_dev, t1_dev, 1, n, no, ft_dev);
    MLCC_CHECK_LAUNCH();
    k_na_right<<<blocks_for(int64_t(n) * no), 256, 0, s>>>(ft_dev, t1_dev, 1, n, no);
    MLCC_CHECK_LAUNCH();
    k_na_two_electron<<<blocks_for(nn), 256, 0, s>>>(lt_dev, Dt, nj, n, no, 1.0, ft_dev);
    MLCC_CHECK_LAUNCH();
    return MLCC_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MLCC_E_CUDA;
  }
}

// Davidson vector arithmetic of the split-precision phase in binary32.
//
// GB300 issues about two binary64 FMAs per SM and clock, less than HBM feeds these
// kernels as soon as a loaded element takes part in more than one product: the
// multi-vector dot products and the skinny subspace GEMMs of the Davidson solver were
// bound by the FP64 pipe, not by memory. In the low-precision phase (whose sigma-vectors
// carry relative errors near 1e-7) the same operations read the binary64 vectors, convert
// every element to binary32 with integer operations (truncation; magnitudes below the
// binary32 normal range become 0, NaN becomes Inf) and multiply-add in binary32. Per-thread
// partial sums are widened to binary64 for the cross-thread reduction and for the
// alpha / beta update of the output, so no binary64 arithmetic runs per element.
#include "internal.cuh"
#include "fp_convert.cuh"

#include <algorithm>

namespace mlcc {

namespace {

__device__ __forceinline__ float d2f(double x) { return d2f_bits(x); }
__device__ __forceinline__ float d2f(float x) { return x; }
__device__ __forceinline__ double f2d(float f) { return f2d_bits(f); }
// store of a binary32 result: widened exactly, or kept
__device__ __forceinline__ void st32(double* p, float v) { *p = f2d_bits(v); }
__device__ __forceinline__ void st32(float* p, float v) { *p = v; }
__device__ __forceinline__ double ld64(const double* p) { return *p; }
__device__ __forceinline__ void st64(double* p, double v) { *p = v; }
__device__ __forceinline__ void st64(float* p, double v) { *p = d2f_bits(v); }
__device__ __forceinline__ double ld64(const float* p) { return f2d_bits(*p); }

constexpr int DOT32_BLOCKS = 1216;   // 8 blocks of 256 threads per SM of a GB300
constexpr int DOT32_CHUNK = 16;   // x-vectors per pass over the y-vectors

// partial[k][blk]: the block's share of x_k . y, DOT32_CHUNK vectors x_k per pass over y.
// Four strided elements per iteration keep several loads in flight per thread (a single
// vector pair per thread is otherwise latency-bound).
template <typename TX, typename TY>
__global__ void k_dots32(const TX* x, int64_t ldx, int nx, const TY* y, int64_t n, double* partial) {
  __shared__ double red[DOT32_CHUNK][256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t st = int64_t(gridDim.x) * blockDim.x;
  for (int k0 = 0; k0 < nx; k0 += DOT32_CHUNK) {
    const int kc = min(DOT32_CHUNK, nx - k0);
    float acc[DOT32_CHUNK];
#pragma unroll
    for (int c = 0; c < DOT32_CHUNK; ++c) acc[c] = 0.0f;
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * st < n; i += 4 * st) {
      const float y0 = d2f(y[i]), y1 = d2f(y[i + st]), y2 = d2f(y[i + 2 * st]), y3 = d2f(y[i + 3 * st]);
#pragma unroll
      for (int c = 0; c < DOT32_CHUNK; ++c)
        if (c < kc) {
          const TX* xc = x + int64_t(k0 + c) * ldx;
          const float a0 = d2f(xc[i]), a1 = d2f(xc[i + st]), a2 = d2f(xc[i + 2 * st]), a3 = d2f(xc[i + 3 * st]);
          acc[c] = fmaf(a0, y0, fmaf(a1, y1, fmaf(a2, y2, fmaf(a3, y3, acc[c]))));
        }
    }
    for (; i < n; i += st) {
      const float yi = d2f(y[i]);
#pragma unroll
      for (int c = 0; c < DOT32_CHUNK; ++c)
        if (c < kc) acc[c] = fmaf(d2f(x[int64_t(k0 + c) * ldx + i]), yi, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < DOT32_CHUNK; ++c) {
      if (c >= kc) continue;   // kc is the same in every thread
      double v = f2d(acc[c]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kc) {
      double v = 0.0;
      for (int w = 0; w < int(blockDim.x / 32); ++w) v += red[threadIdx.x][w];
      partial[int64_t(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

// partial[(k * NY + j)][blk] for DOT32_CHUNK x-vectors per pass and NY <= 4 y-vectors
template <int NY, typename TX, typename TY, int CH = (NY >= 3 ? 8 : DOT32_CHUNK)>   // CH * NY accumulators
__global__ void k_dots_block32(const TX* x, int64_t ldx, int nx, const TY* y, int64_t ldy, int64_t n,
                               double* partial) {
  constexpr int DOT32_CHUNK = CH;
  __shared__ double red[DOT32_CHUNK * NY][256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < nx; k0 += DOT32_CHUNK) {
    const int kc = min(DOT32_CHUNK, nx - k0);
    float acc[DOT32_CHUNK][NY];
#pragma unroll
    for (int c = 0; c < DOT32_CHUNK; ++c)
#pragma unroll
      for (int j = 0; j < NY; ++j) acc[c][j] = 0.0f;
    const int64_t st = int64_t(gridDim.x) * blockDim.x;
    int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + st < n; i += 2 * st) {   // two strided elements per iteration
      float yv[NY], yw[NY];
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        yv[j] = d2f(y[int64_t(j) * ldy + i]);
        yw[j] = d2f(y[int64_t(j) * ldy + i + st]);
      }
#pragma unroll
      for (int c = 0; c < DOT32_CHUNK; ++c) {
        if (c < kc) {
          const float xv = d2f(x[int64_t(k0 + c) * ldx + i]), xw = d2f(x[int64_t(k0 + c) * ldx + i + st]);
#pragma unroll
          for (int j = 0; j < NY; ++j) acc[c][j] = fmaf(xv, yv[j], fmaf(xw, yw[j], acc[c][j]));
        }
      }
    }
    for (; i < n; i += st) {
      float yv[NY];
#pragma unroll
      for (int j = 0; j < NY; ++j) yv[j] = d2f(y[int64_t(j) * ldy + i]);
#pragma unroll
      for (int c = 0; c < DOT32_CHUNK; ++c) {
        if (c < kc) {
          const float xv = d2f(x[int64_t(k0 + c) * ldx + i]);
#pragma unroll
          for (int j = 0; j < NY; ++j) acc[c][j] = fmaf(xv, yv[j], acc[c][j]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DOT32_CHUNK; ++c)
      if (c < kc) {   // kc is the same in every thread
#pragma unroll
        for (int j = 0; j < NY; ++j) {
          double v = f2d(acc[c][j]);
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) red[c * NY + j][warp] = v;
        }
      }
    __syncthreads();
    if (threadIdx.x < kc * NY) {
      double v = 0.0;
      for (int w = 0; w < int(blockDim.x / 32); ++w) v += red[threadIdx.x][w];
      const int c = threadIdx.x / NY, j = threadIdx.x - c * NY;
      partial[int64_t((k0 + c) * NY + j) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

__global__ void k_dots32_stage2(const double* partial, int nblk, double* out) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partial[int64_t(k) * nblk + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}

// Binary32 storage with every vector 16-byte aligned and n a multiple of 4: the same block
// dot products with float4 loads (four elements per load instruction, CH + NY loads of 16 B
// in flight per thread), so that the pass runs at the memory's rate rather than the
// load-issue rate. partial[(k * NY + j)][blk] as in k_dots_block32.
template <int NY, int CH>
__global__ void k_dots_block32_v4(const float* __restrict__ x, int64_t ldx, int nx, const float* __restrict__ y,
                                  int64_t ldy, int64_t n4, double* partial) {
  __shared__ double red[CH * NY][256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t st = int64_t(gridDim.x) * blockDim.x;
  for (int k0 = 0; k0 < nx; k0 += CH) {
    const int kc = min(CH, nx - k0);
    float acc[CH][NY];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int j = 0; j < NY; ++j) acc[c][j] = 0.0f;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n4; i += st) {
      float4 yv[NY];
#pragma unroll
      for (int j = 0; j < NY; ++j) yv[j] = __ldg(reinterpret_cast<const float4*>(y + int64_t(j) * ldy) + i);
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (c < kc) {
          const float4 xv = __ldg(reinterpret_cast<const float4*>(x + int64_t(k0 + c) * ldx) + i);
#pragma unroll
          for (int j = 0; j < NY; ++j)
            acc[c][j] = fmaf(xv.x, yv[j].x, fmaf(xv.y, yv[j].y, fmaf(xv.z, yv[j].z, fmaf(xv.w, yv[j].w, acc[c][j]))));
        }
      }
    }
    // only the kc x NY accumulators in use (kc is the same in every thread)
#pragma unroll
    for (int c = 0; c < CH; ++c)
      if (c < kc) {
#pragma unroll
        for (int j = 0; j < NY; ++j) {
          double v = f2d(acc[c][j]);
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) red[c * NY + j][warp] = v;
        }
      }
    __syncthreads();
    if (threadIdx.x < kc * NY) {
      double v = 0.0;
      for (int w = 0; w < int(blockDim.x / 32); ++w) v += red[threadIdx.x][w];
      const int c = threadIdx.x / NY, j = threadIdx.x - c * NY;
      partial[int64_t((k0 + c) * NY + j) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

// the skinny binary32 GEMM with four columns per thread and float4 loads of B (ldb and N
// multiples of 4, B 16-byte aligned); op(A) (K <= 64) staged in shared memory
template <int MM, bool TA, typename TC>
__global__ void k_skinny32_v4(int64_t M, int64_t N4, int64_t K, const double* A, int64_t lda,
                              const float* __restrict__ B, int64_t ldb, TC* C, int64_t ldc, double alpha,
                              double beta) {
  __shared__ float As[MM * 64];
  for (int t = threadIdx.x; t < MM * 64; t += blockDim.x) {
    const int m = t / 64, k = t - m * 64;
    As[t] = (m < M && k < K) ? d2f(TA ? A[int64_t(k) * lda + m] : A[int64_t(m) * lda + k]) : 0.0f;
  }
  __syncthreads();
  const int64_t n4 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (n4 >= N4) return;
  float4 acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t k = 0; k < K; ++k) {
    const float4 b = __ldg(reinterpret_cast<const float4*>(B + k * ldb) + n4);
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      const float a = As[m * 64 + k];
      acc[m].x = fmaf(a, b.x, acc[m].x);
      acc[m].y = fmaf(a, b.y, acc[m].y);
      acc[m].z = fmaf(a, b.z, acc[m].z);
      acc[m].w = fmaf(a, b.w, acc[m].w);
    }
  }
#pragma unroll
  for (int m = 0; m < MM; ++m)
    if (m < M) {
      TC* cp = C + m * ldc + 4 * n4;
      const float r[4] = {acc[m].x, acc[m].y, acc[m].z, acc[m].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (sizeof(TC) == 8) {
          const double v = alpha * f2d(r[q]);
          st64(cp + q, (beta == 0.0) ? v : v + beta * ld64(cp + q));
        } else {
          const float a = float(alpha), bb = float(beta);
          st32(cp + q, (bb == 0.0f) ? a * r[q] : fmaf(a, r[q], bb * d2f(cp[q])));
        }
      }
    }
}

// C[m][n] = alpha sum_k op(A)[m][k] B[k][n] + beta C[m][n] for M <= MM, one thread per
// column n; op(A) (K <= 64) is staged in shared memory as binary32
template <int MM, bool TA, typename TB, typename TC>
__global__ void k_skinny32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const TB* B,
                           int64_t ldb, TC* C, int64_t ldc, double alpha, double beta) {
  __shared__ float As[MM * 64];
  for (int t = threadIdx.x; t < MM * 64; t += blockDim.x) {
    const int m = t / 64, k = t - m * 64;
    As[t] = (m < M && k < K) ? d2f(TA ? A[int64_t(k) * lda + m] : A[int64_t(m) * lda + k]) : 0.0f;
  }
  __syncthreads();
  const int64_t n = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (n >= N) return;
  float acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = 0.0f;
  int64_t k = 0;
  for (; k + 4 <= K; k += 4) {
    const float b0 = d2f(B[k * ldb + n]), b1 = d2f(B[(k + 1) * ldb + n]);
    const float b2 = d2f(B[(k + 2) * ldb + n]), b3 = d2f(B[(k + 3) * ldb + n]);
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      const float* a = As + m * 64 + k;
      acc[m] = fmaf(a[0], b0, fmaf(a[1], b1, fmaf(a[2], b2, fmaf(a[3], b3, acc[m]))));
    }
  }
  for (; k < K; ++k) {
    const float b = d2f(B[k * ldb + n]);
#pragma unroll
    for (int m = 0; m < MM; ++m) acc[m] = fmaf(As[m * 64 + k], b, acc[m]);
  }
#pragma unroll
  for (int m = 0; m < MM; ++m)
    if (m < M) {
      TC* cp = C + m * ldc + n;
      const float a = float(alpha), b = float(beta);
      if (sizeof(TC) == 8) {
        const double v = alpha * f2d(acc[m]);
        st64(cp, (beta == 0.0) ? v : v + beta * ld64(cp));
      } else {
        st32(cp, (b == 0.0f) ? a * acc[m] : fmaf(a, acc[m], b * d2f(*cp)));
      }
    }
}

template <int MM, typename TB, typename TC>
void launch_skinny32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta, const TB* B,
                     int64_t ldb, TC* C, int64_t ldc, double alpha, double beta, cudaStream_t s) {
  const unsigned blocks = unsigned((N + 255) / 256);
  if (ta) k_skinny32<MM, true, TB, TC><<<blocks, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  else k_skinny32<MM, false, TB, TC><<<blocks, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta);
  MLCC_CHECK_LAUNCH();
}
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <int MM, typename TC>
void launch_skinny32_v4(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta, const float* B,
                        int64_t ldb, TC* C, int64_t ldc, double alpha, double beta, cudaStream_t s) {
  const int64_t N4 = N / 4;
  const unsigned blocks = unsigned((N4 + 255) / 256);
  if (ta) k_skinny32_v4<MM, true, TC><<<blocks, 256, 0, s>>>(M, N4, K, A, lda, B, ldb, C, ldc, alpha, beta);
  else k_skinny32_v4<MM, false, TC><<<blocks, 256, 0, s>>>(M, N4, K, A, lda, B, ldb, C, ldc, alpha, beta);
  MLCC_CHECK_LAUNCH();
}

template <typename TB, typename TC>
bool skinny32_t(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta, const TB* B, int64_t ldb,
                TC* C, int64_t ldc, double alpha, double beta, cudaStream_t s) {
  if (M < 1 || M > 16 || K > 64 || K < 0 || N < 1) return false;
  MLCC_REQUIRE((N + 255) / 256 < (int64_t(1) << 31), "skinny32: N too large");
  if constexpr (sizeof(TB) == 4) {
    if (N % 4 == 0 && ldb % 4 == 0 && aligned16(B) && K > 0) {
      const float* Bf = reinterpret_cast<const float*>(B);
      if (M <= 1) launch_skinny32_v4<1>(M, N, K, A, lda, ta, Bf, ldb, C, ldc, alpha, beta, s);
      else if (M <= 4) launch_skinny32_v4<4>(M, N, K, A, lda, ta, Bf, ldb, C, ldc, alpha, beta, s);
      else if (M <= 8) launch_skinny32_v4<8>(M, N, K, A, lda, ta, Bf, ldb, C, ldc, alpha, beta, s);
      else launch_skinny32_v4<16>(M, N, K, A, lda, ta, Bf, ldb, C, ldc, alpha, beta, s);
      return true;
    }
  }
  if (M <= 1) launch_skinny32<1>(M, N, K, A, lda, ta, B, ldb, C, ldc, alpha, beta, s);
  else if (M <= 4) launch_skinny32<4>(M, N, K, A, lda, ta, B, ldb, C, ldc, alpha, beta, s);
  else if (M <= 8) launch_skinny32<8>(M, N, K, A, lda, ta, B, ldb, C, ldc, alpha, beta, s);
  else launch_skinny32<16>(M, N, K, A, lda, ta, B, ldb, C, ldc, alpha, beta, s);
  return true;
}

template <typename TX, typename TY>
void dots32_t(const TX* x, int64_t ldx, int nx, const TY* y, int64_t n, double* out_dev, Arena& ws,
              cudaStream_t s) {
  if (nx <= 0) return;
  Scope sc(ws);
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, DOT32_BLOCKS)));
  double* partial = ws.get<double>(size_t(nx) * blocks);
  bool v4 = false;
  if constexpr (sizeof(TX) == 4 && sizeof(TY) == 4)
    v4 = n % 4 == 0 && ldx % 4 == 0 && aligned16(x) && aligned16(y);
  if (v4) {
    if constexpr (sizeof(TX) == 4 && sizeof(TY) == 4)
      k_dots_block32_v4<1, DOT32_CHUNK><<<blocks, 256, 0, s>>>(reinterpret_cast<const float*>(x), ldx, nx,
                                                                reinterpret_cast<const float*>(y), 0, n / 4, partial);
  } else {
    k_dots32<TX, TY><<<blocks, 256, 0, s>>>(x, ldx, nx, y, n, partial);
  }
  MLCC_CHECK_LAUNCH();
  k_dots32_stage2<<<nx, 256, 0, s>>>(partial, blocks, out_dev);
  MLCC_CHECK_LAUNCH();
}

template <typename TX, typename TY>
void dots_block32_t(const TX* x, int64_t ldx, int nx, const TY* y, int64_t ldy, int ny, int64_t n,
                    double* out_dev, Arena& ws, cudaStream_t s) {
  if (nx <= 0 || ny <= 0) return;
  MLCC_REQUIRE(ny <= 4, "dots_block: at most 4 y-vectors");
  Scope sc(ws);
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, DOT32_BLOCKS)));
  double* partial = ws.get<double>(size_t(nx) * ny * blocks);
  bool v4 = false;
  if constexpr (sizeof(TX) == 4 && sizeof(TY) == 4)
    v4 = n % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && aligned16(x) && aligned16(y);
  if (v4) {
    if constexpr (sizeof(TX) == 4 && sizeof(TY) == 4) {
      const float* xf = reinterpret_cast<const float*>(x);
      const float* yf = reinterpret_cast<const float*>(y);
      switch (ny) {
        case 1: k_dots_block32_v4<1, 16><<<blocks, 256, 0, s>>>(xf, ldx, nx, yf, ldy, n / 4, partial); break;
        case 2: k_dots_block32_v4<2, 16><<<blocks, 256, 0, s>>>(xf, ldx, nx, yf, ldy, n / 4, partial); break;
        case 3: k_dots_block32_v4<3, 8><<<blocks, 256, 0, s>>>(xf, ldx, nx, yf, ldy, n / 4, partial); break;
        default: k_dots_block32_v4<4, 8><<<blocks, 256, 0, s>>>(xf, ldx, nx, yf, ldy, n / 4, partial); break;
      }
    }
  } else {
    switch (ny) {
      case 1: k_dots_block32<1, TX, TY><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
      case 2: k_dots_block32<2, TX, TY><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
      case 3: k_dots_block32<3, TX, TY><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
      default: k_dots_block32<4, TX, TY><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
    }
  }
  MLCC_CHECK_LAUNCH();
  k_dots32_stage2<<<nx * ny, 256, 0, s>>>(partial, blocks, out_dev);
  MLCC_CHECK_LAUNCH();
}

__global__ void k_cvt_d2f(const double* x, float* y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = d2f_bits(x[i]);
}
__global__ void k_cvt_f2d(const float* x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = f2d_bits(x[i]);
}
__global__ void k_scale_f(float* x, int64_t n, float a) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= a;
}
int stream_blocks(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 65535))); }

}  // namespace

void dots32(const double* x, int64_t ldx, int nx, const double* y, int64_t n, double* out_dev, Arena& ws,
            cudaStream_t s) {
  dots32_t(x, ldx, nx, y, n, out_dev, ws, s);
}
void dots_block32(const double* x, int64_t ldx, int nx, const double* y, int64_t ldy, int ny, int64_t n,
                  double* out_dev, Arena& ws, cudaStream_t s) {
  dots_block32_t(x, ldx, nx, y, ldy, ny, n, out_dev, ws, s);
}
bool skinny32(const Gemm& g, cudaStream_t s) {
  if (g.tb || g.reduce || g.batch != 1) return false;
  return skinny32_t(g.M, g.N, g.K, g.A, g.lda, g.ta, g.B, g.ldb, g.C, g.ldc, g.alpha, g.beta, s);
}

// binary32 vector storage (the Davidson basis of a split-precision phase)
void dots_f32(const float* x, int64_t ldx, int nx, const float* y, int64_t n, double* out_dev, Arena& ws,
              cudaStream_t s) {
  dots32_t(x, ldx, nx, y, n, out_dev, ws, s);
}
void dots_block_f32(const float* x, int64_t ldx, int nx, const float* y, int64_t ldy, int ny, int64_t n,
                    double* out_dev, Arena& ws, cudaStream_t s) {
  dots_block32_t(x, ldx, nx, y, ldy, ny, n, out_dev, ws, s);
}
void combine_f32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta, const float* B,
                 int64_t ldb, void* C, bool c_f32, int64_t ldc, double alpha, double beta, cudaStream_t s) {
  const bool ok = c_f32 ? skinny32_t(M, N, K, A, lda, ta, B, ldb, static_cast<float*>(C), ldc, alpha, beta, s)
                        : skinny32_t(M, N, K, A, lda, ta, B, ldb, static_cast<double*>(C), ldc, alpha, beta, s);
  MLCC_REQUIRE(ok, "combine_f32: at most 16 outputs of at most 64 vectors");
}
void cvt_d2f(const double* x, float* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_cvt_d2f<<<stream_blocks(n), 256, 0, s>>>(x, y, n);
  MLCC_CHECK_LAUNCH();
}
void cvt_f2d(const float* x, double* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_cvt_f2d<<<stream_blocks(n), 256, 0, s>>>(x, y, n);
  MLCC_CHECK_LAUNCH();
}
void scale_f32(float* x, int64_t n, double a, cudaStream_t s) {
  if (n <= 0) return;
  k_scale_f<<<stream_blocks(n), 256, 0, s>>>(x, n, float(a));
  MLCC_CHECK_LAUNCH();
}

}  // namespace mlcc

// Binary64 building blocks of libmlcc: device arena, kernel timers, a tiled DGEMM on the
// CUDA cores (batched and batch-reduced), strided permutations, a pairwise einsum engine
// built from those two, and deterministic reductions. gemm_f64 is the one entry of every
// contraction: under a LowpScope its large products go to the tensor cores (split
// bfloat16, or the binary64 emulation), under a Vec32Scope its skinny products and the dot
// products multiply in binary32 (vec32.cu).
#include "internal.cuh"
#include "tc_common.cuh"

#include <algorithm>
#include <cstring>
#include <atomic>
#include <thread>

namespace mlcc {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }
void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------------
Arena::~Arena() {
  if (base_) cudaFree(base_);
}
void Arena::reserve(size_t bytes) {
  if (base_) cudaFree(base_);
  base_ = nullptr;
  cap_ = top_ = hw_ = 0;
  if (bytes == 0) return;
  MLCC_CUDA(cudaMalloc(&base_, bytes));
  cap_ = bytes;
}
void* Arena::alloc(size_t bytes) {
  size_t off = (top_ + 255) & ~size_t(255);
  size_t need = off + ((bytes + 255) & ~size_t(255));
  if (need > cap_)
    throw Error(MLCC_E_OOM, "workspace arena exhausted: need " + std::to_string(need) +
                                " of " + std::to_string(cap_) + " bytes");
  top_ = need;
  hw_ = std::max(hw_, top_);
  return base_ + off;
}

// ---------------------------------------------------------------------------------
cudaEvent_t KernelTimer::get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  MLCC_CUDA(cudaEventCreate(&e));
  return e;
}
void KernelTimer::begin(const char* fam, cudaStream_t s, double flop, cudaEvent_t* a,
                        cudaEvent_t* b) {
  *a = get_event();
  *b = get_event();
  MLCC_CUDA(cudaEventRecord(*a, s));
  recs[fam].push_back({*a, *b, flop});
}
void KernelTimer::reset() {
  for (auto& kv : recs)
    for (auto& r : kv.second) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
  recs.clear();
}
KernelTimer::~KernelTimer() {
  reset();
  for (auto e : pool) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------------
// DGEMM: 64 x 64 output tile per CTA, 256 threads, each thread a 4 x 4 register block,
// K stepped by 16 through double-buffered shared memory.
namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct GP {
  int64_t M, N, K;
  const double* A; int64_t lda, sA;
  const double* B; int64_t ldb, sB;
  double* C; int64_t ldc, sC;
  double alpha, beta;
  int64_t batch;
  int reduce;       // 1: sum over batches inside the CTA's share
  double* partial;  // reduce with several splits: [split][M][N]
  int64_t kchunk;   // > 0: split K, CTA z takes [z * kchunk, (z + 1) * kchunk)
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) k_dgemm(GP p) {
  __shared__ double As[2][BK][BM];
  __shared__ double Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  int64_t b_begin, b_end, b_step;
  int64_t kb0 = 0, kb1 = p.K;
  if (p.reduce) {
    b_begin = blockIdx.z;
    b_end = p.batch;
    b_step = gridDim.z;
  } else if (p.kchunk > 0) {
    b_begin = 0;
    b_end = 1;
    b_step = 1;
    kb0 = int64_t(blockIdx.z) * p.kchunk;
    kb1 = min(p.K, kb0 + p.kchunk);
  } else {
    b_begin = blockIdx.z;
    b_end = blockIdx.z + 1;
    b_step = 1;
  }
  const int64_t nk = (kb1 - kb0 + BK - 1) / BK;
  for (int64_t b = b_begin; b < b_end; b += b_step) {
    const double* A = p.A + b * p.sA;
    const double* B = p.B + b * p.sB;
    double ra[4], rb[4];
    auto load = [&](int64_t kt) {
      const int64_t k0 = kb0 + kt * BK;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = tid + NT * r;
        int mm, kk;
        if (!TA) { mm = e >> 4; kk = e & 15; } else { kk = e >> 6; mm = e & 63; }
        const int64_t gm = m0 + mm, gk = k0 + kk;
        ra[r] = (gm < p.M && gk < kb1) ? (TA ? A[gk * p.lda + gm] : A[gm * p.lda + gk]) : 0.0;
        int nn, kb;
        if (!TB) { kb = e >> 6; nn = e & 63; } else { nn = e >> 4; kb = e & 15; }
        const int64_t gn = n0 + nn, gkb = k0 + kb;
        rb[r] = (gn < p.N && gkb < kb1) ? (TB ? B[gn * p.ldb + gkb] : B[gkb * p.ldb + gn]) : 0.0;
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = tid + NT * r;
        int mm, kk;
        if (!TA) { mm = e >> 4; kk = e & 15; } else { kk = e >> 6; mm = e & 63; }
        As[buf][kk][mm] = ra[r];
        int nn, kb;
        if (!TB) { kb = e >> 6; nn = e & 63; } else { nn = e >> 4; kb = e & 15; }
        Bs[buf][kb][nn] = rb[r];
      }
    };
    load(0);
    store(0);
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) load(kt + 1);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        double a[4], bb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[buf][k][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[buf][k][tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], bb[c], acc[r][c]);
      }
      if (kt + 1 < nk) store(buf ^ 1);
      __syncthreads();
    }
  }
  if ((p.reduce || p.kchunk > 0) && gridDim.z > 1) {
    double* P = p.partial + int64_t(blockIdx.z) * p.M * p.N;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t gm = m0 + ty * 4 + r;
      if (gm >= p.M) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gn = n0 + tx * 4 + c;
        if (gn < p.N) P[gm * p.N + gn] = acc[r][c];
      }
    }
    return;
  }
  double* C = p.C + ((p.reduce || p.kchunk > 0) ? 0 : int64_t(blockIdx.z) * p.sC);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t gm = m0 + ty * 4 + r;
    if (gm >= p.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t gn = n0 + tx * 4 + c;
      if (gn >= p.N) continue;
      double* cp = C + gm * p.ldc + gn;
      const double v = p.alpha * acc[r][c];
      *cp = (p.beta == 0.0) ? v : v + p.beta * (*cp);
    }
  }
}

// C = alpha * sum_s partial[s] + beta * C, summed in split order (deterministic).
__global__ void k_reduce_partials(const double* partial, int nsplit, int64_t M, int64_t N,
                                  double* C, int64_t ldc, double alpha, double beta) {
  const int64_t total = M * N;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += partial[int64_t(k) * total + i];
    const int64_t m = i / N, n = i - m * N;
    double* cp = C + m * ldc + n;
    *cp = (beta == 0.0) ? alpha * s : alpha * s + beta * (*cp);
  }
}
// Skinny shapes are bandwidth-bound: a 64 x 64 tile would waste up to 63/64 of its work.
// M <= 16: one thread (or warp, for a transposed B) per output column n.
template <int MM, bool TA, bool TB>
__global__ void k_skinny_m(GP p) {
  if (!TB) {
    // the small operand A (M x K, K <= 64 here) is staged in shared memory once per block
    __shared__ double As[MM * 64];
    const bool staged = p.K <= 64;
    if (staged) {
      for (int t = threadIdx.x; t < MM * 64; t += blockDim.x) {
        const int m = t / 64, k = t - m * 64;
        As[t] = (m < p.M && k < p.K) ? (TA ? p.A[int64_t(k) * p.lda + m] : p.A[int64_t(m) * p.lda + k]) : 0.0;
      }
      __syncthreads();
    }
    const int64_t n = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (n >= p.N) return;
    double acc[MM];
#pragma unroll
    for (int m = 0; m < MM; ++m) acc[m] = 0.0;
    if (staged) {
      int64_t k = 0;
      for (; k + 4 <= p.K; k += 4) {
        const double b0 = p.B[k * p.ldb + n], b1 = p.B[(k + 1) * p.ldb + n];
        const double b2 = p.B[(k + 2) * p.ldb + n], b3 = p.B[(k + 3) * p.ldb + n];
#pragma unroll
        for (int m = 0; m < MM; ++m) {
          const double* a = As + m * 64 + k;
          acc[m] = fma(a[0], b0, fma(a[1], b1, fma(a[2], b2, fma(a[3], b3, acc[m]))));
        }
      }
      for (; k < p.K; ++k) {
        const double b = p.B[k * p.ldb + n];
#pragma unroll
        for (int m = 0; m < MM; ++m) acc[m] = fma(As[m * 64 + k], b, acc[m]);
      }
    } else {
      // K split over blockIdx.y when p.kchunk > 0 (partials reduced afterwards)
      const int64_t k0 = p.kchunk > 0 ? int64_t(blockIdx.y) * p.kchunk : 0;
      const int64_t k1 = p.kchunk > 0 ? min(p.K, k0 + p.kchunk) : p.K;
      for (int64_t k = k0; k < k1; ++k) {
        const double b = p.B[k * p.ldb + n];
#pragma unroll
        for (int m = 0; m < MM; ++m)
          if (m < p.M) acc[m] = fma(TA ? p.A[k * p.lda + m] : p.A[m * p.lda + k], b, acc[m]);
      }
    }
    if (p.partial) {
      double* part = p.partial + int64_t(blockIdx.y) * p.M * p.N;
#pragma unroll
      for (int m = 0; m < MM; ++m)
        if (m < p.M) part[m * p.N + n] = acc[m];
      return;
    }
#pragma unroll
    for (int m = 0; m < MM; ++m)
      if (m < p.M) {
        double* cp = p.C + m * p.ldc + n;
        const double v = p.alpha * acc[m];
        *cp = (p.beta == 0.0) ? v : v + p.beta * (*cp);
      }
  } else {
    const int64_t n = blockIdx.x * int64_t(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (n >= p.N) return;
    double acc[MM];
#pragma unroll
    for (int m = 0; m < MM; ++m) acc[m] = 0.0;
    for (int64_t k = lane; k < p.K; k += 32) {
      const double b = p.B[n * p.ldb + k];
#pragma unroll
      for (int m = 0; m < MM; ++m)
        if (m < p.M) acc[m] = fma(TA ? p.A[k * p.lda + m] : p.A[m * p.lda + k], b, acc[m]);
    }
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      double v = acc[m];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && m < p.M) {
        double* cp = p.C + m * p.ldc + n;
        const double w = p.alpha * v;
        *cp = (p.beta == 0.0) ? w : w + p.beta * (*cp);
      }
    }
  }
}
// N == 1: y[m] = sum_k op(A)[m][k] x[k]; a warp per row (A row-major) or a thread per row.
template <bool TA>
__global__ void k_gemv_n1(GP p) {
  if (!TA) {
    const int64_t m = blockIdx.x * int64_t(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (m >= p.M) return;
    double acc = 0.0;
    for (int64_t k = lane; k < p.K; k += 32) acc = fma(p.A[m * p.lda + k], p.B[k * p.ldb], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      double* cp = p.C + m * p.ldc;
      const double v = p.alpha * acc;
      *cp = (p.beta == 0.0) ? v : v + p.beta * (*cp);
    }
  } else {
    const int64_t m = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (m >= p.M) return;
    double acc = 0.0;
    for (int64_t k = 0; k < p.K; ++k) acc = fma(p.A[k * p.lda + m], p.B[k * p.ldb], acc);
    double* cp = p.C + m * p.ldc;
    const double v = p.alpha * acc;
    *cp = (p.beta == 0.0) ? v : v + p.beta * (*cp);
  }
}
template <int MM>
static void launch_skinny(const GP& p, bool ta, bool tb, cudaStream_t s, int ksplit = 1) {
  if (!tb) {
    const dim3 blocks{unsigned((p.N + 255) / 256), unsigned(ksplit), 1};
    if (ta) k_skinny_m<MM, true, false><<<blocks, 256, 0, s>>>(p);
    else k_skinny_m<MM, false, false><<<blocks, 256, 0, s>>>(p);
  } else {
    const unsigned blocks = unsigned((p.N + 7) / 8);
    if (ta) k_skinny_m<MM, true, true><<<blocks, 256, 0, s>>>(p);
    else k_skinny_m<MM, false, true><<<blocks, 256, 0, s>>>(p);
  }
}
}  // namespace

static thread_local bool g_vec32 = false;
Vec32Scope::Vec32Scope(bool on) : prev(g_vec32) { g_vec32 = on; }
Vec32Scope::~Vec32Scope() { g_vec32 = prev; }
void Vec32Scope::set(bool on) { g_vec32 = on; }
bool vec32_active() { return g_vec32; }

static thread_local int g_lowp = 0;
static thread_local int* g_lowp_err = nullptr;
static thread_local OperandCache* g_lowp_cache = nullptr;
LowpScope::LowpScope(int precision, int* err_flag, OperandCache* cache)
    : prev(g_lowp), err(err_flag), prev_err(g_lowp_err), prev_cache(g_lowp_cache) {
  g_lowp = precision;
  g_lowp_err = err_flag;
  g_lowp_cache = cache;
}
LowpScope::~LowpScope() {
  g_lowp = prev;
  g_lowp_err = prev_err;
  g_lowp_cache = prev_cache;
}
int lowp_precision() { return g_lowp; }
int* lowp_error_flag() { return g_lowp_err; }
OperandCache* lowp_cache() { return g_lowp_cache; }

void reduce_partials(const double* partial, int nsplit, int64_t M, int64_t N, double* C,
                     int64_t ldc, double alpha, double beta, cudaStream_t s) {
  const int64_t total = M * N;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096)));
  k_reduce_partials<<<blocks, 256, 0, s>>>(partial, nsplit, M, N, C, ldc, alpha, beta);
  MLCC_CHECK_LAUNCH();
}

void gemm_f64(const Gemm& g, Arena& ws, cudaStream_t s, int sm_count) {
  if (g.M <= 0 || g.N <= 0) return;
  // large products go to the tensor cores; GEMV-like shapes (a side below 16) are bound
  // by reading their large operand once, which the binary64 kernels do without converting it
  if (g_lowp != 0 && g.K > 0 && g.batch > 0 && g.M >= 16 && g.N >= 16) {
    const double flop = 2.0 * double(g.M) * double(g.N) * double(g.K) * double(g.batch);
    if (flop >= 2e8 && gemm_tc(g, g_lowp, ws, s, sm_count, g_lowp_err)) return;
  }
  if (g.K <= 0 || g.batch <= 0) {
    // empty contraction: C = beta * C for each output matrix
    const int64_t nb = g.reduce ? 1 : std::max<int64_t>(g.batch, 1);
    for (int64_t b = 0; b < nb; ++b) {
      int64_t dims[2] = {g.M, g.N};
      int64_t st[2] = {g.ldc, 1};
      permute_f64(2, dims, g.C + b * g.sC, st, g.C + b * g.sC, st, 0.0, g.beta, s);
    }
    return;
  }
  GP p;
  p.M = g.M; p.N = g.N; p.K = g.K;
  p.A = g.A; p.lda = g.lda; p.sA = g.sA;
  p.B = g.B; p.ldb = g.ldb; p.sB = g.sB;
  p.C = g.C; p.ldc = g.ldc; p.sC = g.sC;
  p.alpha = g.alpha; p.beta = g.beta;
  p.batch = g.batch;
  p.reduce = g.reduce ? 1 : 0;
  p.partial = nullptr;
  p.kchunk = 0;
  if (!g.reduce && g.batch == 1 && g.M <= 16 && g.N >= 64) {
    if (g_vec32 && skinny32(g, s)) return;
    // few column blocks and a long K (beyond what is staged): split K over blockIdx.y
    int64_t ks = 1;
    size_t mk = ws.mark();
    const int64_t nblocks = (g.N + 255) / 256;
    if (!g.tb && g.K > 64 && nblocks < 2LL * std::max(sm_count, 1)) {
      ks = std::min<int64_t>({(4LL * std::max(sm_count, 1) + nblocks - 1) / nblocks, g.K / 64, 1024});
      while (ks > 1 && ks * g.M * g.N * 8 > (int64_t(1) << 30)) ks /= 2;
      if (ks > 1) {
        p.kchunk = (g.K + ks - 1) / ks;
        ks = (g.K + p.kchunk - 1) / p.kchunk;
        p.partial = ws.get<double>(size_t(ks) * g.M * g.N);
      } else {
        ks = 1;
      }
    }
    if (g.M <= 1) launch_skinny<1>(p, g.ta, g.tb, s, int(ks));
    else if (g.M <= 4) launch_skinny<4>(p, g.ta, g.tb, s, int(ks));
    else if (g.M <= 8) launch_skinny<8>(p, g.ta, g.tb, s, int(ks));
    else launch_skinny<16>(p, g.ta, g.tb, s, int(ks));
    MLCC_CHECK_LAUNCH();
    if (ks > 1) {
      const int64_t total = g.M * g.N;
      const int blocks = int(std::min<int64_t>((total + 255) / 256, 4096));
      k_reduce_partials<<<blocks, 256, 0, s>>>(p.partial, int(ks), g.M, g.N, g.C, g.ldc, g.alpha, g.beta);
      MLCC_CHECK_LAUNCH();
    }
    ws.release(mk);
    return;
  }
  if (!g.reduce && g.batch == 1 && g.N == 1 && g.M >= 64) {
    if (!g.ta) k_gemv_n1<false><<<unsigned((g.M + 7) / 8), 256, 0, s>>>(p);
    else k_gemv_n1<true><<<unsigned((g.M + 255) / 256), 256, 0, s>>>(p);
    MLCC_CHECK_LAUNCH();
    return;
  }
  const int64_t tm = (g.M + BM - 1) / BM, tn = (g.N + BN - 1) / BN;
  MLCC_REQUIRE(tm < 65536, "gemm_f64: M too large for the grid");
  int64_t gz = 1;
  size_t mk = ws.mark();
  if (g.reduce) {
    const int64_t tiles = tm * tn;
    const int64_t want = (4LL * std::max(sm_count, 1) + tiles - 1) / tiles;
    gz = std::max<int64_t>(1, std::min<int64_t>({g.batch, want, 4096}));
    // cap the partial buffer at 1 GiB
    while (gz > 1 && gz * g.M * g.N * 8 > (int64_t(1) << 30)) gz /= 2;
    if (gz > 1) p.partial = ws.get<double>(size_t(gz) * g.M * g.N);
  } else if (g.batch == 1 && tm * tn < 2LL * std::max(sm_count, 1) && g.K >= 64) {
    // too few output tiles to fill the GPU: split K over CTAs, reduce the partials (one SM
    // takes about 0.5 ms for a 64 x 64 x 500 binary64 tile, so even short K is split)
    const int64_t tiles = tm * tn;
    const int64_t want = (4LL * std::max(sm_count, 1) + tiles - 1) / tiles;
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(want, g.K / 32));
    while (splits > 1 && splits * g.M * g.N * 8 > (int64_t(1) << 30)) splits /= 2;
    if (splits > 1) {
      p.kchunk = ((g.K + splits - 1) / splits + BK - 1) / BK * BK;
      splits = (g.K + p.kchunk - 1) / p.kchunk;
      p.partial = ws.get<double>(size_t(splits) * g.M * g.N);
    }
    gz = splits;
  } else {
    gz = g.batch;
    MLCC_REQUIRE(gz < 65536, "gemm_f64: batch too large for the grid");
  }
  dim3 grid{unsigned(tn), unsigned(tm), unsigned(gz)};
  if (!g.ta && !g.tb) k_dgemm<false, false><<<grid, NT, 0, s>>>(p);
  else if (g.ta && !g.tb) k_dgemm<true, false><<<grid, NT, 0, s>>>(p);
  else if (!g.ta && g.tb) k_dgemm<false, true><<<grid, NT, 0, s>>>(p);
  else k_dgemm<true, true><<<grid, NT, 0, s>>>(p);
  MLCC_CHECK_LAUNCH();
  if ((g.reduce || p.kchunk > 0) && gz > 1) {
    const int64_t total = g.M * g.N;
    const int blocks = int(std::min<int64_t>((total + 255) / 256, 4096));
    k_reduce_partials<<<blocks, 256, 0, s>>>(p.partial, int(gz), g.M, g.N, g.C, g.ldc,
                                              g.alpha, g.beta);
    MLCC_CHECK_LAUNCH();
  }
  ws.release(mk);
}

// ---------------------------------------------------------------------------------
namespace {
constexpr int MAXD = 8;
struct PP {
  int nd;
  int64_t dims[MAXD];
  int64_t ss[MAXD];
  int64_t ds[MAXD];
  int64_t total;
  double alpha, beta;
  const double* src;
  double* dst;
};
// I: the index type. 32-bit unsigned when every element index and offset fits: the digit
// decomposition of the element index then costs 32-bit divisions instead of 64-bit ones,
// which otherwise bound the kernel rather than its memory traffic.
template <typename I>
__global__ void k_permute(PP p) {
  const I total = I(p.total), st = I(gridDim.x) * I(blockDim.x);
  I dims[MAXD], ss[MAXD], ds[MAXD];
  for (int d = 0; d < p.nd; ++d) {
    dims[d] = I(p.dims[d]);
    ss[d] = I(p.ss[d]);
    ds[d] = I(p.ds[d]);
  }
  for (I i = I(blockIdx.x) * I(blockDim.x) + I(threadIdx.x); i < total; i += st) {
    I rem = i, so = 0, dof = 0;
    for (int d = p.nd - 1; d >= 0; --d) {
      const I q = rem / dims[d];
      const I x = rem - q * dims[d];
      rem = q;
      so += x * ss[d];
      dof += x * ds[d];
    }
    const double v = (p.alpha == 0.0) ? 0.0 : p.alpha * p.src[so];
    p.dst[dof] = (p.beta == 0.0) ? v : v + p.beta * p.dst[dof];
  }
}
// Element index below 2^31 and offsets below 2^32: the index digits come from division by
// invariant integers (Granlund and Montgomery, 1994: q = (umulhi(m, n) + n) >> l with
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, exact for n < 2^31), and a plain copy
// (alpha 1, beta 0) does no binary64 arithmetic.
struct PPF {
  int nd;
  uint32_t dims[MAXD], magic[MAXD], shift[MAXD], ss[MAXD], ds[MAXD];
  uint32_t total;
  double alpha, beta;
  const double* src;
  double* dst;
};
template <bool COPY>
__global__ void k_permute_fast(PPF p) {
  const uint32_t st = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p.total; i += st) {
    uint32_t rem = i, so = 0, dof = 0;
    for (int d = p.nd - 1; d >= 0; --d) {
      const uint32_t q = (__umulhi(p.magic[d], rem) + rem) >> p.shift[d];
      const uint32_t x = rem - q * p.dims[d];
      rem = q;
      so += x * p.ss[d];
      dof += x * p.ds[d];
    }
    if (COPY) {
      p.dst[dof] = p.src[so];
    } else {
      const double v = (p.alpha == 0.0) ? 0.0 : p.alpha * p.src[so];
      p.dst[dof] = (p.beta == 0.0) ? v : v + p.beta * p.dst[dof];
    }
  }
}
}  // namespace

void permute_f64(int nd, const int64_t* dims, const double* src, const int64_t* src_strides,
                 double* dst, const int64_t* dst_strides, double alpha, double beta,
                 cudaStream_t s) {
  MLCC_REQUIRE(nd >= 0 && nd <= MAXD, "permute_f64: too many dimensions");
  PP p;
  p.nd = nd;
  p.total = 1;
  for (int d = 0; d < nd; ++d) {
    p.dims[d] = dims[d];
    p.ss[d] = src_strides[d];
    p.ds[d] = dst_strides[d];
    p.total *= dims[d];
  }
  if (p.total == 0) return;
  p.alpha = alpha;
  p.beta = beta;
  p.src = src;
  p.dst = dst;
  const int blocks = int(std::min<int64_t>((p.total + 255) / 256, 8192));
  // 32-bit indices when the element count and the largest source and destination offsets
  // (plus one grid stride) stay below 2^32
  int64_t smax = 0, dmax = 0;
  for (int d = 0; d < nd; ++d) {
    smax += (dims[d] - 1) * std::abs(src_strides[d]);
    dmax += (dims[d] - 1) * std::abs(dst_strides[d]);
  }
  bool small = p.total + int64_t(blocks) * 256 < (int64_t(1) << 32) && smax < (int64_t(1) << 32) &&
               dmax < (int64_t(1) << 32);
  for (int d = 0; d < nd; ++d) small = small && src_strides[d] >= 0 && dst_strides[d] >= 0;
  if (small && p.total + int64_t(blocks) * 256 < (int64_t(1) << 31)) {
    PPF f;
    f.nd = nd;
    for (int d = 0; d < nd; ++d) {
      const uint64_t dv = uint64_t(dims[d]);
      uint32_t l = 0;
      while ((uint64_t(1) << l) < dv) ++l;
      f.dims[d] = uint32_t(dv);
      f.magic[d] = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - dv)) / dv + 1);
      f.shift[d] = l;
      f.ss[d] = uint32_t(src_strides[d]);
      f.ds[d] = uint32_t(dst_strides[d]);
    }
    f.total = uint32_t(p.total);
    f.alpha = alpha;
    f.beta = beta;
    f.src = src;
    f.dst = dst;
    if (alpha == 1.0 && beta == 0.0) k_permute_fast<true><<<blocks, 256, 0, s>>>(f);
    else k_permute_fast<false><<<blocks, 256, 0, s>>>(f);
  } else if (small) k_permute<uint32_t><<<blocks, 256, 0, s>>>(p);
  else k_permute<int64_t><<<blocks, 256, 0, s>>>(p);
  MLCC_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------------
// einsum engine
namespace {
struct Spec {
  std::string a, b, c;
};
Spec parse(const char* spec) {
  std::string s(spec);
  const size_t comma = s.find(','), arrow = s.find("->");
  Spec r;
  if (comma == std::string::npos) {
    MLCC_REQUIRE(arrow != std::string::npos, std::string("bad einsum spec ") + spec);
    r.a = s.substr(0, arrow);
    r.c = s.substr(arrow + 2);
    return r;
  }
  MLCC_REQUIRE(arrow != std::string::npos && comma < arrow, std::string("bad einsum spec ") + spec);
  r.a = s.substr(0, comma);
  r.b = s.substr(comma + 1, arrow - comma - 1);
  r.c = s.substr(arrow + 2);
  return r;
}
std::vector<int64_t> strides_of(const std::vector<int64_t>& d) {
  std::vector<int64_t> st(d.size());
  int64_t acc = 1;
  for (int i = int(d.size()) - 1; i >= 0; --i) {
    st[i] = acc;
    acc *= d[i];
  }
  return st;
}
bool has(const std::string& s, char c) { return s.find(c) != std::string::npos; }
}  // namespace

void eperm(const char* spec, double alpha, const DT& A, double beta, const DT& C, cudaStream_t s) {
  Spec sp = parse(spec);
  MLCC_REQUIRE(sp.a.size() == A.d.size() && sp.c.size() == C.d.size() && sp.a.size() == sp.c.size(),
               std::string("eperm rank mismatch: ") + spec);
  auto sa = strides_of(A.d), sc = strides_of(C.d);
  std::vector<int64_t> dims(sp.c.size()), ss(sp.c.size()), ds(sp.c.size());
  for (size_t i = 0; i < sp.c.size(); ++i) {
    const size_t j = sp.a.find(sp.c[i]);
    MLCC_REQUIRE(j != std::string::npos, std::string("eperm index missing: ") + spec);
    MLCC_REQUIRE(A.d[j] == C.d[i], std::string("eperm size mismatch: ") + spec);
    dims[i] = C.d[i];
    ss[i] = sa[j];
    ds[i] = sc[i];
  }
  permute_f64(int(dims.size()), dims.data(), A.p, ss.data(), C.p, ds.data(), alpha, beta, s);
}

void einsum(const char* spec, double alpha, const DT& A, const DT& B, double beta, const DT& C,
            Arena& ws, cudaStream_t s, int sm_count) {
  Spec sp = parse(spec);
  MLCC_REQUIRE(sp.a.size() == A.d.size() && sp.b.size() == B.d.size() && sp.c.size() == C.d.size(),
               std::string("einsum rank mismatch: ") + spec);
  std::map<char, int64_t> size;
  auto reg = [&](const std::string& str, const std::vector<int64_t>& d) {
    for (size_t i = 0; i < str.size(); ++i) {
      auto it = size.find(str[i]);
      if (it == size.end()) size[str[i]] = d[i];
      else MLCC_REQUIRE(it->second == d[i], std::string("einsum size mismatch: ") + spec);
    }
  };
  reg(sp.a, A.d);
  reg(sp.b, B.d);
  reg(sp.c, C.d);
  std::string bat, mi, ni, ka, kb;
  for (char ch : sp.c) {
    const bool ia = has(sp.a, ch), ib = has(sp.b, ch);
    MLCC_REQUIRE(ia || ib, std::string("einsum output index not in inputs: ") + spec);
    if (ia && ib) bat += ch;
    else if (ia) mi += ch;
    else ni += ch;
  }
  for (char ch : sp.a) {
    if (!has(sp.c, ch)) {
      MLCC_REQUIRE(has(sp.b, ch), std::string("einsum index summed in one operand only: ") + spec);
      ka += ch;
    }
  }
  for (char ch : sp.b) {
    if (!has(sp.c, ch)) {
      MLCC_REQUIRE(has(sp.a, ch), std::string("einsum index summed in one operand only: ") + spec);
      kb += ch;
    }
  }
  auto prod = [&](const std::string& str) {
    int64_t p = 1;
    for (char ch : str) p *= size[ch];
    return p;
  };
  const int64_t nb = prod(bat), M = prod(mi), N = prod(ni), K = prod(ka);
  // choose the K order (that of A or of B) that needs fewer operand permutations
  auto cost = [&](const std::string& korder) {
    int c = 0;
    if (!(sp.a == bat + mi + korder || sp.a == bat + korder + mi)) c += 1;
    if (!(sp.b == bat + korder + ni || sp.b == bat + ni + korder)) c += 1;
    return c;
  };
  std::string kord = cost(ka) <= cost(kb) ? ka : kb;
  Scope scope(ws);
  // An operand inside the constant ranges of the current operand cache (the Jacobian's
  // value tensors while sigma runs) keeps its GEMM-order copy in that cache, so the GEMM
  // can keep its converted pieces too. Nothing is allocated while the stream captures a
  // graph: the eager evaluation before the capture has filled the cache.
  OperandCache* oc = lowp_cache();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (oc) MLCC_CUDA(cudaStreamIsCapturing(s, &cap));
  auto operand = [&](const DT& X, const std::string& from, const std::string& to, bool& cst) -> const double* {
    cst = oc && oc->constant(X.p);
    const std::string sps = from + "->" + to;
    DT t;
    for (char ch : to) t.d.push_back(size[ch]);
    const size_t count = size_t(t.size());
    if (cst) {
      for (auto& e : oc->perms)
        if (e.src == X.p && e.dims == X.d && e.spec == sps) return e.p;
      void* mem = nullptr;
      if (cap == cudaStreamCaptureStatusNone && cudaMalloc(&mem, count * 8) == cudaSuccess) {
        oc->blocks.push_back(mem);
        t.p = static_cast<double*>(mem);
        eperm(sps.c_str(), 1.0, X, 0.0, t, s);
        oc->perms.push_back({X.p, X.d, sps, t.p});
        return t.p;
      }
      if (cap == cudaStreamCaptureStatusNone) cudaGetLastError();
      cst = false;
    }
    t.p = ws.get<double>(count);
    eperm(sps.c_str(), 1.0, X, 0.0, t, s);
    return t.p;
  };
  Gemm g;
  g.M = M; g.N = N; g.K = K;
  g.batch = nb;
  // A operand
  const double* Ap = A.p;
  if (sp.a == bat + mi + kord) { g.ta = false; g.lda = K; g.a_const = oc && oc->constant(A.p); }
  else if (sp.a == bat + kord + mi) { g.ta = true; g.lda = M; g.a_const = oc && oc->constant(A.p); }
  else {
    bool cst = false;
    Ap = operand(A, sp.a, bat + mi + kord, cst);
    g.a_const = cst;
    g.ta = false;
    g.lda = K;
  }
  g.A = Ap;
  g.sA = M * K;
  const double* Bp = B.p;
  if (sp.b == bat + kord + ni) { g.tb = false; g.ldb = N; g.b_const = oc && oc->constant(B.p); }
  else if (sp.b == bat + ni + kord) { g.tb = true; g.ldb = K; g.b_const = oc && oc->constant(B.p); }
  else {
    bool cst = false;
    Bp = operand(B, sp.b, bat + kord + ni, cst);
    g.b_const = cst;
    g.tb = false;
    g.ldb = N;
  }
  g.B = Bp;
  g.sB = K * N;
  if (sp.c == bat + mi + ni) {
    g.C = C.p;
    g.ldc = N;
    g.sC = M * N;
    g.alpha = alpha;
    g.beta = beta;
    gemm_f64(g, ws, s, sm_count);
  } else {
    DT t;
    t.p = ws.get<double>(size_t(nb * M * N));
    for (char ch : bat + mi + ni) t.d.push_back(size[ch]);
    g.C = t.p;
    g.ldc = N;
    g.sC = M * N;
    g.alpha = alpha;
    g.beta = 0.0;
    gemm_f64(g, ws, s, sm_count);
    const std::string sps = bat + mi + ni + "->" + sp.c;
    eperm(sps.c_str(), 1.0, t, beta, C, s);
  }
}

// ---------------------------------------------------------------------------------
namespace {
__global__ void k_fill(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}
__global__ void k_axpby(double* y, const double* x, int64_t n, double a, double b) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = (b == 0.0) ? a * x[i] : a * x[i] + b * y[i];
}
constexpr int DOT_BLOCKS = 512;
constexpr int DOT_CHUNK = 8;
// partial[k][blk] = sum over the block's grid-stride share of x_k * y; each pass over y
// serves DOT_CHUNK vectors x_k (one read of y per chunk)
__global__ void k_dots_stage1(const double* x, int64_t ldx, int nx, const double* y, int64_t n,
                              double* partial) {
  __shared__ double red[DOT_CHUNK][256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < nx; k0 += DOT_CHUNK) {
    const int kc = min(DOT_CHUNK, nx - k0);
    double acc[DOT_CHUNK];
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c) acc[c] = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
      const double yi = y[i];
#pragma unroll
      for (int c = 0; c < DOT_CHUNK; ++c)
        if (c < kc) acc[c] = fma(x[int64_t(k0 + c) * ldx + i], yi, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c) {
      double v = acc[c];
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
// partial[(k * ny + j)][blk] for DOT_CHUNK x-vectors per pass and NY <= 4 y-vectors
template <int NY>
__global__ void k_dots_block1(const double* x, int64_t ldx, int nx, const double* y, int64_t ldy,
                              int64_t n, double* partial) {
  __shared__ double red[DOT_CHUNK * NY][256 / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < nx; k0 += DOT_CHUNK) {
    const int kc = min(DOT_CHUNK, nx - k0);
    double acc[DOT_CHUNK][NY];
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c)
#pragma unroll
      for (int j = 0; j < NY; ++j) acc[c][j] = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
      double yv[NY];
#pragma unroll
      for (int j = 0; j < NY; ++j) yv[j] = y[int64_t(j) * ldy + i];
#pragma unroll
      for (int c = 0; c < DOT_CHUNK; ++c) {
        if (c < kc) {
          const double xv = x[int64_t(k0 + c) * ldx + i];
#pragma unroll
          for (int j = 0; j < NY; ++j) acc[c][j] = fma(xv, yv[j], acc[c][j]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c)
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        double v = acc[c][j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[c * NY + j][warp] = v;
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

__global__ void k_dots_stage2(const double* partial, int nblk, double* out) {
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
}  // namespace

void fill(double* p, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = int(std::min<int64_t>((n + 255) / 256, 8192));
  k_fill<<<blocks, 256, 0, s>>>(p, n, v);
  MLCC_CHECK_LAUNCH();
}
void axpby(double* y, const double* x, int64_t n, double a, double b, cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = int(std::min<int64_t>((n + 255) / 256, 8192));
  k_axpby<<<blocks, 256, 0, s>>>(y, x, n, a, b);
  MLCC_CHECK_LAUNCH();
}
void dots(const double* x, int64_t ldx, int nx, const double* y, int64_t n, double* out_dev,
          Arena& ws, cudaStream_t s) {
  if (nx <= 0) return;
  if (g_vec32) return dots32(x, ldx, nx, y, n, out_dev, ws, s);
  Scope sc(ws);
  int blocks = int(std::min<int64_t>((n + 255) / 256, DOT_BLOCKS));
  blocks = std::max(blocks, 1);
  double* partial = ws.get<double>(size_t(nx) * blocks);
  k_dots_stage1<<<blocks, 256, 0, s>>>(x, ldx, nx, y, n, partial);
  MLCC_CHECK_LAUNCH();
  k_dots_stage2<<<nx, 256, 0, s>>>(partial, blocks, out_dev);
  MLCC_CHECK_LAUNCH();
}
void dots_block(const double* x, int64_t ldx, int nx, const double* y, int64_t ldy, int ny,
                int64_t n, double* out_dev, Arena& ws, cudaStream_t s) {
  if (nx <= 0 || ny <= 0) return;
  if (g_vec32) return dots_block32(x, ldx, nx, y, ldy, ny, n, out_dev, ws, s);
  MLCC_REQUIRE(ny <= 4, "dots_block: at most 4 y-vectors");
  Scope sc(ws);
  int blocks = int(std::min<int64_t>((n + 255) / 256, DOT_BLOCKS));
  blocks = std::max(blocks, 1);
  double* partial = ws.get<double>(size_t(nx) * ny * blocks);
  switch (ny) {
    case 1: k_dots_block1<1><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
    case 2: k_dots_block1<2><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
    case 3: k_dots_block1<3><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
    default: k_dots_block1<4><<<blocks, 256, 0, s>>>(x, ldx, nx, y, ldy, n, partial); break;
  }
  MLCC_CHECK_LAUNCH();
  k_dots_stage2<<<nx * ny, 256, 0, s>>>(partial, blocks, out_dev);
  MLCC_CHECK_LAUNCH();
}

void copy_d2h(double* h, const double* d, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  MLCC_CUDA(cudaMemcpyAsync(h, d, size_t(n) * 8, cudaMemcpyDeviceToHost, s));
  MLCC_CUDA(cudaStreamSynchronize(s));
}
void copy_h2d(double* d, const double* h, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  MLCC_CUDA(cudaMemcpyAsync(d, h, size_t(n) * 8, cudaMemcpyHostToDevice, s));
}

}  // namespace mlcc

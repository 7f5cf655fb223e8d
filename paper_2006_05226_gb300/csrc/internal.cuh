// Internal declarations shared by the libmlcc translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <atomic>
#include <map>
#include <stdexcept>

#include "../../include/mlcc.h"

namespace mlcc {

// ---------------------------------------------------------------------------------
// Errors: every failure becomes an mlcc::Error caught at the ABI boundary.
struct Error : std::runtime_error {
  mlcc_status status;
  Error(mlcc_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};
void set_last_error(const std::string& msg);

#define MLCC_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      throw ::mlcc::Error(e_ == cudaErrorMemoryAllocation ? MLCC_E_OOM : MLCC_E_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(e_));       \
    }                                                                                \
  } while (0)
// every kernel launch is followed by MLCC_CHECK_LAUNCH(), which also counts it
void count_launch();
void count_launches(int64_t n);   // kernels of a replayed CUDA graph
#define MLCC_CHECK_LAUNCH()          \
  do {                               \
    ::mlcc::count_launch();          \
    MLCC_CUDA(cudaGetLastError());   \
  } while (0)
#define MLCC_REQUIRE(cond, msg)                                      \
  do {                                                               \
    if (!(cond)) throw ::mlcc::Error(MLCC_E_ARG, std::string(msg));  \
  } while (0)

// Runs an entry point's body; every mlcc::Error and std::exception becomes a status code
// with its message in mlcc_last_error(), so no exception crosses the C ABI.
template <class F>
mlcc_status guard(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MLCC_E_CUDA;
  } catch (...) {
    set_last_error("unknown error");
    return MLCC_E_CUDA;
  }
}

// ---------------------------------------------------------------------------------
// Device arena: one cudaMalloc, bump allocation with marks. Allocations are 256-byte
// aligned so every TMA / vector access starts on an aligned boundary.
class Arena {
 public:
  Arena() = default;
  ~Arena();
  void reserve(size_t bytes);
  void* alloc(size_t bytes);
  template <class T> T* get(size_t n) { return static_cast<T*>(alloc(n * sizeof(T))); }
  size_t mark() const { return top_; }
  void release(size_t m) { top_ = m; }
  size_t capacity() const { return cap_; }
  size_t high_water() const { return hw_; }
  const char* base() const { return base_; }
 private:
  char* base_ = nullptr;
  size_t cap_ = 0, top_ = 0, hw_ = 0;
};

// RAII scratch scope on an arena.
struct Scope {
  Arena& a;
  size_t m;
  explicit Scope(Arena& ar) : a(ar), m(ar.mark()) {}
  ~Scope() { a.release(m); }
};

// ---------------------------------------------------------------------------------
// Per-context kernel timing (CUDA events around launches of one kernel family).
struct KernelTimer {
  bool enabled = false;
  struct Rec { cudaEvent_t a, b; double flop; };
  std::map<std::string, std::vector<Rec>> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get_event();
  void begin(const char* fam, cudaStream_t s, double flop, cudaEvent_t* a, cudaEvent_t* b);
  void reset();
  ~KernelTimer();
};

}  // namespace mlcc

struct mlcc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  mlcc::KernelTimer timer;
  int sm_count = 0;
  int64_t budget = 0;                 // device-memory budget of the context (0: none)
  std::atomic<int64_t> held{0};       // workspace bytes of the context's live systems
};

namespace mlcc {

// ---------------------------------------------------------------------------------
// Dense binary64 GEMM on the CUDA cores (row-major):
//   C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b]             (batch mode)
//   C    = alpha * sum_b op(A[b]) op(B[b]) + beta * C          (reduce mode)
// op(A) is M x K (A[m*lda+k], or A[k*lda+m] when ta), op(B) is K x N.
struct Gemm {
  bool ta = false, tb = false;
  int64_t M = 0, N = 0, K = 0;
  double alpha = 1.0, beta = 0.0;
  const double* A = nullptr; int64_t lda = 0, sA = 0;
  const double* B = nullptr; int64_t ldb = 0, sB = 0;
  double* C = nullptr; int64_t ldc = 0, sC = 0;
  int64_t batch = 1;
  bool reduce = false;
  bool a_const = false, b_const = false;   // operand unchanged until the cache is cleared
};
void gemm_f64(const Gemm& g, Arena& ws, cudaStream_t s, int sm_count);

// Low-precision routing: while a LowpScope is alive on this thread, gemm_f64 sends large
// GEMMs to the tcgen05 tensor-core path (bfloat16 pieces per mlcc_precision, fp32
// accumulation per split, binary64 reduction); everything else stays binary64.
struct OperandCache;   // bfloat16 pieces of constant GEMM operands (per system)
struct LowpScope {
  int prev;
  int* err;
  int* prev_err;
  OperandCache* prev_cache;
  LowpScope(int precision, int* err_flag, OperandCache* cache = nullptr);
  ~LowpScope();
};
int lowp_precision();
// the split-bfloat16 precisions (a low-precision phase); MLCC_FP64 and MLCC_FP64E are
// binary64-class
inline bool is_split_precision(int p) { return p == MLCC_BF16 || p == MLCC_BF16X3 || p == MLCC_BF16X6; }
int* lowp_error_flag();
OperandCache* lowp_cache();
OperandCache* operand_cache_new();
void operand_cache_clear(OperandCache* c);
void operand_cache_free(OperandCache* c);
// device memory ranges whose contents stay fixed while the cache is valid
void operand_cache_set_ranges(OperandCache* c, const std::vector<std::pair<const char*, size_t>>& r);
bool gemm_tc(const Gemm& g, int precision, Arena& ws, cudaStream_t s, int sm_count, int* err);
// MLCC_FP64E: binary64 GEMM from exact integer slices on the tensor cores (tc_emu.cu);
// gemm_emu returns false, launching nothing, exactly when gemm_emu_fits is false
bool gemm_emu(const Gemm& g, Arena& ws, cudaStream_t s, int sm_count, int* err);
bool gemm_emu_fits(const Gemm& g, const Arena& ws);
// C = alpha * sum_s partial[s] + beta * C (deterministic order)
void reduce_partials(const double* partial, int nsplit, int64_t M, int64_t N, double* C,
                     int64_t ldc, double alpha, double beta, cudaStream_t s);

// Strided permute-accumulate: dst = alpha * src (re-indexed) + beta * dst, both given by
// dims and element strides in the order of the destination's loop nest (<= 8 dims).
void permute_f64(int nd, const int64_t* dims, const double* src, const int64_t* src_strides,
                 double* dst, const int64_t* dst_strides, double alpha, double beta,
                 cudaStream_t s);

// Contiguous row-major device tensor (binary64).
struct DT {
  double* p = nullptr;
  std::vector<int64_t> d;
  int64_t size() const { int64_t n = 1; for (auto x : d) n *= x; return n; }
};

// Pairwise tensor contraction C = alpha * contract(A, B) + beta * C following an einsum
// specification "ab,bc->ac". Indices shared by A, B and C are batch indices, indices in
// A and C (B and C) are rows (columns), indices in A and B only are summed. Operands are
// brought to GEMM layout by permute kernels when their order requires it.
void einsum(const char* spec, double alpha, const DT& A, const DT& B, double beta, const DT& C,
            Arena& ws, cudaStream_t s, int sm_count);
// C = alpha * permute(A) + beta * C with a spec "abcd->cdab".
void eperm(const char* spec, double alpha, const DT& A, double beta, const DT& C, cudaStream_t s);

// Elementwise / reduction helpers (binary64).
void fill(double* p, int64_t n, double v, cudaStream_t s);
void axpby(double* y, const double* x, int64_t n, double a, double b, cudaStream_t s);  // y = a x + b y
// Deterministic dot products: out_dev[k] = sum_i x_k[i] y[i] for k < nx (x_k at x + k*ldx).
void dots(const double* x, int64_t ldx, int nx, const double* y, int64_t n, double* out_dev,
          Arena& ws, cudaStream_t s);
// out_dev[k * ny + j] = x_k . y_j for k < nx, j < ny (ny <= 4): one pass over each x_k
void dots_block(const double* x, int64_t ldx, int nx, const double* y, int64_t ldy, int ny,
                int64_t n, double* out_dev, Arena& ws, cudaStream_t s);
// Binary32 arithmetic on binary64 vectors (vec32.cu): while a Vec32Scope is on for this
// thread, dots, dots_block and the skinny GEMMs (M <= 16, K <= 64, B not transposed)
// convert each loaded element to binary32 and multiply-add in binary32 (the Davidson
// vector work of a split-precision phase); everything else is unchanged.
struct Vec32Scope {
  bool prev;
  explicit Vec32Scope(bool on);
  ~Vec32Scope();
  void set(bool on);
};
bool vec32_active();
void dots32(const double* x, int64_t ldx, int nx, const double* y, int64_t n, double* out_dev,
            Arena& ws, cudaStream_t s);
void dots_block32(const double* x, int64_t ldx, int nx, const double* y, int64_t ldy, int ny,
                  int64_t n, double* out_dev, Arena& ws, cudaStream_t s);
bool skinny32(const Gemm& g, cudaStream_t s);
// binary32 vector storage: dot products, C = alpha op(A) B + beta C with B [K][N] binary32
// and C binary32 (c_f32) or binary64 (M <= 16, K <= 64), conversions, scaling
void dots_f32(const float* x, int64_t ldx, int nx, const float* y, int64_t n, double* out_dev,
              Arena& ws, cudaStream_t s);
void dots_block_f32(const float* x, int64_t ldx, int nx, const float* y, int64_t ldy, int ny,
                    int64_t n, double* out_dev, Arena& ws, cudaStream_t s);
void combine_f32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool ta, const float* B,
                 int64_t ldb, void* C, bool c_f32, int64_t ldc, double alpha, double beta, cudaStream_t s);
void cvt_d2f(const double* x, float* y, int64_t n, cudaStream_t s);
void cvt_f2d(const float* x, double* y, int64_t n, cudaStream_t s);
void scale_f32(float* x, int64_t n, double a, cudaStream_t s);
void copy_d2h(double* h, const double* d, int64_t n, cudaStream_t s);
void copy_h2d(double* d, const double* h, int64_t n, cudaStream_t s);

}  // namespace mlcc

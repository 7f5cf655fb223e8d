// Shared pieces of the tensor-core GEMM units: the generic binary64 operand view, the
// cache of converted constant operands and the launch interface of the emulation mode.
#pragma once
#include <cuda_bf16.h>

#include <string>
#include <tuple>
#include <vector>

#include "internal.cuh"

namespace mlcc {

inline int64_t pad64(int64_t k) { return (k + 63) / 64 * 64; }

// Generic operand of a tensor-core GEMM: dst[r][s * Kp + kk] = piece_s(X(r, kk)) with
//   r  = rb * Mrow + m  (row batches, stride sRow),  kk = kb * Kblk + k  (K batches, stride sK)
//   X(r, kk) = base[rb * sRow + kb * sK + (tr ? k * ld + m : m * ld + k)]
struct GOp {
  const double* base;
  int64_t R, Mrow, sRow, Ktot, Kblk, sK, ld, Kp;
  int tr, S;
  int piece[6];
};
__device__ __forceinline__ double gop_load(const GOp& o, int64_t r, int64_t kk) {
  if (r >= o.R || kk >= o.Ktot) return 0.0;
  // the batch divisions only when the operand is batched (uniform branches)
  int64_t rb = 0, m = r, kb = 0, k = kk;
  if (o.Mrow < o.R) {
    rb = r / o.Mrow;
    m = r - rb * o.Mrow;
  }
  if (o.Kblk < o.Ktot) {
    kb = kk / o.Kblk;
    k = kk - kb * o.Kblk;
  }
  return o.base[rb * o.sRow + kb * o.sK + (o.tr ? k * o.ld + m : m * o.ld + k)];
}

// Converted copies of GEMM operands that stay fixed while the cache is valid (one per
// system; cleared when the Jacobian ground state changes).
struct OperandCache {
  struct Entry {
    std::tuple<const void*, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int, int, int> key;
    __nv_bfloat16* p;
  };
  std::vector<Entry> entries;
  // binary64 copies of constant einsum operands in GEMM order (source, dims, permutation)
  struct Perm {
    const void* src;
    std::vector<int64_t> dims;
    std::string spec;
    double* p;
  };
  std::vector<Perm> perms;
  std::vector<void*> blocks;
  std::vector<std::pair<const char*, size_t>> ranges;
  bool constant(const void* p) const {
    const char* q = static_cast<const char*>(p);
    for (auto& r : ranges)
      if (q >= r.first && q < r.first + r.second) return true;
    return false;
  }
};

// Emulation mode of the tcgen05 GEMM: A [M][S*Kp], B [N][S*Kp] hold S integer slices of
// Kp = 64 * kbp K elements each; chunk z of group g (gstart[g] <= z < gstart[g + 1])
// sums, over at most `ch` K blocks of the slice pairs (i, g - i) concatenated in i, the
// products A_i B_(g-i) into part[z][M][ldp] (fp32, exact while ch * 64 * max|q|^2 <= 2^24:
// 4096 products of digits |q| <= 64).
constexpr int TC_EMU_MAX_S = 8;
void tc_gemm_emu_launch(const __nv_bfloat16* A, const __nv_bfloat16* B, int64_t M, int64_t N, int S,
                        int64_t Kp, int ch, const int* gstart, float* part, int64_t ldp, int* err,
                        cudaStream_t s);
// binary64 GEMM emulated with exact integer slices on the tensor cores (tc_emu.cu);
// false when the shape or the workspace does not allow it.
bool gemm_emu(const Gemm& g, Arena& ws, cudaStream_t s, int sm_count, int* err);
bool gemm_emu_fits(const Gemm& g, const Arena& ws);

}  // namespace mlcc

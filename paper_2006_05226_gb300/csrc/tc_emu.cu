// Binary64 GEMM emulated on the tcgen05 tensor cores with exact integer slices
// (the error-free splitting of Ozaki's scheme, arranged for bfloat16 and fp32 accumulate).
//
// GB300 issues about two binary64 FMAs per SM and clock, so a binary64 contraction with
// operand reuse is bound by the FP64 pipe, not by HBM. Here each operand row r (a row of
// A, or a column of B, along the contraction index k) is scaled by 2^(F - E_r), E_r the
// exponent of the row's largest magnitude (|x| < 2^E_r), and rounded to an integer X of at
// most F = 6 + 7 (S - 1) bits, written as S signed digits of base 2^7:
//     X = sum_{s<S} q_s 2^(7 (S - 1 - s)),   |q_s| <= 64   (each exact in bfloat16).
// Then, with 0-based digit indices,
//     C_mn = 2^(E_m + E_n - 2F) sum_{s,t} 2^(7 (2S - 2 - s - t)) sum_k qA_s[m][k] qB_t[n][k]
// of which the pairs with s + t <= S - 1 are kept: every term down to 2^(-7 (S - 1)) of the
// leading one, the rest lies below the rounding of X. A product of two digits is at most
// 2^12 in magnitude, so an fp32 tensor-core accumulation of at most 4096 of them stays an
// exact integer (|sum| <= 2^24). The GEMM kernel sums each group g = s + t in chunks of at
// most 4096 products and writes the exact chunk sums; a reduction combines them in 64-bit
// integers and rounds the total to binary64 (once for K <= 2^17), then applies
// 2^(E_m + E_n ...), alpha and beta. With S = 8 (F = 55, 36 digit pairs) the truncation and
// the rounding of X cost about 2^-53 of 2^(E_m + E_n) per product, the binary64 level of a
// product of the row maxima. Seven-bit digits (rather than eight) need 36 pairs instead of
// 28 but four times fewer exact chunks: the chunk planes written by the GEMM and read by
// the reduction, which bound both kernels, shrink about threefold.
#include "system.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace mlcc {

namespace {

constexpr int EMU_S = 8;              // digits per operand element
constexpr int EMU_BITS = 7;           // digit base 2^7, |digit| <= 64
constexpr int EMU_F = (EMU_BITS - 1) + EMU_BITS * (EMU_S - 1);   // 55 bits of X
constexpr int EMU_CH = 64;            // K blocks of 64 per exact fp32 chunk (4096 products)
constexpr int EMU_HI = 28;            // the 64-bit combination: T = hi 2^EMU_HI + lo
static_assert(EMU_CH * 64 * (1 << (2 * (EMU_BITS - 1))) <= (1 << 24), "chunk sums must stay exact in fp32");
constexpr int EMU_NONFINITE = 1 << 30;
constexpr int64_t EMU_MAX_K = int64_t(1) << 20;   // keeps the 64-bit combination exact
constexpr int64_t EMU_MIN_MN = 16;                 // narrower products stay on the FMA units

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}
// E with max|x| < 2^E from the bit pattern of the largest magnitude (integer compares
// order non-negative binary64 values, NaN and Inf above every finite value)
__device__ __forceinline__ int exponent_of_max(unsigned long long m) {
  if (m == 0) return 0;   // zero row: every digit is zero
  const int ef = int(m >> 52);
  if (ef == 0x7FF) return EMU_NONFINITE;
  if (ef > 0) return ef - 1022;          // m = 1.f * 2^(ef - 1023)
  const int p = 63 - __clzll(m);         // subnormal: m = fraction * 2^-1074
  return p + 1 - 1074;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Largest |x| per operand row as binary64 bit patterns, merged over K chunks with
// atomicMax (blockIdx.y is the chunk), then turned into exponents.
// K contiguous in the source: one warp per row
__global__ void k_emu_rowmax_direct(GOp o, int64_t kchunk, unsigned long long* mx) {
  const int lane = threadIdx.x & 31;
  const int64_t k0 = int64_t(blockIdx.y) * kchunk, k1 = min(o.Ktot, k0 + kchunk);
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < o.R; r += nwarps) {
    unsigned long long m = 0;
    for (int64_t kk = k0 + lane; kk < k1; kk += 32) m = umax64(m, abs_bits(gop_load(o, r, kk)));
    for (int off = 16; off > 0; off >>= 1) m = umax64(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    if (lane == 0 && m) atomicMax(mx + r, m);
  }
}
// rows contiguous in the source: 32 rows per block, 8 lanes over k each
__global__ void k_emu_rowmax_tr(GOp o, int64_t kchunk, unsigned long long* mx) {
  __shared__ unsigned long long red[8][33];
  const int64_t r = int64_t(blockIdx.x) * 32 + threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.y) * kchunk, k1 = min(o.Ktot, k0 + kchunk);
  unsigned long long m = 0;
  if (r < o.R)
    for (int64_t kk = k0 + threadIdx.y; kk < k1; kk += 8) m = umax64(m, abs_bits(gop_load(o, r, kk)));
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && r < o.R) {
    for (int y = 1; y < 8; ++y) m = umax64(m, red[y][threadIdx.x]);
    if (m) atomicMax(mx + r, m);
  }
}
__global__ void k_emu_exponents(const unsigned long long* mx, int64_t R, int* ex) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < R; r += int64_t(gridDim.x) * blockDim.x)
    ex[r] = exponent_of_max(mx[r]);
}

// bfloat16 bit pattern of an integer |q| <= 128 (exact)
__device__ __forceinline__ __nv_bfloat16 small_int_bf16(int q) {
  unsigned short h = 0;
  if (q != 0) {
    const unsigned a = unsigned(q < 0 ? -q : q);
    const int p = 31 - __clz(a);   // a = 2^p (1 + f), p <= 7
    h = static_cast<unsigned short>((q < 0 ? 0x8000u : 0u) | (unsigned(p + 127) << 7) | ((a << (7 - p)) & 0x7Fu));
  }
  return __ushort_as_bfloat16(h);
}
// The EMU_S digits of X = round(x 2^(F - E)), most significant first, by integer
// arithmetic on the binary64 fields (round half away from zero on the magnitude, then
// round-to-nearest digits so every digit stays within [-128, 128]).
__device__ __forceinline__ void emu_digits(double x, int E, __nv_bfloat16 q[EMU_S]) {
  constexpr int F = EMU_F;
  long long X = 0;
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ef = int((b >> 52) & 0x7FF);
  if (E != EMU_NONFINITE && ef != 0x7FF && (b << 1) != 0) {
    const unsigned long long mant = (b & ((1ull << 52) - 1)) | (ef ? (1ull << 52) : 0ull);
    const int e = ef ? ef : 1;                 // |x| = mant * 2^(e - 1075)
    const int sh = e - 1075 + F - E;           // |X| = mant * 2^sh < 2^F since |x| < 2^E
    unsigned long long mag;
    if (sh >= 0) mag = mant << sh;
    else if (sh > -63) mag = (mant + (1ull << (-sh - 1))) >> (-sh);
    else mag = 0;
    X = (b >> 63) ? -static_cast<long long>(mag) : static_cast<long long>(mag);
  }
#pragma unroll
  for (int s = 0; s < EMU_S; ++s) {
    const int shift = EMU_BITS * (EMU_S - 1 - s);
    long long d = X;
    if (shift > 0) d = (X + (1LL << (shift - 1))) >> shift;   // arithmetic shift: floor
    X -= d * (1LL << shift);
    q[s] = small_int_bf16(int(d));
  }
}

// K contiguous in the source: dst[r][s * Kp + kk], one thread per (r, kk), kk fastest
__global__ void k_emu_slice_direct(GOp o, const int* ex, __nv_bfloat16* dst) {
  const int64_t total = o.R * o.Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / o.Kp, kk = t - r * o.Kp;
    __nv_bfloat16 q[EMU_S];
    emu_digits(gop_load(o, r, kk), ex[r], q);
#pragma unroll
    for (int s = 0; s < EMU_S; ++s) dst[r * (EMU_S * o.Kp) + s * o.Kp + kk] = q[s];
  }
}
// rows contiguous in the source: 32 x 32 tiles through shared memory
__global__ void k_emu_slice_tr(GOp o, const int* ex, __nv_bfloat16* dst) {
  __shared__ double tile[32][33];
  const int64_t r0 = int64_t(blockIdx.x) * 32, k0 = int64_t(blockIdx.y) * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) tile[y][threadIdx.x] = gop_load(o, r0 + threadIdx.x, k0 + y);
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, kk = k0 + threadIdx.x;
    if (r >= o.R || kk >= o.Kp) continue;
    __nv_bfloat16 q[EMU_S];
    emu_digits(tile[threadIdx.x][y], ex[r], q);
#pragma unroll
    for (int s = 0; s < EMU_S; ++s) dst[r * (EMU_S * o.Kp) + s * o.Kp + kk] = q[s];
  }
}

struct EmuRed {
  const float* P;          // [chunk][M][ldp] exact chunk sums
  int64_t M, Nw, ldp;
  int gstart[TC_EMU_MAX_S + 1];
  const int* ea;           // [M] row exponents of A
  const int* eb;           // [Nw] row exponents of B (this panel)
  double alpha, beta;
  double* C;               // [M][ldc]
  int64_t ldc;
  int64_t n0;              // first output column of the panel
  int64_t nb, sCb;         // batched output columns (nb > 0): column b nb + c at C + b sCb + c
  // element index below 2^31: t / Nw and col / nb by division by invariant integers
  // (Granlund and Montgomery, 1994: q = (umulhi(m, n) + n) >> l, exact for n < 2^31)
  int small;
  uint32_t nw_magic, nw_shift, nb_magic, nb_shift;
};
__device__ __forceinline__ uint32_t div_inv(uint32_t n, uint32_t magic, uint32_t shift) {
  return (__umulhi(magic, n) + n) >> shift;
}
// x 2^e: a multiplication by the power of two while it is a normal binary64 number (the
// same correctly rounded result as ldexp), ldexp beyond
__device__ __forceinline__ double scale_pow2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __longlong_as_double(static_cast<long long>(e + 1023) << 52);
  return ldexp(x, e);
}
// C = alpha 2^(E_m + E_n - 2F + 7 (S - 1)) T + beta C with T = sum_g 2^(7 (S - 1 - g)) G_g,
// G_g the integer sum of group g's chunks; T is held exactly as hi 2^28 + lo (both exact in
// binary64 while K <= 2^17) and rounded once.
__global__ void k_emu_reduce(EmuRed r) {
  const int64_t total = r.M * r.Nw, plane = r.M * r.ldp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    int64_t m, n;
    if (r.small) {
      m = div_inv(uint32_t(t), r.nw_magic, r.nw_shift);
      n = t - m * r.Nw;
    } else {
      m = t / r.Nw;
      n = t - m * r.Nw;
    }
    const float* p = r.P + m * r.ldp + n;
    long long hi = 0, lo = 0;
#pragma unroll
    for (int g = 0; g < EMU_S; ++g) {
      long long G = 0;
      for (int z = r.gstart[g]; z < r.gstart[g + 1]; ++z) G += static_cast<long long>(__float2int_rn(p[z * plane]));
      const int sh = EMU_BITS * (EMU_S - 1 - g);
      if (sh >= EMU_HI) hi += G * (1LL << (sh - EMU_HI));
      else lo += G * (1LL << sh);
    }
    const int ea = r.ea[m], eb = r.eb[n];
    double v;
    if (ea == EMU_NONFINITE || eb == EMU_NONFINITE) {
      v = __longlong_as_double(0x7FF8000000000000LL);
    } else {
      v = fma(static_cast<double>(hi), double(1LL << EMU_HI), static_cast<double>(lo));
      v = scale_pow2(v, ea + eb - 2 * EMU_F + EMU_BITS * (EMU_S - 1));
    }
    int64_t col = r.n0 + n, cb = 0;
    if (r.nb > 0) {
      cb = r.small ? int64_t(div_inv(uint32_t(col), r.nb_magic, r.nb_shift)) : col / r.nb;
      col -= cb * r.nb;
    }
    double* c = r.C + cb * r.sCb + m * r.ldc + col;
    double out = (r.alpha == 0.0) ? 0.0 : r.alpha * v;
    if (r.beta != 0.0) out += r.beta * *c;
    *c = out;
  }
}

// magic number and shift of the division by d (1 <= d < 2^31) for dividends below 2^31
void div_inv_consts(int64_t d, uint32_t* magic, uint32_t* shift) {
  uint32_t l = 0;
  while ((uint64_t(1) << l) < uint64_t(d)) ++l;
  *magic = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - uint64_t(d))) / uint64_t(d) + 1);
  *shift = l;
}

int grid_for(int64_t total, int threads) {
  return int(std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 65535)));
}

void emu_convert(const GOp& o, int* ex, __nv_bfloat16* dst, Arena& ws, cudaStream_t s) {
  {
    // row maxima: enough (row block, K chunk) blocks to fill the GPU even for few rows
    Scope sc(ws);
    unsigned long long* mx = ws.get<unsigned long long>(size_t(o.R));
    MLCC_CUDA(cudaMemsetAsync(mx, 0, size_t(o.R) * 8, s));
    const int64_t rblocks = o.tr ? (o.R + 31) / 32 : (o.R + 7) / 8;
    const int64_t nk = std::max<int64_t>(1, std::min<int64_t>({(o.Ktot + 255) / 256, (1216 + rblocks - 1) / rblocks, 65535}));
    const int64_t kchunk = (o.Ktot + nk - 1) / nk;
    MLCC_REQUIRE(rblocks < (int64_t(1) << 31), "gemm_emu: grid");
    const dim3 grid{unsigned(std::min<int64_t>(rblocks, o.tr ? (int64_t(1) << 31) - 1 : 65535)), unsigned(nk), 1};
    if (!o.tr) k_emu_rowmax_direct<<<grid, 256, 0, s>>>(o, kchunk, mx);
    else k_emu_rowmax_tr<<<grid, dim3(32, 8), 0, s>>>(o, kchunk, mx);
    MLCC_CHECK_LAUNCH();
    k_emu_exponents<<<grid_for(o.R, 256), 256, 0, s>>>(mx, o.R, ex);
    MLCC_CHECK_LAUNCH();
  }
  if (!o.tr) {
    k_emu_slice_direct<<<grid_for(o.R * o.Kp, 256), 256, 0, s>>>(o, ex, dst);
    MLCC_CHECK_LAUNCH();
  } else {
    MLCC_REQUIRE((o.R + 31) / 32 < (int64_t(1) << 31) && (o.Kp + 31) / 32 < 65536, "gemm_emu: grid");
    dim3 blk(32, 8), grd(unsigned((o.R + 31) / 32), unsigned((o.Kp + 31) / 32));
    k_emu_slice_tr<<<grd, blk, 0, s>>>(o, ex, dst);
    MLCC_CHECK_LAUNCH();
  }
}

size_t slice_bytes(const GOp& o) { return size_t(o.R) * EMU_S * o.Kp * 2; }

// slices and row exponents of an operand, from the cache when it is marked constant
const __nv_bfloat16* emu_operand(const GOp& o, int side, bool cacheable, Arena& ws, cudaStream_t s,
                                 const int** ex_out) {
  OperandCache* c = lowp_cache();
  if (c && !(cacheable || c->constant(o.base))) c = nullptr;
  const size_t sb = slice_bytes(o), bytes = sb + size_t(o.R) * 4;
  auto fresh = [&](void* mem) {
    auto* d = static_cast<__nv_bfloat16*>(mem);
    int* ex = reinterpret_cast<int*>(static_cast<char*>(mem) + sb);
    emu_convert(o, ex, d, ws, s);
    *ex_out = ex;
    return d;
  };
  if (!c) return fresh(ws.alloc(bytes));
  auto key = std::make_tuple(static_cast<const void*>(o.base), o.R, o.Mrow, o.sRow, o.Ktot, o.Kblk, o.sK, o.ld,
                             o.tr, 1000 + EMU_S, side);
  for (auto& e : c->entries)
    if (e.key == key) {
      *ex_out = reinterpret_cast<const int*>(reinterpret_cast<const char*>(e.p) + sb);
      return e.p;
    }
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fresh(ws.alloc(bytes));
  }
  c->blocks.push_back(mem);
  __nv_bfloat16* d = fresh(mem);
  c->entries.push_back({key, d});
  return d;
}

}  // namespace

namespace {
struct EmuPlan {
  GOp a, b;
  int64_t M, N, Kp, Np;
  int64_t nb, sCb;   // batched output columns (a batch sharing A flattened along N)
  int gstart[TC_EMU_MAX_S + 1];
  int nch;
};
// shapes, chunk table and output panel width; false when the emulation cannot run
bool emu_plan(const Gemm& g, const Arena& ws, EmuPlan& P) {
  const bool batched = !g.reduce && g.batch > 1;
  const bool flatten = batched && g.sB == 0 && g.sC == g.M * g.ldc;
  const bool flat_n = batched && !flatten && g.sA == 0;
  if (batched && !flatten && !flat_n) return false;
  const int64_t M = flatten ? g.M * g.batch : g.M;
  const int64_t Ktot = g.reduce ? g.K * g.batch : g.K;
  const int64_t N = flat_n ? g.N * g.batch : g.N;
  if (M < EMU_MIN_MN || N < EMU_MIN_MN || Ktot < 1 || Ktot > EMU_MAX_K) return false;
  P.nb = flat_n ? g.N : 0;
  P.sCb = flat_n ? g.sC : 0;
  const int64_t Kp = pad64(Ktot), kbp = Kp / 64;
  for (int q = 0; q <= TC_EMU_MAX_S; ++q) P.gstart[q] = 0;
  for (int q = 0; q < EMU_S; ++q) P.gstart[q + 1] = P.gstart[q] + int(((q + 1) * kbp + EMU_CH - 1) / EMU_CH);
  for (int q = EMU_S + 1; q <= TC_EMU_MAX_S; ++q) P.gstart[q] = P.gstart[EMU_S];
  P.nch = P.gstart[EMU_S];
  if (P.nch >= 65536) return false;
  GOp& a = P.a;
  a = GOp{};
  a.base = g.A;
  a.R = M;
  a.Mrow = flatten ? g.M : M;
  a.sRow = flatten ? g.sA : 0;
  a.Ktot = Ktot;
  a.Kblk = g.reduce ? g.K : Ktot;
  a.sK = g.reduce ? g.sA : 0;
  a.ld = g.lda;
  a.Kp = Kp;
  a.tr = g.ta ? 1 : 0;
  a.S = EMU_S;
  GOp& b = P.b;
  b = a;
  b.base = g.B;
  b.R = N;
  b.Mrow = flat_n ? g.N : N;
  b.sRow = flat_n ? g.sB : 0;
  b.sK = g.reduce ? g.sB : 0;
  b.ld = g.ldb;
  b.tr = g.tb ? 0 : 1;
  // workspace: slices of both operands (unless cached), then the chunk planes of a panel
  // of output columns as wide as the rest allows (a multiple of 256, the tile width)
  const size_t ops = slice_bytes(a) + slice_bytes(b) + size_t(M + N) * 4 + 4 * 256;
  const size_t free_bytes = ws.capacity() > ws.mark() + ops + (size_t(1) << 22)
                                ? ws.capacity() - ws.mark() - ops - (size_t(1) << 22) : 0;
  const size_t per_col = size_t(P.nch) * M * 4;
  const int64_t cols = int64_t(free_bytes / per_col) / 4 * 4;   // partial rows padded to 4
  int64_t Np = (N + 3) / 4 * 4 <= cols ? N : (cols >= 256 ? cols / 256 * 256 : cols);
  if (Np < 1) return false;
  P.M = M;
  P.N = N;
  P.Kp = Kp;
  P.Np = Np;
  return true;
}
}  // namespace

bool gemm_emu_fits(const Gemm& g, const Arena& ws) {
  EmuPlan P;
  return emu_plan(g, ws, P);
}

bool gemm_emu(const Gemm& g, Arena& ws, cudaStream_t s, int sm_count, int* err) {
  (void)sm_count;
  EmuPlan P;
  if (!emu_plan(g, ws, P)) return false;
  const GOp &a = P.a, &b = P.b;
  const int64_t M = P.M, N = P.N, Kp = P.Kp, Np = P.Np;
  const int nch = P.nch;
  const int* gstart = P.gstart;
  Scope sc(ws);
  const int *ea = nullptr, *eb = nullptr;
  const __nv_bfloat16* As = emu_operand(a, 0, g.a_const, ws, s, &ea);
  const __nv_bfloat16* Bs = emu_operand(b, 1, g.b_const, ws, s, &eb);
  const int64_t ldp = (Np + 3) / 4 * 4;
  float* part = ws.get<float>(size_t(nch) * M * ldp);
  for (int64_t n0 = 0; n0 < N; n0 += Np) {
    const int64_t nw = std::min(Np, N - n0), ldw = (nw + 3) / 4 * 4;
    tc_gemm_emu_launch(As, Bs + n0 * EMU_S * Kp, M, nw, EMU_S, Kp, EMU_CH, gstart, part, ldw, err, s);
    EmuRed r;
    r.P = part;
    r.M = M;
    r.Nw = nw;
    r.ldp = ldw;
    for (int q = 0; q <= TC_EMU_MAX_S; ++q) r.gstart[q] = q <= EMU_S ? gstart[q] : nch;
    r.ea = ea;
    r.eb = eb + n0;
    r.alpha = g.alpha;
    r.beta = g.beta;
    r.C = g.C;
    r.ldc = g.ldc;
    r.n0 = n0;
    r.nb = P.nb;
    r.sCb = P.sCb;
    // 32-bit index arithmetic when every element index, grid stride and batched column fits
    const int64_t blocks = grid_for(M * nw, 256);
    r.small = (M * nw + blocks * 256 < (int64_t(1) << 31) && n0 + nw < (int64_t(1) << 31)) ? 1 : 0;
    r.nw_magic = r.nw_shift = r.nb_magic = r.nb_shift = 0;
    if (r.small) {
      div_inv_consts(nw, &r.nw_magic, &r.nw_shift);
      if (P.nb > 0) div_inv_consts(P.nb, &r.nb_magic, &r.nb_shift);
    }
    k_emu_reduce<<<unsigned(blocks), 256, 0, s>>>(r);
    MLCC_CHECK_LAUNCH();
  }
  return true;
}

}  // namespace mlcc

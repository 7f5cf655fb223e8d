// Tensor-core (tcgen05) GEMMs for the Cholesky-rank doubles contractions of the
// mixed-precision path:  C[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * C[m][n]
// with A, B bfloat16 and K-major (K contiguous, padded to a multiple of 64), the
// accumulator fp32 in tensor memory and C binary64.
//
// A persistent grid of one CTA per SM computes 128 x 256 tiles: TMA (cp.async.bulk.tensor,
// 128-byte swizzle) fills a 4-stage shared-memory ring; one elected thread issues
// tcgen05.mma (kind::f16, M = 128, N = 256, K = 16) into one of two 256-column TMEM
// accumulators and releases stages with tcgen05.commit; four epilogue warps read the other
// accumulator with tcgen05.ld and write C through a shared-memory transpose (coalesced row
// segments) while the next tile's MMAs run. Whole waves of tiles run data-parallel, the
// remaining tiles stream-K (K ranges of equal length per CTA, partial tiles combined after).
// Every mbarrier wait is bounded: on timeout the thread records an error flag and the CTA
// winds down (freeing its TMEM) instead of spinning.
//
// Split precision: an operand x is written as x = x0 + x1 + x2 with bfloat16 pieces; the
// products x0 y0 (MLCC_BF16), + x0 y1 + x1 y0 (MLCC_BF16X3) and + x0 y2 + x1 y1 + x2 y0
// (MLCC_BF16X6) are laid out as extra K segments, so one GEMM of depth S * K sums them.
//
// k_tc_gemm_emu is the same pipeline for the binary64 emulation (MLCC_FP64E, tc_emu.cu):
// exact fp32 sums of integer-digit products, several K chunks per CTA into two TMEM
// accumulators in turn, each chunk drained through shared memory to its own fp32 plane.
// Batches that share A are flattened along N with a batched output-column mapping.
#include "system.cuh"
#include "tc_common.cuh"
#include "fp_convert.cuh"
#include "tc_schedule.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

namespace mlcc {

namespace {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;             // 16 KB
constexpr int B_BYTES = BN * BK * 2;             // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;   // 48 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
// emulation kernel: plus a 32 x 33 fp32 staging block per epilogue warp (coalesced stores)
constexpr int EMU_STAGE_FLOATS = 32 * 33;
constexpr int SMEM_BYTES_EMU = SMEM_BYTES + 4 * EMU_STAGE_FLOATS * 4;
constexpr int THREADS = 192;                     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz
constexpr int EMU_MAX_S = TC_EMU_MAX_S;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false (and flags the error) on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
      atomicExch(err, code);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr & 0x3FFFF) >> 4);
  d |= uint64_t(16 >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;   // stride byte offset
  d |= uint64_t(1) << 46;           // descriptor version
  d |= uint64_t(2) << 61;           // 128-byte swizzle
  return d;
}
// instruction descriptor for kind::f16: bf16 x bf16 -> fp32, both K-major, M = 128, N = BN
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

// Persistent schedule (tc_schedule.h): whole waves of tiles data-parallel, the remainder
// stream-K with its shared tiles fixed up by k_tc_sk_fixup. Each CTA runs its segments
// through two TMEM accumulators in turn, so the epilogue of one tile overlaps the MMAs of
// the next.
struct TcParams {
  int64_t M, N;
  int m_fast;         // 1: consecutive tiles run over M
  int64_t tm, tn;     // tile rows, tile columns
  sched::Plan plan;   // tiles, K blocks, data-parallel tiles, stream-K share
  double* C;
  int64_t ldc;
  double alpha, beta;
  float* slots;     // stream-K partial tiles: [2 G][BM][BN]
  int* err;
  // batched output columns (nb > 0): column b * nb + c of the product lands at
  // C + b * sCb + row * ldc + c (a batch of products that share A, flattened along N)
  int64_t nb, sCb;
};
__device__ __forceinline__ void tile_origin(const TcParams& p, int64_t tile, int64_t& m0, int64_t& n0) {
  int64_t mt, nt;
  if (p.m_fast) {
    mt = tile % p.tm;
    nt = tile / p.tm;
  } else {
    nt = tile % p.tn;
    mt = tile / p.tn;
  }
  m0 = mt * BM;
  n0 = nt * BN;
}
__device__ __forceinline__ double* out_ptr(const TcParams& p, int64_t row, int64_t col) {
  if (p.nb > 0) {
    const int64_t cb = col / p.nb;
    return p.C + cb * p.sCb + row * p.ldc + (col - cb * p.nb);
  }
  return p.C + row * p.ldc + col;
}
// the CTA's segments in order (every role of the CTA walks the same list)
struct TcWalk {
  sched::Walk w;
  __device__ explicit TcWalk(const TcParams& p) { w.start(p.plan, blockIdx.x, gridDim.x); }
  __device__ bool next(const TcParams& p, sched::Seg& sg) { return w.next(p.plan, sg); }
};
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // barriers: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2]; then the TMEM slot
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);   // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer over the K blocks of every segment of this CTA
      TcWalk w(p);
      sched::Seg sg;
      int it = 0;
      bool ok = true;
      while (ok && w.next(p, sg)) {
        int64_t m0, n0;
        tile_origin(p, sg.tile, m0, n0);
        for (int kb = sg.kb0; kb < sg.kb1; ++kb) {
          const int s = it % STAGES;
          if (it >= STAGES && !mbar_wait(empty0 + 8 * s, ((it / STAGES) - 1) & 1, p.err, 1)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = smem_u32(smem + s * STAGE_BYTES);
          mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
          tma_load_2d(a_dst, &tmA, full0 + 8 * s, kb * BK, int(m0));
          tma_load_2d(a_dst + A_BYTES, &tmB, full0 + 8 * s, kb * BK, int(n0));
          ++it;
        }
      }
      // drain: the copies this thread issued land before the CTA can exit
      for (int j = max(0, it - STAGES); j < it; ++j) mbar_wait(full0 + 8 * (j % STAGES), (j / STAGES) & 1, p.err, 4);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: segment u accumulates into TMEM columns (u & 1) * BN
      constexpr uint32_t idesc = instr_desc();
      TcWalk w(p);
      sched::Seg sg;
      int it = 0, u = 0;
      bool ok = true;
      while (ok && w.next(p, sg)) {
        const int b = u & 1;
        // the epilogue has drained segment u - 2 from this accumulator
        if (u >= 2 && !mbar_wait(acce0 + 8 * b, ((u >> 1) - 1) & 1, p.err, 5)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + uint32_t(b * BN);
        for (int kb = sg.kb0; kb < sg.kb1; ++kb) {
          const int s = it % STAGES;
          if (!mbar_wait(full0 + 8 * s, (it / STAGES) & 1, p.err, 2)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_addr = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t ad = smem_desc(a_addr), bd = smem_desc(a_addr + A_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint32_t acc = (kb > sg.kb0 || k > 0) ? 1u : 0u;
            // advance 16 bf16 (32 bytes) along K inside the swizzled 128-byte rows
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tmem),
                "l"(ad + uint64_t(2 * k)), "l"(bd + uint64_t(2 * k)), "r"(idesc), "r"(acc));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                       : "memory");
          ++it;
        }
        if (ok)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(accf0 + 8 * b)
                       : "memory");
        ++u;
      }
    }
  } else {
    // epilogue: warps 2..5 own TMEM lanes 32*(warp % 4) .. +31. Each 32 x 32 block of the
    // accumulator goes through shared memory (lane = row when read from TMEM, lane = column
    // when stored), so that every warp store writes 32 consecutive elements of one row
    const int q = warp & 3;
    float* stg = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256) + q * EMU_STAGE_FLOATS;
    TcWalk w(p);
    sched::Seg sg;
    int u = 0;
    while (w.next(p, sg)) {
      const int b = u & 1;
      if (!mbar_wait(accf0 + 8 * b, (u >> 1) & 1, p.err, 3)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int64_t m0, n0;
      tile_origin(p, sg.tile, m0, n0);
      const int64_t rbase = m0 + 32 * q;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + (uint32_t(32 * q) << 16) + uint32_t(b * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        if (sg.slot >= 0) {
          // a share of a stream-K tile: the whole 32 x 32 block into the CTA's slot
          float* dst = p.slots + (int64_t(sg.slot) * BM + 32 * q) * BN + c0 + lane;
          for (int i = 0; i < 32; ++i) dst[int64_t(i) * BN] = stg[i * 33 + lane];
        } else {
          const int64_t col = n0 + c0 + lane;
          const int64_t left = p.M - rbase;
          const int nrow = left <= 0 ? 0 : (left >= 32 ? 32 : int(left));
          if (col < p.N && nrow > 0) {
            double* cp = out_ptr(p, rbase, col);   // rows of the column are ldc apart
            if (p.beta == 0.0) {
              for (int i = 0; i < nrow; ++i) cp[int64_t(i) * p.ldc] = p.alpha * double(stg[i * 33 + lane]);
            } else {
              // independent loads of C first, so their latencies overlap
              double cv[32];
#pragma unroll
              for (int i = 0; i < 32; ++i) cv[i] = i < nrow ? cp[int64_t(i) * p.ldc] : 0.0;
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (i < nrow) cp[int64_t(i) * p.ldc] = p.alpha * double(stg[i * 33 + lane]) + p.beta * cv[i];
            }
          }
        }
        __syncwarp();
      }
      // this warp has read the accumulator: the MMAs of segment u + 2 may overwrite it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * b);
      ++u;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// C for the stream-K tiles that several CTAs share: block (r, y) takes rows
// [y * FIX_ROWS, (y + 1) * FIX_ROWS) of stream-K tile r and adds the CTAs' fp32 partials in
// CTA order (deterministic), then applies alpha and beta. The CTAs and their slots are
// found once per block.
constexpr int FIX_ROWS = 16;
constexpr int TC_MAX_G = 1024;
__global__ void __launch_bounds__(256) k_tc_sk_fixup(TcParams p) {
  __shared__ int sl[TC_MAX_G];
  __shared__ int ns;
  const int64_t r = blockIdx.x;
  if (threadIdx.x == 0) ns = sched::fixup_slots(p.plan, r, sl, TC_MAX_G);
  __syncthreads();
  const int n = ns;
  if (n == 0) return;
  int64_t m0, n0;
  tile_origin(p, p.plan.dp_tiles + r, m0, n0);
  const int i0 = int(blockIdx.y) * FIX_ROWS;
  for (int t = threadIdx.x; t < FIX_ROWS * BN; t += blockDim.x) {
    const int i = i0 + t / BN, jc = t % BN;
    const int64_t row = m0 + i, col = n0 + jc;
    if (row >= p.M || col >= p.N) continue;
    double v = 0.0;
    for (int q = 0; q < n; ++q) v += double(p.slots[(int64_t(sl[q]) * BM + i) * BN + jc]);
    double* cp = out_ptr(p, row, col);
    *cp = (p.beta == 0.0) ? p.alpha * v : p.alpha * v + p.beta * *cp;
  }
}

// ---------------------------------------------------------------------------------
// Emulation mode (binary64 from integer digits, tc_emu.cu): the operands hold S digit
// slices of kbp K blocks each; digit pair (i, j) belongs to group g = i + j. Chunk z of
// group g (gstart[g] <= z < gstart[g + 1]) sums at most ch K blocks of the pairs
// (i, g - i), concatenated in i, into the fp32 plane part32[z][M][ldp]. Each CTA takes
// chunks [z0, z0 + cpb) of one 128 x 256 tile and accumulates them into two TMEM
// accumulators in turn: the epilogue drains chunk c while the MMAs of chunk c + 1 run.
struct EmuParams {
  int64_t M, N;
  int S, kbp, ch, nch, cpb;
  int gstart[EMU_MAX_S + 1];
  float* part32;
  int64_t ldp;
  int* err;
};
__device__ __forceinline__ void emu_chunk(const EmuParams& p, int z, int& grp, int& loc0, int& nkb) {
  grp = 0;
  while (grp + 1 < p.S && z >= p.gstart[grp + 1]) ++grp;
  loc0 = (z - p.gstart[grp]) * p.ch;
  nkb = max(0, min(p.ch, (grp + 1) * p.kbp - loc0));
}
__global__ void __launch_bounds__(THREADS, 1)
k_tc_gemm_emu(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EmuParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // barriers: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2]; then the TMEM slot
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = int64_t(blockIdx.x) * BM, n0 = int64_t(blockIdx.y) * BN;
  const int z0 = int(blockIdx.z) * p.cpb;
  const int nc = max(0, min(p.nch, z0 + p.cpb) - z0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);   // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer over the K blocks of every chunk of this CTA
      int it = 0;
      bool ok = true;
      for (int c = 0; c < nc && ok; ++c) {
        int grp, loc0, nkb;
        emu_chunk(p, z0 + c, grp, loc0, nkb);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % STAGES;
          if (it >= STAGES && !mbar_wait(empty0 + 8 * s, ((it / STAGES) - 1) & 1, p.err, 11)) {
            ok = false;
            break;
          }
          // group-local block -> digit pair (i, grp - i) and block kk inside the slice
          const int loc = loc0 + kb, i = loc / p.kbp, kk = loc - i * p.kbp;
          const uint32_t a_dst = smem_u32(smem + s * STAGE_BYTES);
          mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
          tma_load_2d(a_dst, &tmA, full0 + 8 * s, (i * p.kbp + kk) * BK, int(m0));
          tma_load_2d(a_dst + A_BYTES, &tmB, full0 + 8 * s, ((grp - i) * p.kbp + kk) * BK, int(n0));
          ++it;
        }
      }
      // drain: the copies this thread issued land before the CTA can exit
      for (int j = max(0, it - STAGES); j < it; ++j) mbar_wait(full0 + 8 * (j % STAGES), (j / STAGES) & 1, p.err, 14);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: chunk c accumulates into TMEM columns (c & 1) * BN
      constexpr uint32_t idesc = instr_desc();
      int it = 0;
      bool ok = true;
      for (int c = 0; c < nc && ok; ++c) {
        const int b = c & 1;
        // the epilogue has drained chunk c - 2 from this accumulator
        if (c >= 2 && !mbar_wait(acce0 + 8 * b, ((c >> 1) - 1) & 1, p.err, 15)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int grp, loc0, nkb;
        emu_chunk(p, z0 + c, grp, loc0, nkb);
        const uint32_t acc_tmem = tmem + uint32_t(b * BN);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % STAGES;
          if (!mbar_wait(full0 + 8 * s, (it / STAGES) & 1, p.err, 12)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_addr = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t ad = smem_desc(a_addr), bd = smem_desc(a_addr + A_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tmem),
                "l"(ad + uint64_t(2 * k)), "l"(bd + uint64_t(2 * k)), "r"(idesc), "r"(acc));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                       : "memory");
          ++it;
        }
        if (ok)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(accf0 + 8 * b)
                       : "memory");
      }
    }
  } else {
    // epilogue: warps 2..5 own TMEM lanes 32*(warp % 4) .. +31; each 32 x 32 block goes
    // through shared memory so that every warp store writes 32 consecutive floats of a row
    const int q = warp & 3;
    float* stg = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256) + q * EMU_STAGE_FLOATS;
    const int64_t rbase = m0 + 32 * q;
    for (int c = 0; c < nc; ++c) {
      const int b = c & 1;
      if (!mbar_wait(accf0 + 8 * b, (c >> 1) & 1, p.err, 13)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* plane = p.part32 + int64_t(z0 + c) * p.M * p.ldp;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + (uint32_t(32 * q) << 16) + uint32_t(b * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // lane = row of the block: stage it, then lane = column: store row by row
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int64_t col = n0 + c0 + lane;
        if (col < p.N) {
          for (int i = 0; i < 32; ++i) {
            const int64_t row = rbase + i;
            if (row < p.M) plane[row * p.ldp + col] = stg[i * 33 + lane];
          }
        }
        __syncwarp();
      }
      // this warp has read the accumulator: the MMAs of chunk c + 2 may overwrite it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * b);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// ---------------------------------------------------------------------------------
// operand preparation: binary64 -> bfloat16 pieces, K-major, K padded to Kp, S segments
struct SplitPattern {
  int S;
  int a[6];
  int b[6];
};
__host__ __device__ inline SplitPattern pattern(int precision) {
  SplitPattern p{};
  if (precision == MLCC_BF16X6) {
    p.S = 6;
    const int a[6] = {0, 0, 1, 0, 1, 2}, b[6] = {0, 1, 0, 2, 1, 0};
    for (int i = 0; i < 6; ++i) { p.a[i] = a[i]; p.b[i] = b[i]; }
  } else if (precision == MLCC_BF16X3) {
    p.S = 3;
    const int a[3] = {0, 0, 1}, b[3] = {0, 1, 0};
    for (int i = 0; i < 3; ++i) { p.a[i] = a[i]; p.b[i] = b[i]; }
  } else {
    p.S = 1;
    p.a[0] = 0;
    p.b[0] = 0;
  }
  return p;
}
// x = x0 + x1 + x2 with bfloat16 pieces of x rounded to binary32 (24 bits: the three
// 8-bit pieces hold all of it). The rounding and the pieces use integer and binary32
// operations only: on GB300 the binary64 pipe would bound these conversion kernels.
__device__ __forceinline__ void split3(double x, __nv_bfloat16 out[3]) {
  const float xf = d2f_rn_bits(x);
  const __nv_bfloat16 h0 = __float2bfloat16_rn(xf);
  const float r1 = xf - __bfloat162float(h0);   // exact: h0 is within 2^-9 of xf
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h1);   // exact for the same reason
  out[0] = h0;
  out[1] = h1;
  out[2] = __float2bfloat16_rn(r2);
}
struct CvtArgs {
  int64_t rows, K, Kp;   // destination rows, true K, padded K
  int S;
  int piece[6];          // split piece per segment
};
// dst[r][s*Kp + k] = piece_s(src(r, k)); transposed source: src(r, k) = src[k * ld + r]
__global__ void k_cvt_transpose(const double* src, int64_t ld, CvtArgs a, __nv_bfloat16* dst) {
  __shared__ double tile[32][33];
  const int64_t r0 = int64_t(blockIdx.x) * 32, k0 = int64_t(blockIdx.y) * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t k = k0 + y, r = r0 + threadIdx.x;
    tile[y][threadIdx.x] = (k < a.K && r < a.rows) ? src[k * ld + r] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, k = k0 + threadIdx.x;
    if (r >= a.rows || k >= a.Kp) continue;
    __nv_bfloat16 pc[3];
    split3(tile[threadIdx.x][y], pc);
    for (int s = 0; s < a.S; ++s) dst[r * (a.S * a.Kp) + s * a.Kp + k] = pc[a.piece[s]];
  }
}
// dst[r][s*Kp + k] = piece_s(src[r * ld + k])  (u_mode: 2 c[r][k] - c[r'][k'] with the
// occupied indices of the pair (r, k) = (ai, bj) exchanged, u = 2c - c(i <-> j))
__global__ void k_cvt_direct(const double* src, int64_t ld, CvtArgs a, int u_mode, int sv, int so,
                             __nv_bfloat16* dst) {
  const int64_t total = a.rows * a.Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / a.Kp, k = t - r * a.Kp;
    double v = 0.0;
    if (k < a.K) {
      v = src[r * ld + k];
      if (u_mode) {
        const int aa = int(r / so), i = int(r - int64_t(aa) * so);
        const int b = int(k / so), j = int(k - int64_t(b) * so);
        v = 2.0 * v - src[(int64_t(aa) * so + j) * ld + int64_t(b) * so + i];
      }
    }
    __nv_bfloat16 pc[3];
    split3(v, pc);
    for (int s = 0; s < a.S; ++s) dst[r * (a.S * a.Kp) + s * a.Kp + k] = pc[a.piece[s]];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn) throw Error(MLCC_E_CUDA, "cuTensorMapEncodeTiled is not available");
  return fn;
}

void make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t kp, int box_rows) {
  MLCC_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0, "TMA base address must be 16-byte aligned");
  MLCC_REQUIRE((kp * 2) % 16 == 0, "TMA row stride must be a multiple of 16 bytes");
  cuuint64_t dims[2] = {cuuint64_t(kp), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(kp * 2)};
  cuuint32_t box[2] = {cuuint32_t(BK), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = get_encode()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(MLCC_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
}
}  // namespace


static void ensure_smem_attr() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES_EMU);
  });
  MLCC_CUDA(e);
}

void tc_gemm_emu_launch(const __nv_bfloat16* A, const __nv_bfloat16* B, int64_t M, int64_t N, int S,
                        int64_t Kp, int ch, const int* gstart, float* part, int64_t ldp, int* err,
                        cudaStream_t s) {
  MLCC_REQUIRE(S >= 1 && S <= EMU_MAX_S && Kp % BK == 0 && ch >= 1, "tc_gemm_emu: bad slicing");
  MLCC_REQUIRE(M < (int64_t(1) << 31) && N < (int64_t(1) << 31), "tc_gemm_emu: size too large");
  MLCC_REQUIRE(ldp % 4 == 0 && ldp >= N, "tc_gemm_emu: partial rows must be padded to 4");
  const int nch = gstart[S];
  MLCC_REQUIRE(nch >= 1, "tc_gemm_emu: no chunks");
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_tc_gemm_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES_EMU);
  });
  MLCC_CUDA(attr);
  CUtensorMap ma, mb;
  make_map(&ma, A, M, S * Kp, BM);
  make_map(&mb, B, N, S * Kp, BN);
  EmuParams p;
  p.M = M;
  p.N = N;
  p.S = S;
  p.kbp = int(Kp / BK);
  p.ch = ch;
  p.nch = nch;
  const int64_t tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  // chunks per CTA: enough CTAs for two waves, at most 8 chunks each
  const int64_t tiles = tm * tn;
  int cpb = int(std::max<int64_t>(1, std::min<int64_t>(8, (tiles * nch) / (2 * 152))));
  p.cpb = cpb;
  for (int g = 0; g <= EMU_MAX_S; ++g) p.gstart[g] = g <= S ? gstart[g] : nch;
  p.part32 = part;
  p.ldp = ldp;
  p.err = err;
  const int64_t nz = (nch + cpb - 1) / cpb;
  MLCC_REQUIRE(tn < 65536 && nz < 65536, "tc_gemm_emu: grid too large");
  const dim3 grid{unsigned(tm), unsigned(tn), unsigned(nz)};
  k_tc_gemm_emu<<<grid, THREADS, SMEM_BYTES_EMU, s>>>(ma, mb, p);
  MLCC_CHECK_LAUNCH();
}

// Bytes of workspace tc_gemm takes for its stream-K partial tiles.
size_t tc_gemm_ws_bytes(int sm_count) { return size_t(2) * std::max(sm_count, 1) * BM * BN * 4 + 256; }

// C = alpha A B^T + beta C for bf16 K-major operands A [M][Kt], B [N][Kt] (Kt = S * Kp),
// on a persistent grid of one CTA per SM (the schedule above TcParams).
void tc_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int64_t M, int64_t N, int64_t Kt,
             double* C, int64_t ldc, double alpha, double beta, int* err, bool m_fast, int sm_count,
             Arena& ws, cudaStream_t s, int64_t nb, int64_t sCb) {
  MLCC_REQUIRE(Kt % BK == 0 && Kt > 0, "tc_gemm: K must be a positive multiple of 64");
  MLCC_REQUIRE(M > 0 && N > 0 && M < (int64_t(1) << 31) && N < (int64_t(1) << 31), "tc_gemm: bad size");
  ensure_smem_attr();
  CUtensorMap ma, mb;
  make_map(&ma, A, M, Kt, BM);
  make_map(&mb, B, N, Kt, BN);
  TcParams p;
  p.M = M;
  p.N = N;
  p.m_fast = m_fast ? 1 : 0;
  p.tm = (M + BM - 1) / BM;
  p.tn = (N + BN - 1) / BN;
  const int64_t tiles = p.tm * p.tn;
  const int64_t G = std::min(std::max(sm_count, 1), TC_MAX_G);
  p.plan = sched::plan(tiles, Kt / BK, G);
  const int64_t grid = p.plan.grid;
  p.C = C;
  p.ldc = ldc;
  p.alpha = alpha;
  p.beta = beta;
  p.err = err;
  p.nb = nb;
  p.sCb = sCb;
  p.slots = p.plan.sk_iters > 0 ? ws.get<float>(size_t(2) * G * BM * BN) : nullptr;
  k_tc_gemm<<<unsigned(grid), THREADS, SMEM_BYTES_EMU, s>>>(ma, mb, p);
  MLCC_CHECK_LAUNCH();
  if (p.plan.sk_iters > 0) {
    k_tc_sk_fixup<<<dim3(unsigned(tiles - p.plan.dp_tiles), BM / FIX_ROWS), 256, 0, s>>>(p);
    MLCC_CHECK_LAUNCH();
  }
}

void cvt_operand(const double* src, int64_t ld, int64_t rows, int64_t K, bool transpose, bool u_mode,
                 int sv, int so, int precision, bool side_a, __nv_bfloat16* dst, cudaStream_t s) {
  SplitPattern pt = pattern(precision);
  CvtArgs a;
  a.rows = rows;
  a.K = K;
  a.Kp = pad64(K);
  a.S = pt.S;
  for (int i = 0; i < pt.S; ++i) a.piece[i] = side_a ? pt.a[i] : pt.b[i];
  if (transpose) {
    dim3 blk(32, 8), grd(unsigned((rows + 31) / 32), unsigned((a.Kp + 31) / 32));
    k_cvt_transpose<<<grd, blk, 0, s>>>(src, ld, a, dst);
  } else {
    const int64_t total = rows * a.Kp;
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 32768)));
    k_cvt_direct<<<blocks, 256, 0, s>>>(src, ld, a, u_mode ? 1 : 0, sv, so, dst);
  }
  MLCC_CHECK_LAUNCH();
}

int split_segments(int precision) { return pattern(precision).S; }

namespace {
// K contiguous in the source: one thread per destination element, kk fastest
__global__ void k_gop_direct(GOp o, __nv_bfloat16* dst) {
  const int64_t total = o.R * o.Kp;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = t / o.Kp, kk = t - r * o.Kp;
    __nv_bfloat16 pc[3];
    split3(gop_load(o, r, kk), pc);
    for (int s2 = 0; s2 < o.S; ++s2) dst[r * (o.S * o.Kp) + s2 * o.Kp + kk] = pc[o.piece[s2]];
  }
}
// rows contiguous in the source: 32 x 32 tiles through shared memory
__global__ void k_gop_tr(GOp o, __nv_bfloat16* dst) {
  __shared__ double tile[32][33];
  const int64_t r0 = int64_t(blockIdx.x) * 32, k0 = int64_t(blockIdx.y) * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) tile[y][threadIdx.x] = gop_load(o, r0 + threadIdx.x, k0 + y);
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, kk = k0 + threadIdx.x;
    if (r >= o.R || kk >= o.Kp) continue;
    __nv_bfloat16 pc[3];
    split3(tile[threadIdx.x][y], pc);
    for (int s2 = 0; s2 < o.S; ++s2) dst[r * (o.S * o.Kp) + s2 * o.Kp + kk] = pc[o.piece[s2]];
  }
}
void convert_gop(GOp o, __nv_bfloat16* dst, cudaStream_t s) {
  if (!o.tr) {
    const int64_t total = o.R * o.Kp;
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 32768)));
    k_gop_direct<<<blocks, 256, 0, s>>>(o, dst);
  } else {
    MLCC_REQUIRE((o.R + 31) / 32 < (int64_t(1) << 31) && (o.Kp + 31) / 32 < 65536, "convert: grid");
    dim3 blk(32, 8), grd(unsigned((o.R + 31) / 32), unsigned((o.Kp + 31) / 32));
    k_gop_tr<<<grd, blk, 0, s>>>(o, dst);
  }
  MLCC_CHECK_LAUNCH();
}
}  // namespace

void operand_cache_set_ranges(OperandCache* c, const std::vector<std::pair<const char*, size_t>>& r) {
  if (c) c->ranges = r;
}
OperandCache* operand_cache_new() { return new OperandCache(); }
void operand_cache_clear(OperandCache* c) {
  if (!c) return;
  for (void* b : c->blocks) cudaFree(b);
  c->blocks.clear();
  c->entries.clear();
  c->perms.clear();
}
void operand_cache_free(OperandCache* c) {
  operand_cache_clear(c);
  delete c;
}
// converted operand, from the cache when the operand is marked constant
static const __nv_bfloat16* get_operand(const GOp& o, int side, bool cacheable, Arena& ws, cudaStream_t s) {
  OperandCache* c = lowp_cache();
  if (c && !(cacheable || c->constant(o.base))) c = nullptr;
  const size_t bytes = size_t(o.R) * o.S * o.Kp * 2;
  if (!c) {
    __nv_bfloat16* d = ws.get<__nv_bfloat16>(size_t(o.R) * o.S * o.Kp);
    convert_gop(o, d, s);
    return d;
  }
  auto key = std::make_tuple(static_cast<const void*>(o.base), o.R, o.Mrow, o.sRow, o.Ktot, o.Kblk, o.sK, o.ld,
                             o.tr, o.S * 16 + o.piece[o.S > 1 ? 1 : 0], side);
  for (auto& e : c->entries)
    if (e.key == key) return e.p;
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    __nv_bfloat16* d = ws.get<__nv_bfloat16>(size_t(o.R) * o.S * o.Kp);
    convert_gop(o, d, s);
    return d;
  }
  c->blocks.push_back(mem);
  auto* d = static_cast<__nv_bfloat16*>(mem);
  convert_gop(o, d, s);
  c->entries.push_back({key, d});
  return d;
}

// A binary64 GEMM (the Gemm of internal.cuh) on the tensor cores. Supported: a single
// product, a batch reduction (batches concatenated along K), and a batch with a shared B
// whose outputs are stacked rows (batches concatenated along M). Returns false (and does
// nothing) for other shapes or when the workspace is too small.
bool gemm_tc(const Gemm& g, int precision, Arena& ws, cudaStream_t s, int sm_count, int* err) {
  if (precision == MLCC_FP64E) return gemm_emu(g, ws, s, sm_count, err);
  // a batch sharing B with stacked outputs flattens along M; a batch sharing A flattens
  // along N (batched output columns)
  const bool batched = !g.reduce && g.batch > 1;
  const bool flatten = batched && g.sB == 0 && g.sC == g.M * g.ldc;
  const bool flat_n = batched && !flatten && g.sA == 0;
  if (batched && !flatten && !flat_n) return false;
  const int64_t M = flatten ? g.M * g.batch : g.M;
  const int64_t Ktot = g.reduce ? g.K * g.batch : g.K;
  const int64_t N = flat_n ? g.N * g.batch : g.N;
  const SplitPattern pt = pattern(precision);
  const int64_t Kp = pad64(Ktot), Kt = pt.S * Kp;
  const size_t need = size_t(M + N) * Kt * 2 + 4 * 256 + tc_gemm_ws_bytes(sm_count);
  if (ws.mark() + need + (size_t(1) << 22) > ws.capacity()) return false;
  Scope sc(ws);
  GOp a{};
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
  a.S = pt.S;
  for (int i = 0; i < pt.S; ++i) a.piece[i] = pt.a[i];
  GOp b = a;
  b.base = g.B;
  b.R = N;
  b.Mrow = flat_n ? g.N : N;
  b.sRow = flat_n ? g.sB : 0;
  b.sK = g.reduce ? g.sB : 0;
  b.ld = g.ldb;
  b.tr = g.tb ? 0 : 1;
  for (int i = 0; i < pt.S; ++i) b.piece[i] = pt.b[i];
  const __nv_bfloat16* Abf = get_operand(a, 0, g.a_const, ws, s);
  const __nv_bfloat16* Bbf = get_operand(b, 1, g.b_const, ws, s);
  tc_gemm(Abf, Bbf, M, N, Kt, g.C, g.ldc, g.alpha, g.beta, err, true, sm_count, ws, s, flat_n ? g.N : 0,
          flat_n ? g.sC : 0);
  return true;
}

// The two rank GEMMs of sigma in low precision.
//   outer: C[dS][dS] = A^T B   with A, B [nj][dS] binary64 (A = the cached Lai)
//   inner: C[nj][dS] = A B     with A [nj][dS] (the cached Lov), B [dS][dS] = u(c) built here
void rank_gemm_lowp(mlcc_system* S, bool outer, const double* A, const double* B, double* C,
                    double alpha, double beta, int precision, bool b_is_u_source) {
  cudaStream_t s = S->ctx->stream;
  const int64_t dS = S->dS, nj = S->nj;
  const int seg = split_segments(precision);
  Scope sc(S->ws);
  if (outer) {
    const int64_t Kp = pad64(nj), Kt = seg * Kp;
    const __nv_bfloat16* Abf = nullptr;
    if (S->lowp_prec == precision && S->lai_bf) {
      Abf = S->lai_bf;
    } else {
      __nv_bfloat16* t = S->ws.get<__nv_bfloat16>(size_t(dS) * Kt);
      cvt_operand(A, dS, dS, nj, true, false, S->sv, S->so, precision, true, t, s);
      Abf = t;
    }
    __nv_bfloat16* Bbf = S->ws.get<__nv_bfloat16>(size_t(dS) * Kt);
    cvt_operand(B, dS, dS, nj, true, false, S->sv, S->so, precision, false, Bbf, s);
    timed(S, "rank_gemm_tc", 2.0 * double(dS) * double(dS) * double(nj),
          [&] { tc_gemm(Abf, Bbf, dS, dS, Kt, C, dS, alpha, beta, S->tc_err, false, S->ctx->sm_count, S->ws, s, 0, 0); });
  } else {
    const int64_t Kp = pad64(dS), Kt = seg * Kp;
    const __nv_bfloat16* Abf = nullptr;
    if (S->lowp_prec == precision && S->lov_bf) {
      Abf = S->lov_bf;
    } else {
      __nv_bfloat16* t = S->ws.get<__nv_bfloat16>(size_t(nj) * Kt);
      cvt_operand(A, dS, nj, dS, false, false, S->sv, S->so, precision, true, t, s);
      Abf = t;
    }
    // B operand K-major: Bbf[n][k] = B[k][n] (B is u(c), symmetric for physical trial
    // vectors; the transposed read keeps the map identical to the binary64 one for any c)
    __nv_bfloat16* Bbf = S->ws.get<__nv_bfloat16>(size_t(dS) * Kt);
    cvt_operand(B, dS, dS, dS, true, false, S->sv, S->so, precision, false, Bbf, s);
    (void)b_is_u_source;
    timed(S, "rank_gemm_tc", 2.0 * double(nj) * double(dS) * double(dS),
          [&] { tc_gemm(Abf, Bbf, nj, dS, Kt, C, dS, alpha, beta, S->tc_err, true, S->ctx->sm_count, S->ws, s, 0, 0); });
  }
}

// bfloat16 copies of the constant operands (Lai, Lov) at the Jacobian ground state
void lowp_prepare(mlcc_system* S, int precision) {
  if (S->dS == 0) return;
  cudaStream_t s = S->ctx->stream;
  const int64_t dS = S->dS, nj = S->nj;
  const int seg = split_segments(precision);
  const size_t need = sizes::lowp_bytes(sys_dims(S), seg);
  if (S->lowp_arena.capacity() < need) S->lowp_arena.reserve(need);
  S->lowp_arena.release(0);
  S->lai_bf = S->lowp_arena.get<__nv_bfloat16>(size_t(dS) * seg * pad64(nj));
  S->lov_bf = S->lowp_arena.get<__nv_bfloat16>(size_t(nj) * seg * pad64(dS));
  cvt_operand(S->Lai, dS, dS, nj, true, false, S->sv, S->so, precision, true, S->lai_bf, s);
  cvt_operand(S->Lov, dS, nj, dS, false, false, S->sv, S->so, precision, true, S->lov_bf, s);
  S->lowp_prec = precision;
}

void check_tc_error(mlcc_system* S) {
  int h = 0;
  MLCC_CUDA(cudaMemcpyAsync(&h, S->tc_err, 4, cudaMemcpyDeviceToHost, S->ctx->stream));
  MLCC_CUDA(cudaStreamSynchronize(S->ctx->stream));
  if (h != 0) {
    MLCC_CUDA(cudaMemsetAsync(S->tc_err, 0, 4, S->ctx->stream));
    throw Error(MLCC_E_TIMEOUT, "tensor-core GEMM: a pipeline wait timed out (code " + std::to_string(h) + ")");
  }
}

}  // namespace mlcc

// The persistent schedule of the tensor-core GEMM (k_tc_gemm): which CTA computes which
// K-block range of which output tile. Plain C++ with host/device qualifiers under nvcc, so
// that the same arithmetic runs in the kernel and in host tests (g++, no GPU).
//
// G CTAs, one per SM. Tiles [0, dp_tiles) run data-parallel: CTA c takes tiles c, c + G,
// ... with whole K. The remaining tiles run stream-K: their K-block iterations, tile after
// tile, are cut into sk_ctas equal ranges, one for each of CTAs 0 .. sk_ctas - 1, taken
// after their data-parallel tiles. A tile that several CTAs share is written by each of
// them as an fp32 partial into a slot of its own (2c for the first tile of the range of
// CTA c, 2c + 1 for its last); a fix-up adds the partials of a tile in CTA order.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define MLCC_SCHED_FN __host__ __device__ __forceinline__
#else
#define MLCC_SCHED_FN inline
#endif

namespace mlcc {
namespace sched {

struct Plan {
  int64_t tiles = 0, kblocks = 0;
  int64_t dp_tiles = 0;   // data-parallel tiles
  int64_t sk_iters = 0;   // K-block iterations of the stream-K tiles
  int sk_ctas = 0;        // CTAs that share them
  int64_t grid = 0;       // CTAs launched
};

// Whole waves data-parallel; the remainder stream-K over at most G CTAs with at least 8
// K blocks each. A remainder of three quarters of a wave or more runs data-parallel too:
// the idle quarter costs less than stream-K's reads, whose K offsets differ between the
// CTAs that share an operand tile, so that L2 does not keep them.
MLCC_SCHED_FN Plan plan(int64_t tiles, int64_t kblocks, int64_t G) {
  Plan p;
  p.tiles = tiles;
  p.kblocks = kblocks;
  p.dp_tiles = tiles / G * G;
  if (4 * (tiles - p.dp_tiles) >= 3 * G) p.dp_tiles = tiles;
  p.sk_iters = (tiles - p.dp_tiles) * kblocks;
  if (p.sk_iters > 0) {
    const int64_t c = p.sk_iters / 8 < G ? p.sk_iters / 8 : G;
    p.sk_ctas = int(c > 1 ? c : 1);
  }
  if (p.dp_tiles > 0) p.grid = p.dp_tiles < G ? p.dp_tiles : G;
  else p.grid = p.sk_ctas;
  return p;
}

// first stream-K iteration of CTA c (sk_iters for the CTAs without a share)
MLCC_SCHED_FN int64_t sk_begin(const Plan& p, int64_t c) {
  return c >= p.sk_ctas ? p.sk_iters : c * p.sk_iters / p.sk_ctas;
}

// one tile's K-block range [kb0, kb1) for a CTA; slot < 0: the whole tile, written to C
struct Seg {
  int64_t tile;
  int kb0, kb1, slot;
};

// the segments of CTA c in order (every role of the CTA walks the same list)
struct Walk {
  int64_t j, it, it0, it1, c, grid;
  MLCC_SCHED_FN void start(const Plan& p, int64_t cta, int64_t grid_size) {
    c = cta;
    grid = grid_size;
    j = cta;
    it0 = sk_begin(p, cta);
    it1 = sk_begin(p, cta + 1);
    it = it0;
  }
  MLCC_SCHED_FN bool next(const Plan& p, Seg& sg) {
    if (j < p.dp_tiles) {
      sg.tile = j;
      sg.kb0 = 0;
      sg.kb1 = int(p.kblocks);
      sg.slot = -1;
      j += grid;
      return true;
    }
    if (it >= it1) return false;
    const int64_t t = it / p.kblocks;
    const int kb0 = int(it - t * p.kblocks);
    const int64_t rest = it1 - it;
    const int kb1 = rest < p.kblocks - kb0 ? kb0 + int(rest) : int(p.kblocks);
    sg.tile = p.dp_tiles + t;
    sg.kb0 = kb0;
    sg.kb1 = kb1;
    sg.slot = (kb0 == 0 && kb1 == p.kblocks) ? -1 : int(2 * c + (it == it0 ? 0 : 1));
    it += kb1 - kb0;
    return true;
  }
};

// The slots holding the partials of stream-K tile r (0 <= r < tiles - dp_tiles), in CTA
// order, into sl[0 .. cap); returns their number, 0 when one CTA had the whole tile.
MLCC_SCHED_FN int fixup_slots(const Plan& p, int64_t r, int* sl, int cap) {
  const int64_t b = r * p.kblocks, e = b + p.kblocks;
  const int64_t G = p.sk_ctas;
  int64_t c = b * G / p.sk_iters;   // the CTA whose range holds iteration b
  while (c + 1 < G && sk_begin(p, c + 1) <= b) ++c;
  while (c > 0 && sk_begin(p, c) > b) --c;
  if (sk_begin(p, c + 1) >= e) return 0;
  int n = 0;
  for (int64_t cc = c; cc < G && n < cap; ++cc) {
    const int64_t beg = sk_begin(p, cc);
    if (beg >= e) break;
    sl[n++] = int(2 * cc + (beg / p.kblocks == r ? 0 : 1));
  }
  return n;
}

}  // namespace sched
}  // namespace mlcc

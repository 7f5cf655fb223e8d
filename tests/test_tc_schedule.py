"""The persistent schedule of the tensor-core GEMM (csrc/tc_schedule.h), compiled on its own
with g++ and walked on the host for many shapes (no GPU). The kernel and its fix-up run the
same functions. Checked for every shape:
  * every K block of every tile is computed by exactly one CTA; data-parallel tiles are
    whole; the grid is at most the SM count;
  * a shared stream-K tile's partials go to slots 2c / 2c + 1 of its CTAs, no slot twice;
  * the fix-up's slot list of each stream-K tile names exactly the CTAs that computed it,
    in CTA order, and their K ranges add up to the whole tile; an unshared tile has none;
  * balance: the K blocks given to any two CTAs differ by at most one tile's worth, or by
    16 where tiles are shorter (a stream-K share is at least 8 K blocks);
  * a remainder of three quarters of a wave or more runs data-parallel, a smaller one
    stream-K with at least 8 K blocks per CTA where there are that many.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_05226_gb300", "csrc")

DRIVER = r"""
#include "tc_schedule.h"
#include <cstdio>
#include <map>
#include <set>
#include <vector>
using namespace mlcc::sched;

static int fail(const char* what, long tiles, long kb, long G) {
  std::printf("FAIL %s tiles=%ld kblocks=%ld G=%ld\n", what, tiles, kb, G);
  return 1;
}

static int check(long tiles, long kb, long G) {
  const Plan p = plan(tiles, kb, G);
  if (p.grid < 1 || p.grid > G || p.sk_ctas > p.grid) return fail("grid", tiles, kb, G);
  const long rem = tiles - tiles / G * G;
  if (4 * rem >= 3 * G) {
    if (p.dp_tiles != tiles) return fail("large remainder not data-parallel", tiles, kb, G);
  } else if (p.dp_tiles != tiles / G * G) {
    return fail("data-parallel tiles", tiles, kb, G);
  }
  if (p.sk_iters >= 8 && p.sk_iters < 8L * p.sk_ctas) return fail("short stream-K share", tiles, kb, G);
  if (p.sk_iters > 0 && p.sk_iters < 8 && p.sk_ctas != 1) return fail("stream-K CTAs", tiles, kb, G);
  std::vector<int> owner(size_t(tiles * kb), -1);
  std::map<int, Seg> slots;
  long lo = -1, hi = -1;
  for (long c = 0; c < p.grid; ++c) {
    Walk w;
    w.start(p, c, p.grid);
    Seg s;
    long mine = 0;
    while (w.next(p, s)) {
      if (s.tile < 0 || s.tile >= tiles || s.kb0 < 0 || s.kb1 > kb || s.kb1 <= s.kb0)
        return fail("segment range", tiles, kb, G);
      if (s.tile < p.dp_tiles && (s.kb0 != 0 || s.kb1 != kb || s.slot != -1))
        return fail("data-parallel tile not whole", tiles, kb, G);
      for (int k = s.kb0; k < s.kb1; ++k) {
        int& o = owner[size_t(s.tile * kb + k)];
        if (o != -1) return fail("K block computed twice", tiles, kb, G);
        o = int(c);
      }
      if (s.slot >= 0) {
        if (s.slot / 2 != c || c >= p.sk_ctas || slots.count(s.slot)) return fail("slot", tiles, kb, G);
        slots[s.slot] = s;
      }
      mine += s.kb1 - s.kb0;
    }
    lo = (lo < 0 || mine < lo) ? mine : lo;
    hi = mine > hi ? mine : hi;
  }
  for (int o : owner)
    if (o < 0) return fail("K block not computed", tiles, kb, G);
  if (hi - lo > (kb > 16 ? kb : 16)) return fail("balance", tiles, kb, G);
  for (long r = 0; r < tiles - p.dp_tiles; ++r) {
    const long t = p.dp_tiles + r;
    std::set<int> ctas;
    for (long k = 0; k < kb; ++k) ctas.insert(owner[size_t(t * kb + k)]);
    std::vector<int> sl(2048);
    const int n = fixup_slots(p, r, sl.data(), 2048);
    if (ctas.size() == 1) {
      if (n != 0) return fail("unshared tile with slots", tiles, kb, G);
      continue;
    }
    if (n != int(ctas.size())) return fail("slot count", tiles, kb, G);
    long sum = 0, prev = -1;
    for (int q = 0; q < n; ++q) {
      auto it = slots.find(sl[q]);
      if (it == slots.end() || it->second.tile != t) return fail("slot of another tile", tiles, kb, G);
      if (!ctas.count(sl[q] / 2) || sl[q] / 2 <= prev) return fail("slot order", tiles, kb, G);
      prev = sl[q] / 2;
      sum += it->second.kb1 - it->second.kb0;
    }
    if (sum != kb) return fail("partials do not add up", tiles, kb, G);
  }
  return 0;
}

int main() {
  long cases = 0;
  const long kbs[] = {1, 2, 3, 7, 8, 9, 33, 132};
  const long gs[] = {152, 148, 7, 2, 1};
  for (long G : gs)
    for (long kb : kbs)
      for (long tiles = 1; tiles <= 700; ++tiles) {
        if (check(tiles, kb, G)) return 1;
        ++cases;
      }
  // the three-level workload's shapes: ladder, inner and outer rank GEMMs, block contractions
  const long shapes[][2] = {{308, 921}, {940, 564}, {4418, 120}, {242, 132}, {288, 282}, {1128, 72}};
  for (auto& sh : shapes) {
    if (check(sh[0], sh[1], 152)) return 1;
    ++cases;
  }
  std::printf("ok %ld\n", cases);
  return 0;
}
"""


def test_schedule_covers_every_block_once_and_the_fixup_finds_every_partial(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "sched.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "sched"
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr

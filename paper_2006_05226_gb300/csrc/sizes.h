// Device memory of one MLCC solve, allocation by allocation. Plain C++ (no CUDA): the
// allocation sites size their arenas with these functions, and the footprint query that
// the serving loop admits requests by adds them up, so the two cannot drift apart.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>

namespace mlcc {
namespace sizes {

// Orbital-space sizes of a problem after the level partition (Sec. 2.1).
struct Dims {
  int64_t n = 0, no = 0, nv = 0, nj = 0;   // orbitals, occupied, virtual, Cholesky vectors
  int64_t so = 0, sv = 0;                  // CC2-active occupied / virtual (with CCSD)
  int64_t to = 0, tv = 0;                  // CCSD-active occupied / virtual
  int64_t dS = 0;                          // sv * so
  int64_t nd = 0;                          // dS * dS, doubles per vector
  int64_t nn() const { return n * n; }
  int64_t tl() const { return tv * to * tv * to; }   // CCSD-block doubles
  int64_t vector_len() const { return nv * no + nd; }
};

// From per-orbital levels (0 CCS, 1 CC2, 2 CCSD), occupied orbitals first. Returns false
// for sizes or levels outside their ranges.
inline bool dims_from_levels(int64_t n_mo, int64_t n_occ, int64_t n_chol, const int8_t* level, Dims* d) {
  if (!level || n_mo <= 0 || n_occ <= 0 || n_occ >= n_mo || n_chol <= 0) return false;
  Dims r;
  r.n = n_mo;
  r.no = n_occ;
  r.nv = n_mo - n_occ;
  r.nj = n_chol;
  for (int64_t p = 0; p < n_mo; ++p) {
    const int lev = level[p];
    if (lev < 0 || lev > 2) return false;
    const bool occ = p < n_occ;
    if (lev >= 1) ++(occ ? r.so : r.sv);
    if (lev == 2) ++(occ ? r.to : r.tv);
  }
  r.dS = r.sv * r.so;
  r.nd = r.dS * r.dS;
  *d = r;
  return true;
}

inline int64_t pad64(int64_t k) { return (k + 63) / 64 * 64; }

// Persistent buffers of a system: L, L~, h, h~, F~, eps, Lai, Lov, Z, u, x2 at the Jacobian
// ground state, F_ov, t1, X_Ji, Y_aB, the error flag.
inline size_t persist_bytes(const Dims& d) {
  const int64_t nn = d.nn();
  const int64_t per = d.nj * nn * 2 + 3 * nn + d.n + 3 * d.nj * d.dS + d.nd * 2 + d.dS + d.nv * d.no +
                      d.no * d.so + d.sv * d.nv + 2;
  return size_t(per) * 8 + 96 * 256;
}

// Scratch arena of a system: a sigma evaluation (dressing tangent, three doubles-sized
// arrays, [nj][dS] intermediates), GEMM partials, the einsum engine's permuted operands of
// the CCSD block, plus 2^27 doubles of headroom.
inline size_t ws_bytes(const Dims& d) {
  const int64_t nn = d.nn(), tlen = std::max<int64_t>(d.tl(), 1), tb = d.tv + d.to;
  const int64_t ws = d.nj * nn + 4 * nn + 3 * d.nd + 4 * d.nj * d.dS + 4 * d.dS + d.nj * (d.no * d.no + 2) +
                     64 * tlen + d.tv * d.tv * d.tv * d.tv * 4 + d.nj * (tb * tb) * 4 + (int64_t(1) << 27);
  return size_t(ws) * 8;
}

// Value tensors of the CCSD block kept for the Jacobian (zero without a CCSD level).
inline size_t ccsd_cache_bytes(const Dims& d) {
  if (d.to <= 0 || d.tv <= 0) return 0;
  const int64_t o = d.to, v = d.tv;
  // inputs, the value tensors of one residual, g~_Kcbd, and the ladder operands of the
  // tangent: g~ as [(ab)][(cd)] and X_Kbij
  const int64_t need = d.nj * (v * o + v * v + o * o + o * v) + v * v + o * o + 2 * v * v * v * v +
                       14 * (v * o * v * o) + 4 * (o * o * o * o) + 4 * v * v + 4 * o * o + d.no * v * v * v +
                       d.no * v * o * o;
  return size_t(need) * 8 + 64 * 256;
}

// The ground state's constant ladder operand [(ab) | (Kb) | (KL)][(cd)] in binary64 and one
// converted copy of it with `conv_bytes_per_element` (zero without a CCSD level). It lives
// while the ground state runs.
inline size_t gs_ladder_bytes(const Dims& d, int conv_bytes_per_element) {
  if (d.to <= 0 || d.tv <= 0) return 0;
  const int64_t rows = d.tv * d.tv + d.no * d.tv + d.no * d.no, k = d.tv * d.tv;
  return size_t(rows) * size_t(k) * 8 + size_t(rows) * size_t(pad64(k)) * size_t(std::max(conv_bytes_per_element, 0)) +
         size_t(rows) * 4;
}

// bfloat16 pieces of the constant rank-GEMM operands Lai and Lov in a split precision with
// `seg` pieces per product (zero without CC2-active pairs).
inline size_t lowp_bytes(const Dims& d, int seg) {
  if (d.dS == 0 || seg <= 0) return 0;
  return size_t(d.dS) * seg * pad64(d.nj) * 2 + size_t(d.nj) * seg * pad64(d.dS) * 2 + 4096;
}

// Davidson subspace size: max_subspace, or 8 n_roots when it is 0, and at least 3 n_roots.
inline int davidson_max_subspace(int max_subspace, int n_roots) {
  return std::max(max_subspace > 0 ? max_subspace : 8 * n_roots, 3 * n_roots);
}

// Davidson arena: basis and sigma vectors, Ritz vectors, residuals, collapse scratch and
// three single vectors, each of `dim` binary64 elements (binary32 storage uses half).
inline size_t davidson_bytes(int64_t dim, int max_subspace, int n_roots) {
  const int64_t collapse = 2 * int64_t(n_roots);
  return size_t(dim) * 8 * size_t(2 * int64_t(max_subspace) + 2 * int64_t(n_roots) + 2 * collapse + 3) +
         (size_t(1) << 20);
}

// Allowance for the converted copies of constant GEMM operands (the dressed Cholesky
// vectors, Lai, Lov, Z, u and the ladder's g~_(ab)(cd)) that a system caches while sigma runs on the tensor cores:
// `bytes_per_element` summed over the precisions in use (2 per bfloat16 piece; 16 plus
// exponents for the 8 integer digits of the binary64 emulation). An estimate, not a bound
// the cache enforces.
// Each CCSD-block value tensor that an einsum of the sigma rows reads in another order also
// keeps that binary64 copy (with its converted pieces) in the cache.
inline size_t operand_cache_allowance(const Dims& d, int bytes_per_element) {
  if (bytes_per_element <= 0) return 0;
  const int64_t elems = d.nj * d.nn() + 3 * d.nj * d.dS + d.nd + d.tv * d.tv * d.tv * d.tv;
  const int64_t tb = d.tv + d.to;
  const int64_t perm = (d.to > 0 && d.tv > 0) ? d.nj * tb * tb + 16 * d.tl() + 4 * d.to * d.to * d.to * d.to : 0;
  return size_t(elems) * size_t(bytes_per_element) + size_t(perm) * size_t(8 + bytes_per_element);
}

// cudaMalloc hands out large blocks in 2 MiB pages.
inline size_t round_alloc(size_t b) {
  const size_t page = size_t(2) << 20;
  return b == 0 ? 0 : (b + page - 1) / page * page;
}

}  // namespace sizes
}  // namespace mlcc

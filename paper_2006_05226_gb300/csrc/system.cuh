// The device-side state of one MLCC problem and the steps of its hot path.
#pragma once
#include "internal.cuh"
#include "sizes.h"

#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>

namespace mlcc {

// Value or tangent of a tensor in the forward-mode (dual number) evaluation of the
// residual: sigma = A c = dOmega/dh (x + h c) is the tangent of Omega along c.
struct Dual {
  DT v;   // value
  DT d;   // tangent (d.p == nullptr: zero)
};

enum class Mode { Value, Tangent };

// value tensors of the CCSD block at the Jacobian ground state
struct CCSDCache {
  Arena arena;
  std::vector<double*> slots;
  DT G;   // g~_Kcbd = Lt^J_Kc Lt^J_bd, K over all occupied orbitals, c, b, d CCSD-active
  DT G2;  // g~_acbd as a [(ab)][(cd)] matrix: the constant operand of the ladder tangent
  DT X;   // X_Kbij = sum_cd g~_Kcbd t_cidj, for the dressing part of the ladder tangent
  const char* arena_base() const { return arena.base(); }
  size_t arena_size() const { return arena.capacity(); }
};

struct TCGemm;      // tensor-core GEMM plan (mixed precision)
struct SigmaGraphs; // captured Jacobian transformations (solvers.cu)

}  // namespace mlcc

struct mlcc_system {
  mlcc_ctx* ctx = nullptr;
  int n = 0, no = 0, nv = 0, nj = 0;
  int so = 0, sv = 0, to = 0, tv = 0;
  int64_t dS = 0;          // sv * so
  int64_t nd = 0;          // dS * dS
  std::vector<int32_t> perm;   // internal -> caller orbital
  // semicanonical rotation inside each level's occupied and virtual blocks (internal order):
  // the system's orbital k is sum_k' rot[k' * n + k] (re-ordered input orbital k'); empty
  // when the input Fock matrix was already diagonal inside every level block
  std::vector<double> rot;
  std::vector<double> eps_host;
  // persistent device buffers
  double* L = nullptr;     // [nj][n][n] internal order
  double* h = nullptr;     // [n][n]
  double* eps = nullptr;   // [n]
  // current dressing (value)
  double* Lt = nullptr;    // [nj][n][n]
  double* ht = nullptr;    // [n][n]
  double* Ft = nullptr;    // [n][n]
  double* Lai = nullptr;   // [nj][dS]  Lt[J][no+a][i]
  double* Lov = nullptr;   // [nj][dS]  Lt[J][j][no+c] stored at c*so + j
  double* Z = nullptr;     // [nj][dS]  Z^J_bi = u_(bi)(cj) Lov^J_(cj)
  double* u = nullptr;     // [nd]
  double* Fov = nullptr;   // [dS]      F~[j][no+b] at b*so + j
  double* Xji = nullptr;   // [no][so]  X_Ji of the MLCC2 Jacobian
  double* Yab = nullptr;   // [sv][nv]  Y_aB of the MLCC2 Jacobian
  // Jacobian ground state
  bool prepared = false;
  double* t1gs = nullptr;  // [nv][no]
  double* x2gs = nullptr;  // [nd]
  mlcc::CCSDCache* ccsd = nullptr;
  // mixed precision: bfloat16 pieces of the constant GEMM operands, error flag
  mlcc::Arena lowp_arena;
  __nv_bfloat16* lai_bf = nullptr;
  __nv_bfloat16* lov_bf = nullptr;
  int lowp_prec = -1;
  int* tc_err = nullptr;
  mlcc::OperandCache* opcache = nullptr;   // bfloat16 pieces of Jacobian-constant operands
  mlcc::SigmaGraphs* graphs = nullptr;     // CUDA graphs of sigma (mlcc_options.sigma_graph)
  // ground state with a CCSD level: the undressed integrals of the ladder term as one
  // constant operand [(ab) | (Kb) | (KL)][(cd)] (gs_ladder_build), and its converted copies
  double* gsl = nullptr;
  mlcc::OperandCache* gsl_cache = nullptr;
  // J window of a sharded Jacobian transformation (mlcc_sigma_partial): while set, nj, Lt,
  // Lai, Lov and Z describe the Cholesky vectors [jwin0, jwin0 + nj) only
  bool jwin = false;
  int jwin0 = 0;
  mlcc::Arena persist;     // the buffers above
  mlcc::Arena ws;          // scratch
  int64_t workspace_bytes = 0;
};

namespace mlcc {

// the sizes of a system in the form the allocation-size functions take
inline sizes::Dims sys_dims(const mlcc_system* S) {
  sizes::Dims d;
  d.n = S->n; d.no = S->no; d.nv = S->nv; d.nj = S->nj;
  d.so = S->so; d.sv = S->sv; d.to = S->to; d.tv = S->tv;
  d.dS = S->dS; d.nd = S->nd;
  return d;
}

// steps (all on sys->ctx->stream)
void dress(mlcc_system* S, const double* t1, double* Lt, double* ht);
void dress_tangent(mlcc_system* S, const double* c1, double* dLt, double* dht);
void build_fock(mlcc_system* S, const double* ht, const double* Lt, double* Ft);
void build_fock_tangent(mlcc_system* S, const double* dht, const double* dLt, double* dFt);
void gather_vo(mlcc_system* S, const double* X, double* out);
void gather_ov(mlcc_system* S, const double* X, double* out);
void make_u(mlcc_system* S, const double* x2, double* u);
void omega_eval(mlcc_system* S, const double* t1, const double* x2, bool gs_mode,
                const double* tT, double* x2_out, double* om1, double* om2, double* energy);
void jacobian_prepare(mlcc_system* S, const double* t1, const double* x2);
// parts of sigma_eval: the singles terms driven by c1 always run; the others can be left
// out when their rows are not needed (the rows they write are then left as they were)
enum SigmaParts : unsigned {
  SIGMA_DOUBLES_TO_SINGLES = 1u,   // singles terms driven by c2
  SIGMA_CC2_DOUBLES = 2u,          // the P_S rows (and zero P_T rows before the CCSD part)
  SIGMA_CCSD_ROWS = 4u,            // the P_T rows
  SIGMA_ALL = 7u,
  // with this bit only the terms that sum over the Cholesky vectors run (over the system's
  // current J window); the terms built from F~, X, Y, the cached CCSD value tensors, the
  // orbital energies and the trial doubles alone are left out (a J-sharded evaluation adds
  // them on one rank)
  SIGMA_J_ONLY = 8u
};
void sigma_eval(mlcc_system* S, const double* c, double* sigma, int precision, unsigned parts = SIGMA_ALL);
// rho = A^T l (the adjoint on symmetric doubles) for systems without a CCSD level
void sigma_left_eval(mlcc_system* S, const double* l, double* rho, int precision);
// folded CC2 Jacobian: out = A_eff(omega) c (singles and P_T rows; P_S rows zero), dout (if
// not null) = the singles of dA_eff/domega c; w0, w1, w2: scratch vectors of vector_len
void sigma_eff_eval(mlcc_system* S, const double* c, double omega, double* out, double* dout, int precision,
                    double* w0, double* w1, double* w2);
double lowest_ps_denominator(const mlcc_system* S);
// lowest roots of the folded CC2 Jacobian (folded_solve.cu); MLCC_E_ES_NOCONV if not converged
mlcc_status excited_states_folded(mlcc_system* S, const mlcc_options* opt, double* omega_host, double* r_out,
                                  mlcc_es_info* info);
// c1: in tangent mode the singles trial vector (the tangent of g~_acbd is then formed from
// the cached g~_Kcbd instead of from the Cholesky vectors); in value mode the singles
// amplitudes t1 (or NULL), which the ladder term takes with the operand of gs_ladder_build.
void ccsd_block(mlcc_system* S, Mode mode, const Dual& Lai, const Dual& Lac, const Dual& Lki,
                const Dual& Lkc, const Dual& Fvv, const Dual& Foo, const Dual& t, double* om_out,
                bool cache_values, const double* c1, bool rest = true);
void ccsd_cache_free(mlcc_system* S);
// the constant ladder operand of the ground state (S->gsl) from the undressed Cholesky
// vectors, in the current low-precision routing; false (nothing allocated) without a CCSD
// level or when the device memory is short
bool gs_ladder_build(mlcc_system* S);
void gs_ladder_free(mlcc_system* S);
void sigma_graphs_free(mlcc_system* S);
void rank_gemm_lowp(mlcc_system* S, bool outer, const double* A, const double* B, double* C,
                    double alpha, double beta, int precision, bool b_is_u_source);
void lowp_prepare(mlcc_system* S, int precision);
void check_tc_error(mlcc_system* S);

// kernel-family timing (rank_gemm): wraps a callable with events when enabled
template <class F>
void timed(mlcc_system* S, const char* fam, double flop, F&& f) {
  auto& T = S->ctx->timer;
  // NVTX range named after the kernel family (profilers can filter on it)
  struct Range {
    explicit Range(const char* n) { nvtxRangePushA(n); }
    ~Range() { nvtxRangePop(); }
  } range(fam);
  if (!T.enabled) {
    f();
    return;
  }
  cudaEvent_t a, b;
  T.begin(fam, S->ctx->stream, flop, &a, &b);
  f();
  MLCC_CUDA(cudaEventRecord(b, S->ctx->stream));
}

// Consecutive timed phases of one routine: mark("name") closes the open phase and opens
// the next (kernel-timing family "name"); the destructor closes the last one.
struct PhaseMarks {
  mlcc_system* S;
  cudaEvent_t open_end = nullptr;
  explicit PhaseMarks(mlcc_system* sys) : S(sys) {}
  void close() {
    if (open_end) {
      MLCC_CUDA(cudaEventRecord(open_end, S->ctx->stream));
      open_end = nullptr;
    }
  }
  void mark(const char* fam) {
    close();
    auto& T = S->ctx->timer;
    if (!T.enabled) return;
    cudaEvent_t a;
    T.begin(fam, S->ctx->stream, 0.0, &a, &open_end);
  }
  ~PhaseMarks() {
    if (open_end) cudaEventRecord(open_end, S->ctx->stream);
  }
};

}  // namespace mlcc

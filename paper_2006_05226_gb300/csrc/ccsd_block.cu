// CCSD doubles residual on the CCSD-active orbitals (Appendix A, Omega_aibj of MLCCSD)
// and its tangent (the CCSD rows of sigma = A c), through the pairwise einsum engine.
//
// Readings of the printed equation used here (all indices CCSD-active, X1-basis
// integrals everywhere): Y_aick = g~_kiac - 1/2 t^{ad}_{li} g~_kdlc; the occupied
// Fock-like term is -t^{ab}_{ik} (F~_kj + g~_ldkc u^{dc}_{lj}); P^{ab}_{ij} acts on the
// terms with Y, u and F~ (the first line is symmetric already).
#include "system.cuh"

#include <cstring>
#include <map>
#include <string>

namespace mlcc {

void ccsd_cache_free(mlcc_system* S) {
  delete S->ccsd;
  S->ccsd = nullptr;
}

namespace {

// For "Jpq,Jrs->out" (equal operand index patterns, the same contracted indices in the same
// places): out with the free indices of the first operand exchanged for those of the second
// at the same places, e.g. "Jai,Jbj->aibj" gives "bjai". False for other specs.
bool exchange_spec(const char* spec, std::string& swapped) {
  const char* comma = strchr(spec, ',');
  const char* arrow = strstr(spec, "->");
  if (!comma || !arrow || arrow < comma) return false;
  const std::string a(spec, comma), b(comma + 1, arrow), c(arrow + 2);
  if (a.size() != b.size()) return false;
  std::map<char, char> swap;
  for (size_t k = 0; k < a.size(); ++k) {
    const bool fa = c.find(a[k]) != std::string::npos, fb = c.find(b[k]) != std::string::npos;
    if (fa != fb) return false;
    if (!fa) {
      if (a[k] != b[k]) return false;   // contracted: the same index in the same place
      continue;
    }
    if (a[k] == b[k]) return false;     // a batch index: not a pair exchange
    swap[a[k]] = b[k];
    swap[b[k]] = a[k];
  }
  if (swap.empty()) return false;
  swapped = c;
  for (char& ch : swapped) {
    auto it = swap.find(ch);
    if (it == swap.end()) return false;
    ch = it->second;
  }
  return true;
}

// Value / tangent evaluator. In Value mode tensors get values (persistently when caching);
// in Tangent mode values come back from the cache in creation order and tangents are
// computed by the product rule.
struct Eval {
  mlcc_system* S;
  Mode mode;
  bool cache;
  size_t slot = 0;

  int64_t count(const std::vector<int64_t>& d) {
    int64_t n = 1;
    for (auto x : d) n *= x;
    return n;
  }
  Dual make(const std::vector<int64_t>& dims) {
    Dual x;
    x.v.d = dims;
    x.d.d = dims;
    const size_t n = size_t(count(dims));
    if (mode == Mode::Value) {
      if (cache) {
        x.v.p = S->ccsd->arena.get<double>(n);
        S->ccsd->slots.push_back(x.v.p);
      } else {
        x.v.p = S->ws.get<double>(n);
      }
    } else {
      if (slot >= S->ccsd->slots.size()) throw Error(MLCC_E_STATE, "CCSD cache out of sync");
      x.v.p = S->ccsd->slots[slot++];
      x.d.p = S->ws.get<double>(n);
    }
    return x;
  }
  // input tensor: value from the caller (Value) or from the cache; tangent from the caller.
  // j_indexed: the leading index is the Cholesky index; inside a J window the cached value
  // (over every J) is read from the window's first vector on
  Dual input(const Dual& in, bool j_indexed = false) {
    Dual x = make(in.v.p ? in.v.d : in.d.d);
    if (mode == Mode::Tangent && j_indexed && S->jwin)
      x.v.p += int64_t(S->jwin0) * (count(x.v.d) / std::max<int64_t>(x.v.d[0], 1));
    cudaStream_t s = S->ctx->stream;
    if (mode == Mode::Value) {
      MLCC_CUDA(cudaMemcpyAsync(x.v.p, in.v.p, size_t(x.v.size()) * 8, cudaMemcpyDeviceToDevice, s));
    } else if (in.d.p) {
      MLCC_CUDA(cudaMemcpyAsync(x.d.p, in.d.p, size_t(x.d.size()) * 8, cudaMemcpyDeviceToDevice, s));
    } else {
      x.d.p = nullptr;   // zero tangent
    }
    return x;
  }
  void ein(const char* spec, double alpha, const Dual& A, const Dual& B, double beta, Dual& C) {
    cudaStream_t s = S->ctx->stream;
    if (mode == Mode::Value) {
      einsum(spec, alpha, A.v, B.v, beta, C.v, S->ws, s, S->ctx->sm_count);
      return;
    }
    std::string swapped;
    if (&A == &B && A.d.p && exchange_spec(spec, swapped)) {
      // d(A A) = dA A + A dA, and A dA is dA A with the two operands' index groups
      // exchanged: one product and a permuted copy instead of two products
      Scope sc(S->ws);
      DT T;
      T.d = C.d.d;
      T.p = S->ws.get<double>(size_t(T.size()));
      einsum(spec, alpha, A.d, B.v, 0.0, T, S->ws, s, S->ctx->sm_count);
      const std::string out = std::string(strchr(spec, '>') + 1);
      eperm((out + "->" + out).c_str(), 1.0, T, beta, C.d, s);
      eperm((swapped + "->" + out).c_str(), 1.0, T, 1.0, C.d, s);
      return;
    }
    double b = beta;
    bool wrote = false;
    if (A.d.p) {
      einsum(spec, alpha, A.d, B.v, b, C.d, S->ws, s, S->ctx->sm_count);
      b = 1.0;
      wrote = true;
    }
    if (B.d.p) {
      einsum(spec, alpha, A.v, B.d, b, C.d, S->ws, s, S->ctx->sm_count);
      wrote = true;
    }
    if (!wrote) {
      if (beta == 0.0) fill(C.d.p, C.d.size(), 0.0, s);
      else axpby(C.d.p, C.d.p, C.d.size(), 0.0, beta, s);
    }
  }
  // a value tensor whose tangent is never formed (Tangent mode: the cached value only)
  Dual value_only(const std::vector<int64_t>& dims) {
    if (mode == Mode::Value) return make(dims);
    if (slot >= S->ccsd->slots.size()) throw Error(MLCC_E_STATE, "CCSD cache out of sync");
    Dual x;
    x.v.d = dims;
    x.d.d = dims;
    x.v.p = S->ccsd->slots[slot++];
    return x;
  }
  // C = alpha perm(A) + beta C (linear)
  void perm(const char* spec, double alpha, const Dual& A, double beta, Dual& C) {
    cudaStream_t s = S->ctx->stream;
    if (mode == Mode::Value) eperm(spec, alpha, A.v, beta, C.v, s);
    else eperm(spec, alpha, A.d, beta, C.d, s);
  }
};

// Tangent of the ladder term sum_cd g~_acbd t^{cd}_{ij} along a trial vector (c1, dt):
//   sum_cd g~_acbd dt_cidj  -  sum_K (c_aK X_Kbij + c_bK X_Kaji),
// the second part from d g~_acbd = - c_aK g~_Kcbd - c_bK g~_Kdac and the symmetry of t,
// with X_Kbij = sum_cd g~_Kcbd t_cidj built once at the ground state. The first part is one
// GEMM of [(ab)][(cd)] x [(cd)][(ij)] with the cached g~ as its constant operand (2 v^4 o^2
// flop): the O(o^2 v^4) contraction of the CCSD rows, timed as the "ladder_tc" (split
// bfloat16), "ladder_f64e" or "ladder_f64" family by the precision it runs in.
void ladder_tangent(mlcc_system* S, const DT& dt, const double* c1, DT& om_d) {
  cudaStream_t s = S->ctx->stream;
  const int64_t o = S->to, v = S->tv, no = S->no;
  const CCSDCache& C = *S->ccsd;
  Scope sc(S->ws);
  DT W;
  W.d = {v, v, o, o};
  W.p = S->ws.get<double>(size_t(v * v * o * o));
  if (dt.p) {
    DT dcd;
    dcd.d = {v, v, o, o};
    dcd.p = S->ws.get<double>(size_t(v * v * o * o));
    eperm("cidj->cdij", 1.0, dt, 0.0, dcd, s);
    Gemm g;
    g.M = v * v; g.N = o * o; g.K = v * v;
    g.A = C.G2.p; g.lda = v * v; g.a_const = true;
    g.B = dcd.p; g.ldb = o * o;
    g.C = W.p; g.ldc = o * o;
    const int lp = lowp_precision();   // the precision this GEMM runs in
    timed(S, lp == 0 ? "ladder_f64" : (lp == MLCC_FP64E ? "ladder_f64e" : "ladder_tc"),
          2.0 * double(v * v) * double(v * v) * double(o * o), [&] { gemm_f64(g, S->ws, s, S->ctx->sm_count); });
    eperm("abij->aibj", 1.0, W, 1.0, om_d, s);
  }
  // Y[a][(b i j)] = sum_K c_aK X[K][(b i j)]; c1 rows are the CCSD virtuals, stride no
  Gemm gy;
  gy.M = v; gy.N = v * o * o; gy.K = no;
  gy.A = c1; gy.lda = no;
  gy.B = C.X.p; gy.ldb = v * o * o;
  gy.C = W.p; gy.ldc = v * o * o;
  gemm_f64(gy, S->ws, s, S->ctx->sm_count);
  eperm("abij->aibj", -1.0, W, 1.0, om_d, s);
  eperm("baji->aibj", -1.0, W, 1.0, om_d, s);
}

// The ladder term of the ground-state residual, sum_cd g~_acbd t_cidj, from the undressed
// integrals of gs_ladder_build. With the T1 dressing of the virtual rows,
// L~_ac = L_ac - sum_K t_aK L_Kc (K over every occupied orbital, Sec. 2.1),
//   sum_cd g~_acbd t_cidj = sum_cd g_acbd t_cidj - sum_K t_aK U_Kbij - sum_L t_bL U_Laji
//                           + sum_KL t_aK t_bL W_KLij,
// U_Kbij = sum_cd g_Kcbd t_cidj, W_KLij = sum_cd g_KcLd t_cidj (the third term uses the pair
// symmetry of g and t). The three contractions over (cd) are one GEMM against the stacked
// constant operand, 2 (v^2 + n_o v + n_o^2) v^2 o^2 flop, timed as the "gs_ladder_*"
// family; the rest is O(n_o v^2 o^2).
void ladder_value(mlcc_system* S, const DT& t, const double* t1, DT& om) {
  cudaStream_t s = S->ctx->stream;
  const int sm = S->ctx->sm_count;
  const int64_t o = S->to, v = S->tv, no = S->no, oo = o * o;
  const int64_t rows = v * v + no * v + no * no;
  Scope sc(S->ws);
  DT tcd;
  tcd.d = {v, v, o, o};
  tcd.p = S->ws.get<double>(size_t(v * v * oo));
  eperm("cidj->cdij", 1.0, t, 0.0, tcd, s);
  double* W = S->ws.get<double>(size_t(rows * oo));
  Gemm g;
  g.M = rows; g.N = oo; g.K = v * v;
  g.A = S->gsl; g.lda = v * v; g.a_const = true;
  g.B = tcd.p; g.ldb = oo;
  g.C = W; g.ldc = oo;
  const int lp = lowp_precision();
  timed(S, lp == 0 ? "gs_ladder_f64" : (lp == MLCC_FP64E ? "gs_ladder_f64e" : "gs_ladder_tc"),
        2.0 * double(rows) * double(v * v) * double(oo), [&] { gemm_f64(g, S->ws, s, sm); });
  DT Wg;
  Wg.d = {v, v, o, o};
  Wg.p = W;
  eperm("abij->aibj", 1.0, Wg, 1.0, om, s);
  if (!t1 || no == 0) return;
  // Y[a][(b i j)] = sum_K t_aK U[K][(b i j)]: om -= Y_abij + Y_baji
  DT Y;
  Y.d = {v, v, o, o};
  Y.p = S->ws.get<double>(size_t(v * v * oo));
  Gemm gy;
  gy.M = v; gy.N = v * oo; gy.K = no;
  gy.A = t1; gy.lda = no;
  gy.B = W + v * v * oo; gy.ldb = v * oo;
  gy.C = Y.p; gy.ldc = v * oo;
  gemm_f64(gy, S->ws, s, sm);
  eperm("abij->aibj", -1.0, Y, 1.0, om, s);
  eperm("baji->aibj", -1.0, Y, 1.0, om, s);
  // Z[a][(L i j)] = sum_K t_aK W[K][(L i j)], Q[a][b][(ij)] = sum_L t_bL Z[a][L][(ij)]: om += Q_abij
  double* Z = S->ws.get<double>(size_t(v * no * oo));
  Gemm gz;
  gz.M = v; gz.N = no * oo; gz.K = no;
  gz.A = t1; gz.lda = no;
  gz.B = W + (v * v + no * v) * oo; gz.ldb = no * oo;
  gz.C = Z; gz.ldc = no * oo;
  gemm_f64(gz, S->ws, s, sm);
  DT Q;
  Q.d = {v, v, o, o};
  Q.p = S->ws.get<double>(size_t(v * v * oo));
  Gemm gq;
  gq.M = v; gq.N = oo; gq.K = no;
  gq.A = t1; gq.lda = no; gq.sA = 0;
  gq.B = Z; gq.ldb = oo; gq.sB = no * oo;
  gq.C = Q.p; gq.ldc = oo; gq.sC = v * oo;
  gq.batch = v;
  gemm_f64(gq, S->ws, s, sm);
  eperm("abij->aibj", 1.0, Q, 1.0, om, s);
}

}  // namespace

void gs_ladder_free(mlcc_system* S) {
  if (S->gsl) cudaFree(S->gsl);
  S->gsl = nullptr;
  if (S->gsl_cache) operand_cache_free(S->gsl_cache);
  S->gsl_cache = nullptr;
}

// rows (ab): g_acbd; rows (Kb): g_Kcbd; rows (KL): g_KcLd; columns (cd); all from the
// undressed Cholesky vectors, so the operand holds for every iteration of a ground state
bool gs_ladder_build(mlcc_system* S) {
  gs_ladder_free(S);
  if (S->to <= 0 || S->tv <= 0) return false;
  const int64_t v = S->tv, no = S->no, nj = S->nj, n = S->n, nn = n * n;
  const int64_t rows = v * v + no * v + no * no;
  double* p = nullptr;
  if (cudaMalloc(&p, size_t(rows) * size_t(v * v) * 8) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  S->gsl = p;
  S->gsl_cache = operand_cache_new();
  cudaStream_t s = S->ctx->stream;
  const int sm = S->ctx->sm_count;
  Scope sc(S->ws);
  DT Lac, LKc;
  Lac.d = {nj, v, v};
  Lac.p = S->ws.get<double>(size_t(nj * v * v));
  LKc.d = {nj, no, v};
  LKc.p = S->ws.get<double>(size_t(nj * no * v));
  {
    int64_t dims[3] = {nj, v, v}, ss[3] = {nn, n, 1}, ds[3] = {v * v, v, 1};
    permute_f64(3, dims, S->L + no * n + no, ss, Lac.p, ds, 1.0, 0.0, s);
  }
  {
    int64_t dims[3] = {nj, no, v}, ss[3] = {nn, n, 1}, ds[3] = {no * v, v, 1};
    permute_f64(3, dims, S->L + no, ss, LKc.p, ds, 1.0, 0.0, s);
  }
  DT A1, A2, A3;
  A1.d = {v, v, v, v};
  A1.p = p;
  A2.d = {no, v, v, v};
  A2.p = p + v * v * v * v;
  A3.d = {no, no, v, v};
  A3.p = A2.p + no * v * v * v;
  einsum("Jac,Jbd->abcd", 1.0, Lac, Lac, 0.0, A1, S->ws, s, sm);
  einsum("JKc,Jbd->Kbcd", 1.0, LKc, Lac, 0.0, A2, S->ws, s, sm);
  einsum("JKc,JLd->KLcd", 1.0, LKc, LKc, 0.0, A3, S->ws, s, sm);
  return true;
}

void ccsd_block(mlcc_system* S, Mode mode, const Dual& Lai_in, const Dual& Lac_in,
                const Dual& Lki_in, const Dual& Lkc_in, const Dual& Fvv_in, const Dual& Foo_in,
                const Dual& t_in, double* om_out, bool cache_values, const double* c1, bool rest) {
  if (mode == Mode::Value && cache_values) {
    ccsd_cache_free(S);
    S->ccsd = new CCSDCache();
    // every tensor created below (generous: inputs + 4-index intermediates)
    S->ccsd->arena.reserve(sizes::ccsd_cache_bytes(sys_dims(S)));
  }
  Eval E{S, mode, cache_values};
  cudaStream_t s = S->ctx->stream;
  Dual Lai = E.input(Lai_in, true), Lac = E.input(Lac_in, true), Lki = E.input(Lki_in, true);
  Dual Lkc = E.input(Lkc_in, true);   // in tangent mode the ov block has no tangent (NULL)
  Dual Fvv = E.input(Fvv_in), Foo = E.input(Foo_in), t = E.input(t_in);
  const int64_t o = S->to, v = S->tv;
  const std::vector<int64_t> vovo = {v, o, v, o};

  // X1-basis integrals over the CCSD-active orbitals, g~_pqrs = Lt^J_pq Lt^J_rs. The
  // tangent of g~_acbd is not formed: the ladder term, its only use, has its own tangent
  // (ladder_tangent, through the intermediates cached below)
  if (mode == Mode::Tangent && !c1) throw Error(MLCC_E_STATE, "CCSD tangent without the trial singles");
  // the ground state's residual takes the ladder from the undressed integrals (ladder_value)
  const bool undressed_ladder = mode == Mode::Value && !cache_values && S->gsl && !S->jwin;
  Dual g_acbd;
  if (!undressed_ladder) g_acbd = E.value_only({v, v, v, v});
  if (mode == Mode::Value && !undressed_ladder) E.ein("Jac,Jbd->acbd", 1.0, Lac, Lac, 0.0, g_acbd);
  if (mode == Mode::Value && cache_values) {
    // g~_Kcbd for the tangent above
    const int64_t no = S->no, nj = S->nj, n = S->n, nn = n * n;
    DT LKc;
    LKc.d = {nj, no, v};
    LKc.p = S->ws.get<double>(size_t(nj * no * v));
    int64_t dims[3] = {nj, no, v}, ss[3] = {nn, n, 1}, ds[3] = {no * v, v, 1};
    permute_f64(3, dims, S->Lt + no, ss, LKc.p, ds, 1.0, 0.0, s);
    S->ccsd->G.d = {no, v, v, v};
    S->ccsd->G.p = S->ccsd->arena.get<double>(size_t(no * v * v * v));
    einsum("JKc,Jbd->Kcbd", 1.0, LKc, Lac.v, 0.0, S->ccsd->G, S->ws, s, S->ctx->sm_count);
    // the ladder tangent's operands: g~ as [(ab)][(cd)], X_Kbij = sum_cd g~_Kcbd t_cidj
    S->ccsd->G2.d = {v, v, v, v};
    S->ccsd->G2.p = S->ccsd->arena.get<double>(size_t(v * v * v * v));
    eperm("acbd->abcd", 1.0, g_acbd.v, 0.0, S->ccsd->G2, s);
    S->ccsd->X.d = {no, v, o, o};
    S->ccsd->X.p = S->ccsd->arena.get<double>(size_t(no * v * o * o));
    einsum("Kcbd,cidj->Kbij", 1.0, S->ccsd->G, t.v, 0.0, S->ccsd->X, S->ws, s, S->ctx->sm_count);
  }
  Dual g_kilj = E.make({o, o, o, o});
  E.ein("Jki,Jlj->kilj", 1.0, Lki, Lki, 0.0, g_kilj);
  Dual g_kcld = E.make({o, v, o, v});
  E.ein("Jkc,Jld->kcld", 1.0, Lkc, Lkc, 0.0, g_kcld);
  Dual g_kiac = E.make({o, o, v, v});
  E.ein("Jki,Jac->kiac", 1.0, Lki, Lac, 0.0, g_kiac);
  Dual g_aikc = E.make({v, o, o, v});
  E.ein("Jai,Jkc->aikc", 1.0, Lai, Lkc, 0.0, g_aikc);
  // L~_ldkc = 2 g~_ldkc - g~_lckd
  Dual Lg = E.make({o, v, o, v});
  E.perm("ldkc->ldkc", 2.0, g_kcld, 0.0, Lg);
  E.perm("lckd->ldkc", -1.0, g_kcld, 1.0, Lg);
  // u = 2 t - t(i <-> j)
  Dual u = E.make(vovo);
  E.perm("aibj->aibj", 2.0, t, 0.0, u);
  E.perm("ajbi->aibj", -1.0, t, 1.0, u);

  // first line: g~_aibj + g~_acbd t^{cd}_{ij} + t^{ab}_{kl} (g~_kilj + t^{cd}_{ij} g~_kcld)
  Dual om = E.make(vovo);
  E.ein("Jai,Jbj->aibj", 1.0, Lai, Lai, 0.0, om);
  if (undressed_ladder) ladder_value(S, t.v, c1, om.v);
  else if (mode == Mode::Value) E.ein("acbd,cidj->aibj", 1.0, g_acbd, t, 1.0, om);
  else if (rest) ladder_tangent(S, t.d, c1, om.d);   // built from the cached values over all J
  Dual X = E.make({o, o, o, o});
  E.perm("kilj->kilj", 1.0, g_kilj, 0.0, X);
  E.ein("cidj,kcld->kilj", 1.0, t, g_kcld, 1.0, X);
  E.ein("akbl,kilj->aibj", 1.0, t, X, 1.0, om);

  // C: -1/2 t^{bc}_{kj} Y_aick - t^{bc}_{ki} Y_ajck, Y_aick = g~_kiac - 1/2 t^{ad}_{li} g~_kdlc
  Dual Y = E.make({v, o, v, o});
  E.perm("kiac->aick", 1.0, g_kiac, 0.0, Y);
  E.ein("aldi,kdlc->aick", -0.5, t, g_kcld, 1.0, Y);
  Dual CDE = E.make(vovo);
  E.ein("bkcj,aick->aibj", -0.5, t, Y, 0.0, CDE);
  E.ein("bkci,ajck->aibj", -1.0, t, Y, 1.0, CDE);
  // D: 1/2 u^{bc}_{jk} L~_aikc + 1/4 u^{bc}_{jk} L~_ldkc u^{ad}_{il}
  //    = -1/2 u g~_acki + u g~_aikc + 1/4 u (L~ u)
  E.ein("bjck,kiac->aibj", -0.5, u, g_kiac, 1.0, CDE);
  E.ein("bjck,aikc->aibj", 1.0, u, g_aikc, 1.0, CDE);
  Dual Vd = E.make({v, o, o, v});
  E.ein("aidl,ldkc->aikc", 1.0, u, Lg, 0.0, Vd);
  E.ein("bjck,aikc->aibj", 0.25, u, Vd, 1.0, CDE);
  // E: t^{ac}_{ij} (F~_bc - g~_ldkc u^{bd}_{kl}) - t^{ab}_{ik} (F~_kj + g~_ldkc u^{dc}_{lj})
  Dual Fv = E.make({v, v});
  E.perm("bc->bc", 1.0, Fvv, 0.0, Fv);
  E.ein("ldkc,bkdl->bc", -1.0, g_kcld, u, 1.0, Fv);
  E.ein("aicj,bc->aibj", 1.0, t, Fv, 1.0, CDE);
  Dual Fo = E.make({o, o});
  E.perm("kj->kj", 1.0, Foo, 0.0, Fo);
  E.ein("ldkc,dlcj->kj", 1.0, g_kcld, u, 1.0, Fo);
  E.ein("aibk,kj->aibj", -1.0, t, Fo, 1.0, CDE);
  // P^{ab}_{ij}
  E.perm("aibj->aibj", 1.0, CDE, 1.0, om);
  E.perm("bjai->aibj", 1.0, CDE, 1.0, om);

  const DT& res = (mode == Mode::Value) ? om.v : om.d;
  MLCC_CUDA(cudaMemcpyAsync(om_out, res.p, size_t(res.size()) * 8, cudaMemcpyDeviceToDevice, s));
}

}  // namespace mlcc

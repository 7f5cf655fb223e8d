// CCSD doubles residual on the CCSD-active orbitals (Appendix A, Omega_aibj of MLCCSD)
// and its tangent (the CCSD rows of sigma = A c), through the pairwise einsum engine.
//
// Readings of the printed equation used here (all indices CCSD-active, X1-basis
// integrals everywhere): Y_aick = g~_kiac - 1/2 t^{ad}_{li} g~_kdlc; the occupied
// Fock-like term is -t^{ab}_{ik} (F~_kj + g~_ldkc u^{dc}_{lj}); P^{ab}_{ij} acts on the
// terms with Y, u and F~ (the first line is symmetric already).
#include "system.cuh"

namespace mlcc {

void ccsd_cache_free(mlcc_system* S) {
  delete S->ccsd;
  S->ccsd = nullptr;
}

namespace {

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
  // input tensor: value from the caller (Value) or from the cache; tangent from the caller
  Dual input(const Dual& in) {
    Dual x = make(in.v.p ? in.v.d : in.d.d);
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
  // C = alpha perm(A) + beta C (linear)
  void perm(const char* spec, double alpha, const Dual& A, double beta, Dual& C) {
    cudaStream_t s = S->ctx->stream;
    if (mode == Mode::Value) eperm(spec, alpha, A.v, beta, C.v, s);
    else eperm(spec, alpha, A.d, beta, C.d, s);
  }
};

}  // namespace

void ccsd_block(mlcc_system* S, Mode mode, const Dual& Lai_in, const Dual& Lac_in,
                const Dual& Lki_in, const Dual& Lkc_in, const Dual& Fvv_in, const Dual& Foo_in,
                const Dual& t_in, double* om_out, bool cache_values, const double* c1) {
  if (mode == Mode::Value && cache_values) {
    ccsd_cache_free(S);
    S->ccsd = new CCSDCache();
    // every tensor created below (generous: inputs + 4-index intermediates)
    S->ccsd->arena.reserve(sizes::ccsd_cache_bytes(sys_dims(S)));
  }
  Eval E{S, mode, cache_values};
  cudaStream_t s = S->ctx->stream;
  Dual Lai = E.input(Lai_in), Lac = E.input(Lac_in), Lki = E.input(Lki_in);
  Dual Lkc = E.input(Lkc_in);   // in tangent mode the ov block has no tangent (NULL)
  Dual Fvv = E.input(Fvv_in), Foo = E.input(Foo_in), t = E.input(t_in);
  const int64_t o = S->to, v = S->tv;
  const std::vector<int64_t> vovo = {v, o, v, o};

  // X1-basis integrals over the CCSD-active orbitals, g~_pqrs = Lt^J_pq Lt^J_rs
  Dual g_acbd = E.make({v, v, v, v});
  if (mode == Mode::Tangent && c1) {
    // d g~_acbd = - c_aK g~_Kcbd - c_bK g~_Kdac  (d Lt_ac = - c_aK Lt_Kc, Appendix A's route
    // through an intermediate built once at the ground state instead of N_J v^4 work)
    DT cb;
    cb.p = const_cast<double*>(c1);
    cb.d = {v, int64_t(S->no)};
    DT T1;
    T1.d = {v, v, v, v};
    T1.p = S->ws.get<double>(size_t(v * v * v * v));
    einsum("aK,Kcbd->acbd", -1.0, cb, S->ccsd->G, 0.0, T1, S->ws, s, S->ctx->sm_count);
    eperm("acbd->acbd", 1.0, T1, 0.0, g_acbd.d, s);
    eperm("bdac->acbd", 1.0, T1, 1.0, g_acbd.d, s);
  } else {
    E.ein("Jac,Jbd->acbd", 1.0, Lac, Lac, 0.0, g_acbd);
  }
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
  E.ein("acbd,cidj->aibj", 1.0, g_acbd, t, 1.0, om);
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

/*
 * libmlcc -- multilevel CC2 / CCSD ground state and Jacobian transformation on one GPU.
 *
 * Method: arXiv 2006.05226 (Folkestad, Kjonstad, Goletto, Koch), Sec. 2.1 and Appendix A.
 * Given MO Cholesky vectors L^J_pq (Sec. 2.4, g_pqrs = sum_J L^J_pq L^J_rs), the Fock
 * matrix F_pq of the reduced space (Sec. 2.3, Eq. eff_fock) and a partition of the
 * orbitals into CCS-, CC2- and CCSD-active levels (Sec. 2.1), the library solves the
 * MLCC ground-state equations Omega = 0 and finds the lowest eigenvalues of the Jacobian
 * A = dOmega/dx with a Davidson solver built on sigma = A c.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All floating point is IEEE binary64 unless an entry point says otherwise.
 *  - Matrices are row-major. Cholesky vectors are [n_chol][n_mo][n_mo], symmetric in pq.
 *  - The caller's orbital order must list the n_occ occupied orbitals first.
 *  - Inside a system the orbitals are re-ordered by level: occupied orbitals as
 *    [CCSD, CC2-only, CCS-only], then virtual orbitals in the same level order, each
 *    group in ascending caller index. mlcc_orbital_order() returns that permutation.
 *    Every amplitude, residual and trial vector that crosses the ABI uses this internal
 *    order:
 *        singles  [n_vir][n_occ]                     (A, I): all virtuals x all occupied
 *        doubles  [s_vir][s_occ][s_vir][s_occ]       (a, i, b, j): CC2-active orbitals,
 *                 symmetric under (ai) <-> (bj); the CCSD-active orbitals are the
 *                 leading t_occ / t_vir of each range.
 *    A "vector" is singles followed by doubles, vector_len = n_vir n_occ + (s_vir s_occ)^2.
 *    Doubles amplitudes x parameterise X2 = 1/2 sum x_aibj E_ai E_bj; doubles residuals
 *    and sigma doubles are the coefficients in the same expansion (biorthonormal
 *    projection), so sigma = d Omega / dh along (x + h c) in this storage.
 *  - Three-level model: doubles with all four indices CCSD-active (P_T) obey the CCSD
 *    equation built from P_T amplitudes only; every other CC2-active doubles element
 *    obeys the CC2 equation g~ + eps x = 0 (Appendix A, Eq. mlcc2_omega2); singles and
 *    energy use all doubles. No CCSD level gives MLCC2, CCSD = CC2 gives CCS/CCSD.
 *  - Semicanonical basis (Sec. 2.1-2.2): inside each level's occupied-occupied and
 *    virtual-virtual block the system diagonalises F and rotates the Cholesky vectors
 *    with it (an orbital rotation inside a level leaves the model unchanged). Couplings
 *    of F between levels are kept and enter through F~. With F already diagonal inside
 *    every level block nothing is rotated. Amplitudes and vectors refer to the system's
 *    orbitals: mlcc_orbital_order / mlcc_orbitals give them in terms of the caller's.
 *
 * Memory and errors
 * -----------------
 *  - "_dev" pointers are device pointers on the context's device; "_host" pointers are
 *    host pointers. The caller owns every buffer it passes; the library never frees
 *    caller memory. A system allocates its own device workspace (its size is reported
 *    by mlcc_system_info) and frees it in mlcc_system_destroy.
 *  - Entry points return mlcc_status. No exception, abort or device trap crosses the
 *    ABI. On error mlcc_last_error() returns a thread-local message.
 *  - Work is issued on the context's stream (mlcc_ctx_stream); entry points that return
 *    results to host memory synchronise that stream, device-output entry points do not.
 */
#ifndef MLCC_H
#define MLCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MLCC_OK = 0,
  MLCC_E_ARG = -1,          /* invalid argument, size or partition               */
  MLCC_E_OOM = -2,          /* device allocation failed                          */
  MLCC_E_GS_NOCONV = -3,    /* ground state not converged in max_gs_iter         */
  MLCC_E_ES_NOCONV = -4,    /* excited states not converged in max_es_iter       */
  MLCC_E_COMPLEX_ROOT = -5, /* a wanted Ritz value has a non-zero imaginary part */
  MLCC_E_NAN = -6,          /* NaN or Inf met in a residual or sigma             */
  MLCC_E_TIMEOUT = -7,      /* a bounded wait inside a tensor-core kernel expired
                               (about 2 s); the kernel stopped, freed its tensor
                               memory and left the context usable                */
  MLCC_E_CUDA = -8,         /* a CUDA runtime call failed                        */
  MLCC_E_STATE = -9,        /* call order violated (e.g. sigma before prepare)   */
  MLCC_E_REJECTED = -10,    /* serving: footprint above the server's budget      */
  MLCC_E_CANCELLED = -11,   /* serving: cancelled before it started              */
  MLCC_PENDING = 1          /* serving: mlcc_poll on a request still in progress */
} mlcc_status;

typedef enum {
  MLCC_FP64 = 0,    /* every contraction in binary64                                  */
  MLCC_BF16 = 1,    /* the Cholesky-rank doubles contractions of sigma on tcgen05 tensor
                       cores, bfloat16 operands, fp32 accumulation; the rest binary64  */
  MLCC_BF16X3 = 2,  /* as MLCC_BF16 with operands split x = x0 + x1 (bfloat16 pieces)
                       and the products x0y0 + x0y1 + x1y0                             */
  MLCC_BF16X6 = 3,  /* three pieces x0 + x1 + x2 and the six products of order <= 2   */
  MLCC_FP64E = 4    /* binary64 results from the tcgen05 tensor cores: every large GEMM
                       splits each operand row, scaled by a power of two, into 8 signed
                       base-2^7 integer digits (exact in bfloat16), sums the 36 digit
                       products of weight >= 2^-49 of the leading one in fp32 chunks of at
                       most 4096 products (exact integers), combines the chunks in 64-bit
                       integers and rounds to binary64. Error per product about
                       2^-53 |max row of A| |max column of B|; a row of A or column of B
                       holding NaN or Inf gives NaN in its output row or column. Small
                       GEMMs and all element-wise work stay binary64                    */
} mlcc_precision;

typedef enum { MLCC_LEVEL_CCS = 0, MLCC_LEVEL_CC2 = 1, MLCC_LEVEL_CCSD = 2 } mlcc_level;

typedef struct mlcc_ctx mlcc_ctx;
typedef struct mlcc_system mlcc_system;

typedef struct {
  int32_t n_mo;          /* orbitals in the reduced space (occupied first)            */
  int32_t n_occ;         /* doubly occupied orbitals                                  */
  int32_t n_chol;        /* Cholesky vectors N_J                                      */
  const int8_t* level;   /* host [n_mo], mlcc_level per orbital; CCSD must be a
                            subset of CC2 (nested active spaces, Sec. 2.1)            */
} mlcc_problem;

typedef struct {
  int32_t n_occ, n_vir;      /* N_o, N_v                                  */
  int32_t s_occ, s_vir;      /* CC2-active (includes the CCSD-active)     */
  int32_t t_occ, t_vir;      /* CCSD-active                               */
  int64_t n_singles;         /* n_vir * n_occ                             */
  int64_t n_doubles;         /* (s_vir * s_occ)^2                         */
  int64_t vector_len;        /* n_singles + n_doubles                     */
  int64_t workspace_bytes;   /* device memory held by the system          */
} mlcc_dims;

typedef struct {
  int32_t n_roots;        /* excitation energies wanted                               */
  int32_t max_gs_iter;    /* ground-state iterations                                  */
  int32_t max_es_iter;    /* Davidson iterations                                      */
  int32_t diis_dim;       /* DIIS history length                                      */
  int32_t max_subspace;   /* Davidson basis size before collapse (0: 8 n_roots)       */
  int32_t precision;      /* mlcc_precision of sigma inside the Davidson loop          */
  int32_t refine_fp64;    /* with a split-bfloat16 precision: refinement iterations in
                             refine_precision after the low-precision phase. Ground
                             state: if > 0, refine until gs_tol. Davidson: at most
                             refine_fp64 refinement iterations (1 = one Rayleigh-Ritz
                             sweep with refine_precision sigma on the low-precision
                             Ritz vectors), fewer if es_res_tol is met                  */
  int32_t gs_precision;   /* mlcc_precision of the ground-state iterations; the low-
                             precision phase ends when |Omega| < 1e-7, when it stops
                             halving over three iterations, or when below 1e-5 one
                             iteration does not halve it                               */
  double gs_tol;          /* |Omega|_2 threshold                                      */
  double gs_energy_tol;   /* |dE| threshold between iterations                        */
  double es_res_tol;      /* |A R - w R|_2 threshold per root                          */
  double es_omega_tol;    /* |dw| threshold per root                                   */
  double lowp_res_tol;    /* residual threshold of the low-precision phase            */
  int32_t refine_precision; /* precision of the refinement after a low-precision phase
                             (ground-state polish and Davidson sweeps): MLCC_FP64 or
                             MLCC_FP64E                                                 */
  int32_t sigma_graph;    /* non-zero: the Davidson solver captures the Jacobian
                             transformation of each precision in a CUDA graph (after one
                             eager evaluation that fills the operand caches) and replays it
                             for every trial vector, the vector staged through fixed
                             buffers; it saves the launches of the many small kernels of a
                             small system. Results are bitwise those of the eager path.
                             Not used while kernel timing is enabled. Default 0          */
} mlcc_options;

typedef struct {
  double e_hf;            /* sum_I (h_II + F_II), reduced-space reference energy      */
  double e_corr;          /* Eq. mlcc_energy at convergence                           */
  double omega_norm;      /* final |Omega|_2 (singles and CCSD doubles)               */
  int32_t iterations;
  int32_t converged;
} mlcc_gs_info;

typedef struct {
  int32_t iterations;     /* Davidson iterations (both phases)                         */
  int32_t n_sigma;        /* sigma-vectors evaluated                                  */
  int32_t n_sigma_lowp;   /* of which in low precision                                */
  int32_t converged;      /* residual thresholds met (or the refinement sweeps done)  */
  int32_t complex_pair;
  int32_t fp64_sweeps;    /* binary64 iterations after a low-precision phase          */
  double max_residual;    /* max_k |A R_k - w_k R_k|, last evaluation (its precision)  */
} mlcc_es_info;

/* ---- context ------------------------------------------------------------------ */
/* Defaults: 3 roots, 200 GS / 200 ES iterations, DIIS 8, FP64, gs_tol 1e-11,
   gs_energy_tol 1e-12, es_res_tol 1e-8, es_omega_tol 1e-11, lowp_res_tol 1e-4,
   refine_precision FP64. */
void mlcc_default_options(mlcc_options* opt);
/* Creates a context on CUDA device `device` with its own non-blocking stream and no
   device-memory budget of its own (a solve may use what the device has). */
mlcc_status mlcc_ctx_create(int device, mlcc_ctx** out);
/* As mlcc_ctx_create, with a device-memory budget: the systems of this context together
   (their workspace, mlcc_system_info) and each whole solve (mlcc_solve_footprint) may hold
   at most hbm_budget_bytes; a system or solve that would exceed it returns MLCC_E_OOM
   before allocating. hbm_budget_bytes <= 0: no budget. */
mlcc_status mlcc_ctx_create_budget(int device, int64_t hbm_budget_bytes, mlcc_ctx** out);
void mlcc_ctx_destroy(mlcc_ctx* ctx);
/* The cudaStream_t (as void*) that every entry point of this context launches on. */
void* mlcc_ctx_stream(mlcc_ctx* ctx);
const char* mlcc_last_error(void);
/* Kernel timing: when enabled, the library records CUDA events around each launch of
   a kernel family on the context stream: "rank_gemm_tc" (the Cholesky-rank doubles GEMMs
   on tcgen05 tensor cores in a split-bfloat16 precision), "rank_gemm_f64e" (the same
   GEMMs in MLCC_FP64E) and "rank_gemm_f64" (the same GEMMs on the binary64 FMA units);
   and phases of the solvers: "gs_omega" (one ground-state residual), "jacobian_prepare",
   "sigma" (one Jacobian transformation; inside it "sigma_singles", "sigma_doubles_to_singles",
   "sigma_cc2_doubles", "sigma_ccsd_rows", and inside the last the ladder GEMM of the CCSD
   rows, sum_cd g~_acbd c_cidj: "ladder_tc", "ladder_f64e" or "ladder_f64" by precision), "dav_update_G" (subspace matrix), "dav_ritz"
   (Ritz vectors and residuals), "dav_orthonormalise" (Gram-Schmidt of new directions).
   Phases contain the GEMM families launched inside them.
   mlcc_kernel_time returns launches, summed milliseconds and summed algorithmic flops
   (2 M N K of the contraction; split-bfloat16 precisions issue S times as many tensor
   operations, S = 1, 3, 6) since the last reset; it synchronises. */
void mlcc_kernel_timing(mlcc_ctx* ctx, int enable);
mlcc_status mlcc_kernel_time(mlcc_ctx* ctx, const char* family, int64_t* launches,
                             double* total_ms, double* total_flop);
/* Number of kernels libmlcc has launched in this process (all contexts), for accounting. */
int64_t mlcc_launch_count(void);

/* Dense GEMM on the context stream, row-major device matrices:
     C = alpha op(A) op(B) + beta C,  op(A) [M][K] (A[m*lda+k], or A[k*lda+m] if trans_a),
     op(B) [K][N] (B[k*ldb+n], or B[n*ldb+k] if trans_b), C [M][N] (C[m*ldc+n]).
   precision MLCC_FP64 runs on the binary64 FMA units; MLCC_BF16, MLCC_BF16X3, MLCC_BF16X6
   and MLCC_FP64E on the tcgen05 tensor cores as described at mlcc_precision (no fallback:
   a tensor-core precision with M or N below 16 for MLCC_FP64E, or K above 2^20, returns
   MLCC_E_ARG). Scratch is allocated for the call and freed before it returns; the call
   synchronises the stream. This is the contraction engine under every Cholesky-rank
   step of sigma and Omega, exposed for checking its arithmetic. */
mlcc_status mlcc_gemm(mlcc_ctx* ctx, int32_t trans_a, int32_t trans_b, int64_t M, int64_t N, int64_t K,
                      double alpha, const double* a_dev, int64_t lda, const double* b_dev, int64_t ldb,
                      double beta, double* c_dev, int64_t ldc, int32_t precision);

/* ---- system -------------------------------------------------------------------- */
/* Takes device copies of chol (Sec. 2.4 MO Cholesky vectors) and fock (Eq. eff_fock),
   re-orders orbitals by level, recovers the one-electron matrix
   h = F - sum_i (2 g_pqii - g_piiq) (Eq. eff_fock, environment absorbed in h) and
   allocates the workspace. chol_dev / fock_dev may be freed after the call returns. */
mlcc_status mlcc_system_create(mlcc_ctx* ctx, const mlcc_problem* prob,
                               const double* chol_dev, const double* fock_dev,
                               mlcc_system** out);
void mlcc_system_destroy(mlcc_system* sys);
mlcc_status mlcc_system_info(const mlcc_system* sys, mlcc_dims* dims);
/* perm_host[k] = caller index of internal orbital k, k < n_mo (before the semicanonical
   rotation inside each level). */
mlcc_status mlcc_orbital_order(const mlcc_system* sys, int32_t* perm_host);
/* The system's orbitals in the caller's: orbital k of the system is
   sum_p c_host[p * n_mo + k] (caller orbital p), [n_mo][n_mo]. A permutation matrix (from
   mlcc_orbital_order) when no level block needed the semicanonical rotation. */
mlcc_status mlcc_orbitals(const mlcc_system* sys, double* c_host);

/* ---- steps of the hot path (device buffers, internal order, no host sync) ------- */
/* T1-dressing (Sec. 2.1 "Cholesky vectors in the X1 basis", Appendix A):
   Lt^J = (1 - t1) L^J (1 + t1) for every J. t1_dev [n_vir][n_occ];
   lt_dev [n_chol][n_mo][n_mo] (not symmetric). */
mlcc_status mlcc_t1_transform(mlcc_system* sys, const double* t1_dev, double* lt_dev);
/* Fock matrix in the X1 basis (Appendix A, with the one-electron term h~):
   F~ = h~ + sum_J [2 Lt^J (sum_I Lt^J_II) - Lt^J_{:,occ} Lt^J_{occ,:}]; f_dev [n_mo][n_mo]. */
mlcc_status mlcc_fock_t1(mlcc_system* sys, const double* t1_dev, double* f_dev);
/* Ground-state residual with t1 and all doubles as independent inputs (Appendix A:
   Eq. mlcc2_omega_codable for the singles, the analytic CC2 equation on P_S, the MLCCSD
   doubles residual on P_T) and the correlation energy of Eq. mlcc_energy.
   om1_dev [n_singles], om2_dev [n_doubles]; energy_dev: one double (device). */
mlcc_status mlcc_omega(mlcc_system* sys, const double* t1_dev, const double* x2_dev,
                       double* om1_dev, double* om2_dev, double* energy_dev);
/* DIIS-accelerated quasi-Newton solve of Omega = 0 (Sec. 2.1). Outputs the converged
   amplitudes (device) and fills info (host). Keeps them as the Jacobian ground state. */
mlcc_status mlcc_ground_state(mlcc_system* sys, const mlcc_options* opt,
                              double* t1_dev, double* x2_dev, mlcc_gs_info* info);
/* Builds everything sigma needs at the ground state (t1, x2): dressed vectors, F~,
   the MLCC2 intermediates X_Ji and Y_aB (Appendix A) and the CCSD-block value tensors.
   Must precede mlcc_sigma; mlcc_ground_state calls it on success. */
mlcc_status mlcc_jacobian_prepare(mlcc_system* sys, const double* t1_dev,
                                  const double* x2_dev);
/* sigma = A c for n_vec trial vectors (Appendix A, Jacobian transformation):
   c_dev, sigma_dev [n_vec][vector_len]. precision: mlcc_precision. */
mlcc_status mlcc_sigma(mlcc_system* sys, int32_t n_vec, const double* c_dev,
                       double* sigma_dev, int32_t precision);
/* Jacobian transformation split over the Cholesky index (Sec. 2.4: every integral is a sum
   over J, g_pqrs = sum_J L^J_pq L^J_rs, and so is every heavy term of sigma). Writes the part
   of sigma = A c that sums over the Cholesky vectors J in [j_begin, j_end) and, when
   with_rest is non-zero, adds the terms that do not sum over J (those built from F~, the
   MLCC2 intermediates X and Y, the cached CCSD value tensors and the orbital energies).
   Ranks whose ranges tile [0, n_chol), exactly one of them with with_rest, obtain
   mlcc_sigma's result by one sum (an all-reduce) of their outputs per sigma batch. Here
   each rank holds the whole prepared system and the work is what is split. Layout,
   precisions and errors as mlcc_sigma; the range must not be empty (0 <= j_begin < j_end <=
   n_chol, else MLCC_E_ARG), so there are at most n_chol ranks. In a split-bfloat16 precision the cached bfloat16 operands are not used inside a
   range: each call converts its operands. */
mlcc_status mlcc_sigma_partial(mlcc_system* sys, int32_t j_begin, int32_t j_end, int32_t with_rest,
                               int32_t n_vec, const double* c_dev, double* sigma_dev, int32_t precision);
/* Left eigenvectors (the transition moments the paper names as a motivation, Sec. 1, need
   them beside the right ones): rho = A^T l, the adjoint of mlcc_sigma in the plain inner
   product of the vector storage on symmetric doubles (the doubles of l must be symmetric;
   those of rho are symmetrised). Systems without a CCSD level (MLCC2, CC2, CCS and their
   combinations); MLCC_E_ARG otherwise, MLCC_E_STATE before mlcc_jacobian_prepare. Layout
   and precisions as mlcc_sigma. */
mlcc_status mlcc_sigma_left(mlcc_system* sys, int32_t n_vec, const double* l_dev, double* rho_dev,
                            int32_t precision);
/* The lowest opt->n_roots left eigenpairs by the Davidson solver of mlcc_excited_states on
   A^T (same options, the same eigenvalues as the right problem): omega_host [n_roots],
   l_dev [n_roots][vector_len]. With r_dev (the right eigenvectors of the same roots, e.g.
   from mlcc_excited_states) each l_k is scaled so that <l_k, r_k> = 1; NULL: unit 2-norm,
   largest-magnitude element positive. */
mlcc_status mlcc_excited_states_left(mlcc_system* sys, const mlcc_options* opt, double* omega_host,
                                     double* l_dev, const double* r_dev, mlcc_es_info* info);
/* Folded CC2 Jacobian (the CC2 response strategy Sec. 2.1 points to). In the three-level
   model the doubles rows outside the CCSD block (P_S) have the diagonal doubles block
   eps_aibj and no coupling to the CCSD-block doubles (P_T), so an eigenpair (omega, c) of
   A has c_S = (omega - eps_S)^-1 A_S1 c1, and (c1, c_T) is an eigenvector with eigenvalue
   omega of A_eff(omega) = [[A_11 + A_1S (omega - eps_S)^-1 A_S1, A_1T], [A_T1, A_TT]].
   mlcc_sigma_eff applies A_eff(omega[k]) to n_vec vectors c_dev [n_vec][vector_len] in the
   vector layout (only the singles and the P_T doubles of c are read): sigma_dev
   [n_vec][vector_len] gets the singles and P_T rows, zero on P_S. dsigma_dev (or NULL)
   [n_vec][n_singles] gets the singles of dA_eff/domega c = -A_1S (omega - eps_S)^-2 A_S1 c1
   (the P_T rows do not depend on omega). Cost per vector: three partial Jacobian
   transformations (two without dsigma), each with one Cholesky-rank GEMM: the P_S rows of
   sigma(c1, 0), the singles and P_T rows of sigma(c1, c_S + c_T), and the
   doubles-to-singles part of sigma(0, x_S); in `precision`. Each omega[k] (host) must lie below the lowest
   P_S denominator (mlcc_fold_window), else MLCC_E_ARG; MLCC_E_STATE before
   mlcc_jacobian_prepare. Scratch: three vectors, allocated for the call; synchronises. */
mlcc_status mlcc_sigma_eff(mlcc_system* sys, int32_t n_vec, const double* omega_host,
                           const double* c_dev, double* sigma_dev, double* dsigma_dev,
                           int32_t precision);
/* The lowest P_S denominator min eps_aibj over P_S (Hartree; 1e300 without P_S pairs):
   the folded problem is used for omega below it. */
mlcc_status mlcc_fold_window(const mlcc_system* sys, double* omega_max);
/* Lowest opt->n_roots excitation energies below the lowest P_S denominator from the folded
   CC2 Jacobian (mlcc_sigma_eff), by a Davidson-type solver whose subspaces hold only
   singles and CCSD-block doubles (n_vir n_occ + (t_vir t_occ)^2 elements per vector) and are
   kept across omega updates: each trial vector b keeps A_eff(w_b) b and dA_eff/domega b at
   the omega w_b it was applied at, and the projected problem uses the first-order model in
   omega - w_b. Stage 1 finds all roots roughly with one omega; stage 2 refines each root in
   its own subspace, restarting from the Ritz vector applied exactly at omega until every
   vector of the subspace was applied within 1e-7 Ha of it and the model residual is below
   opt->es_res_tol. opt->precision (MLCC_FP64 or MLCC_FP64E) is the sigma precision;
   opt->max_es_iter bounds each stage; opt->max_subspace the subspace (0: 8 n_roots).
   omega_host [n_roots] ascending; r_dev [n_roots][vector_len] or NULL: the unfolded
   eigenvectors (c1, c_S(omega) + c_T), unit 2-norm, largest-magnitude element positive.
   info->n_sigma counts partial Jacobian transformations (three per application). Needs
   2 n_roots <= n_vir n_occ. MLCC_E_ES_NOCONV if a root does not converge (or two roots
   settle on the same eigenpair); MLCC_E_COMPLEX_ROOT (info->complex_pair = 1) if a wanted
   eigenvalue is one of a complex pair, whose real part is then reported. */
mlcc_status mlcc_excited_states_folded(mlcc_system* sys, const mlcc_options* opt,
                                       double* omega_host, double* r_dev, mlcc_es_info* info);
/* Davidson solve for the lowest opt->n_roots eigenpairs of A at the prepared ground
   state. omega_host [n_roots] (Hartree, ascending); r_dev [n_roots][vector_len]
   (unit 2-norm, largest-magnitude element positive) or NULL; info (host). */
mlcc_status mlcc_excited_states(mlcc_system* sys, const mlcc_options* opt,
                                double* omega_host, double* r_dev, mlcc_es_info* info);

/* ---- whole solve ------------------------------------------------------------------- */
/* What a whole solve returns (Sec. 2.1: the converged ground state, the energy and the lowest
   eigenpairs of the Jacobian). gs and es are filled by the call. The arrays are the
   caller's, NULL where not wanted; omega is required. For mlcc_solve every array is host
   memory; for mlcc_solve_device t1, x2 and r are device memory on the context's device and
   the others host memory. Amplitudes and vectors are in the system's orbital order and
   basis (see Conventions); perm and orbitals relate it to the caller's. */
typedef struct {
  mlcc_gs_info gs;
  mlcc_es_info es;
  double* omega;      /* [n_roots] excitation energies, Hartree, ascending                  */
  double* residual;   /* [n_roots] |A R_k - w_k R_k|_2 at the last evaluation, in its
                         precision (binary64-class after a refinement sweep)               */
  double* t1;         /* [n_vir][n_occ] converged singles amplitudes                      */
  double* x2;         /* [n_doubles] converged doubles on the CC2-active pairs, the layout
                         under Conventions (the analytic CC2 doubles outside the CCSD block) */
  double* r;          /* [n_roots][vector_len] right eigenvectors, unit 2-norm, largest-
                         magnitude element positive                                        */
  int32_t* perm;      /* [n_mo] as mlcc_orbital_order                                      */
  double* orbitals;   /* [n_mo][n_mo] as mlcc_orbitals                                     */
} mlcc_result;

/* Copies chol_host / fock_host to the device, builds the system, runs the ground state and
   the excited states, fills *res and frees everything it allocated. On MLCC_E_GS_NOCONV
   or MLCC_E_ES_NOCONV (and MLCC_E_COMPLEX_ROOT) the outputs hold the last iterate. */
mlcc_status mlcc_solve(mlcc_ctx* ctx, const mlcc_problem* prob, const double* chol_host,
                       const double* fock_host, const mlcc_options* opt, mlcc_result* res);

/* As mlcc_solve, with chol_dev / fock_dev on the context's device (borrowed for the call;
   the caller keeps ownership). The system copies them, so they may be reused after the
   call returns. */
mlcc_status mlcc_solve_device(mlcc_ctx* ctx, const mlcc_problem* prob, const double* chol_dev,
                              const double* fock_dev, const mlcc_options* opt, mlcc_result* res);

/* Length of a Davidson vector of the problem, n_vir n_occ + (s_vir s_occ)^2 (the layout
   under "Conventions"), from the sizes and levels alone; -1 if they are invalid. */
int64_t mlcc_vector_len(const mlcc_problem* prob);

/* Device memory that mlcc_solve of this problem with these options holds at its peak, in
   bytes: the system (Cholesky vectors, their dressed copies, intermediates and scratch),
   then either the device copies of the inputs (while the system is built) or the
   amplitudes, the CCSD value tensors, the bfloat16 operands, the Davidson subspace and an
   allowance for the converted operand copies of the tensor-core precisions. Allocations
   are counted in 2 MiB pages. The serving loop admits requests by this number. */
mlcc_status mlcc_solve_footprint(const mlcc_problem* prob, const mlcc_options* opt, int64_t* bytes);

/* ---- serving loop ----------------------------------------------------------------- */
/* A server runs independent whole solves (mlcc_solve) submitted as requests. It has
   n_slots slots, each a host worker thread with its own context and stream, and a device
   memory budget. Admission: the oldest waiting request starts when a slot is free and the
   footprints (mlcc_solve_footprint) of the running requests plus its own fit in the
   budget; requests start in submission order, none overtakes an older one. Requests
   that are admitted together run concurrently on their own streams, so their kernels
   overlap on the device. A request whose solve runs out of device memory while other
   requests run goes back to the head of the queue until one of them finishes (at most 3
   admissions). Each request's result is that of mlcc_solve on the same inputs alone. */
typedef struct mlcc_server mlcc_server;

typedef struct {
  int32_t status;          /* the solve's mlcc_status; MLCC_E_CANCELLED if cancelled first */
  int32_t slot;            /* slot that ran it (-1: it never ran)                          */
  int32_t attempts;        /* admissions: 1, more after out-of-memory retries              */
  int32_t n_roots;         /* entries written to omega_host                                */
  int64_t footprint_bytes; /* the footprint it was admitted with                           */
  double t_submit;         /* seconds since the server was created (host steady clock):    */
  double t_start;          /*   submitted, last admitted, finished; latency is              */
  double t_finish;         /*   t_finish - t_submit                                         */
  mlcc_gs_info gs;
  mlcc_es_info es;
} mlcc_request_result;

typedef struct {
  int32_t n_slots;
  int32_t running, waiting, peak_running;
  int64_t budget_bytes, in_use_bytes, peak_bytes;   /* footprints admitted at once */
  int64_t submitted, finished, cancelled, retried;
} mlcc_server_info;

/* Creates a server on CUDA device `device` with n_slots in [1, 64] slots. hbm_budget_bytes
   <= 0 takes 90% of the device memory free at creation. */
mlcc_status mlcc_server_create(int device, int32_t n_slots, int64_t hbm_budget_bytes,
                               mlcc_server** out);
/* Cancels the requests that have not started, waits for the running ones and frees the
   server, with the results nobody polled. No other call on the server may be in progress. */
void mlcc_server_destroy(mlcc_server* srv);
/* Queues a whole solve and returns its ticket (> 0). The problem (with its level array)
   and the options are copied; chol_host and fock_host are borrowed: the caller keeps them
   valid and unchanged until mlcc_poll has returned the request's result.
   MLCC_E_REJECTED: the footprint exceeds the whole budget (the request is not queued). */
mlcc_status mlcc_submit(mlcc_server* srv, const mlcc_problem* prob, const double* chol_host,
                        const double* fock_host, const mlcc_options* opt, uint64_t* ticket);
/* Waits up to wait_ms milliseconds (0: no wait; < 0: until it finishes) for the request.
   Finished: fills *res and omega_host [n_roots] (the request's excitation energies,
   ascending, Hartree), forgets the ticket and returns MLCC_OK; the request's own status
   is res->status (with mlcc_last_error() set to its message when it failed). Still in
   progress: MLCC_PENDING. Unknown (or already polled) ticket: MLCC_E_ARG. One thread at
   a time should poll a given ticket. */
mlcc_status mlcc_poll(mlcc_server* srv, uint64_t ticket, int64_t wait_ms, mlcc_request_result* res,
                      double* omega_host);
/* Removes a request that has not started (its poll then reports MLCC_E_CANCELLED).
   MLCC_E_STATE if it has started or finished, MLCC_E_ARG for an unknown ticket. */
mlcc_status mlcc_cancel(mlcc_server* srv, uint64_t ticket);
mlcc_status mlcc_server_stats(mlcc_server* srv, mlcc_server_info* info);

/* ---- active-space selection: correlated natural transition orbitals ----------------- */
/* CNTOs (Sec. 2.2, Eqs. M, N, approx_double_1, approx_double_2, select_CNTOs): from the
   lowest n_states CCS excitation vectors R_ai (unit 2-norm) and energies omega, the
   approximate doubles
     R_aibj = -gbar_aibj / ((1 + delta_{ai,bj}) (eps_a + eps_b - eps_i - eps_j - omega)),
     gbar_aibj = P^{ab}_{ij} (sum_{cJ} R_ci L^J_bj L^J_ac - sum_{kJ} R_bk L^J_kj L^J_ai),
   then M_ij = sum_a R_ai R_aj + 1/2 sum_abk (1 + delta_{ai,bk} delta_ij) R_aibk R_ajbk and
   N_ab = sum_i R_ai R_bi + 1/2 sum_ijc (1 + delta_{ai,cj} delta_ab) R_aicj R_bicj summed over
   the states, and their eigenpairs: the eigenvectors of M (N) rotate the occupied
   (virtual) orbitals, and those of the largest eigenvalues are the active ones.
   Inputs: canonical orbitals (fock_dev diagonal, else MLCC_E_ARG) in the caller's order
   (occupied first), chol_dev [n_chol][n_mo][n_mo] symmetric, both device memory on the
   context's device. All outputs are host memory owned by the caller. The doubles are
   built and contracted in blocks of rows, so their (n_vir n_occ)^2 size is never held at
   once. precision: mlcc_precision of the large contractions (MLCC_FP64, MLCC_FP64E or a
   split-bfloat16 one); the CCS states are solved in binary64. Synchronises. */
typedef struct {
  double* omega;         /* [n_states] CCS excitation energies, Hartree; required          */
  double* m;             /* [n_occ][n_occ] M summed over the states, or NULL               */
  double* n;             /* [n_vir][n_vir] N summed over the states, or NULL               */
  double* occ_values;    /* [n_occ] eigenvalues of M, descending; required                 */
  double* occ_vectors;   /* [n_occ][n_occ] row-major, column k the eigenvector of
                            occ_values[k] (largest-magnitude component positive), or NULL */
  double* vir_values;    /* [n_vir] eigenvalues of N, descending; required                 */
  double* vir_vectors;   /* [n_vir][n_vir] as occ_vectors, or NULL                         */
  int32_t n_occ_active;  /* in: n_o^a, the active occupied CNTOs                          */
  int32_t n_vir_active;  /* in: n_v^a, or <= 0 for Eq. select_CNTOs, n_v^a = (N_v / N_o)
                            n_o^a rounded to the nearest integer; out: the value used      */
  int32_t block_rows;    /* in: rows (pairs ai) of the doubles built at once; 0: about
                            128 MiB of doubles per block                                   */
  int32_t reserved;      /* zero                                                           */
} mlcc_cnto_result;
mlcc_status mlcc_cnto(mlcc_ctx* ctx, int32_t n_mo, int32_t n_occ, int32_t n_chol,
                      const double* chol_dev, const double* fock_dev, int32_t n_states,
                      int32_t precision, mlcc_cnto_result* res);

/* ---- Cholesky vectors: MO-screened decomposition and MO vectors ---------------------- */
/* Sec. 2.4. The AO integral matrix g has rows and columns indexed by AO pairs (ab):
   g[(ab)][(cd)] = (ab|cd), symmetric positive semi-definite, row-major [n_pairs][n_pairs]
   device memory. The decomposition takes, one at a time, the pair K with the largest
   screened diagonal w[K] D[K] (D the diagonal updated by the vectors so far) and stops when
   that value is below tau (Eq. standard_cholesky; w = 1 without screening); each new vector
   is L[:, J] = (g[:, K] - L[:, :J] L[K, :J]^T) / sqrt(D[K]).

   mlcc_mo_screening: w_dev [n_ao * n_ao], w[(ab)] = nu_a nu_b with nu_a = max_p C[a][p]^2
   over the active MO coefficients c_active_dev [n_ao][n_active] (Eqs. mo_screening and
   cd_screening). No synchronisation. */
mlcc_status mlcc_mo_screening(mlcc_ctx* ctx, int32_t n_ao, int32_t n_active, const double* c_active_dev,
                              double* w_dev);
/* The decomposition: w_dev [n_pairs] or NULL (unscreened); l_dev [n_pairs][max_vectors]
   (column J is vector J); pivots_host [max_vectors] the basis pairs in order; diag_dev
   [n_pairs] or NULL: the final D; *n_vectors the vectors made (at most max_vectors).
   Synchronises (the host reads each step's largest diagonal to decide the stop). */
mlcc_status mlcc_cholesky_decompose(mlcc_ctx* ctx, int64_t n_pairs, const double* g_dev, const double* w_dev,
                                    double tau, int32_t max_vectors, int32_t* pivots_host, double* l_dev,
                                    double* diag_dev, int32_t* n_vectors);
/* Algorithm 1: MO Cholesky vectors from the basis, L^J_pq = sum_K X_pqK [Q^-T]_KJ with
   X_pqK = sum_ab C_ap C_bq (ab|K) and S = g[B, B] = Q Q^T. g_dev as above with n_pairs =
   n_ao^2; pivots_host [n_vectors]; c_dev [n_ao][n_mo]; lmo_dev [n_vectors][n_mo][n_mo] (the
   layout of mlcc_problem's Cholesky vectors). MLCC_E_ARG if S is not positive definite.
   Synchronises. */
mlcc_status mlcc_cholesky_mo_vectors(mlcc_ctx* ctx, int32_t n_ao, int32_t n_mo, const double* g_dev,
                                     const int32_t* pivots_host, int32_t n_vectors, const double* c_dev,
                                     double* lmo_dev);

/* ---- allocation-free variant ------------------------------------------------------ */
/* The paper has no counterpart to this entry point; it exists for callers that cannot let
   a library allocate device memory: a program that reserves the device memory for its own
   pool (so cudaMalloc would fail or escape its accounting), or one that cannot accept the
   device-wide synchronisation cudaMalloc / cudaFree may cause.

   mlcc_fock_t1_noalloc computes the same quantities as mlcc_t1_transform and mlcc_fock_t1
   (dressed Cholesky vectors Lt^J = (1 - t1) L^J (1 + t1) and the X1-basis Fock matrix
   F~ = h~ + sum_J [2 Lt^J (sum_I Lt^J_II) - Lt^J[:, I] Lt^J[I, :]] with
   h = F - sum_J [2 L^J (sum_I L^J_II) - L^J[:, I] L^J[I, :]]) without a system and
   without allocating: every buffer is the caller's, in the caller's orbital order
   (occupied first): chol_dev [n_chol][n_mo][n_mo], fock_dev and ft_dev [n_mo][n_mo],
   t1_dev [n_mo - n_occ][n_occ], lt_dev [n_chol][n_mo][n_mo]. Work goes on `stream`
   (a cudaStream_t, NULL for the default stream); the call does not synchronise.
   Scratch: a static device array of 2 * MLCC_NOALLOC_MAX_CHOL doubles (512 KiB), held by
   every device that loads the library until the process exits; n_chol above the limit
   returns MLCC_E_ARG. Each call looks up the array's address on the current device (the
   first call on a device also loads the library's device code there: make that first call
   before any stream capture). All calls share the array, so calls whose work overlaps on
   the device race; order them on one stream. */
#define MLCC_NOALLOC_MAX_CHOL 32768
mlcc_status mlcc_fock_t1_noalloc(int32_t n_mo, int32_t n_occ, int32_t n_chol,
                                 const double* chol_dev, const double* fock_dev,
                                 const double* t1_dev, double* lt_dev, double* ft_dev,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MLCC_H */

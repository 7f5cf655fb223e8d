// Tensor-core (tcgen05) Cholesky-rank GEMMs for the mixed-precision path.
#include "system.cuh"

namespace mlcc {
void rank_gemm_lowp(mlcc_system* S, bool outer, const double* A, const double* B, double* C,
                    double alpha, double beta) {
  (void)S; (void)outer; (void)A; (void)B; (void)C; (void)alpha; (void)beta;
  throw Error(MLCC_E_ARG, "MLCC_BF16 precision is not available in this build");
}
}  // namespace mlcc

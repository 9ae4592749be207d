// k_assemble_general_mass.cu -- the general-mesh LOR assembly with the
// reaction term's sub-hex mass blocks (kernel in k_assemble_impl.cuh).
#include "k_assemble_impl.cuh"

cudaError_t lor_assemble_general_mass_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                               const double* beta, double* vals, cudaStream_t s) {
  return assemble_dispatch<double, true, true>(m, T, kappa, beta, vals, s);
}

cudaError_t lor_assemble_general_mass_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                               const double* beta, float* vals, cudaStream_t s) {
  return assemble_dispatch<float, true, true>(m, T, kappa, beta, vals, s);
}

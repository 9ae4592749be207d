// k_assemble_general.cu -- the macro-element LOR assembly on a general
// conforming hex mesh (no reaction term): the same sub-hex blocks, DOFs from
// the element-to-DOF map and CSR positions by binary search in the row of the
// pattern built from that map (kernel in k_assemble_impl.cuh).  The reaction
// variant is instantiated in k_assemble_general_mass.cu.
#include "k_assemble_impl.cuh"

cudaError_t lor_assemble_general_mass_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                               const double* beta, double* vals, cudaStream_t s);
cudaError_t lor_assemble_general_mass_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                               const double* beta, float* vals, cudaStream_t s);

cudaError_t lor_assemble_general_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                          const double* beta, double* vals, cudaStream_t s) {
  if (beta) return lor_assemble_general_mass_dispatch(m, T, kappa, beta, vals, s);
  return assemble_dispatch<double, false, true>(m, T, kappa, nullptr, vals, s);
}

cudaError_t lor_assemble_general_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                          const double* beta, float* vals, cudaStream_t s) {
  if (beta) return lor_assemble_general_mass_dispatch(m, T, kappa, beta, vals, s);
  return assemble_dispatch<float, false, true>(m, T, kappa, nullptr, vals, s);
}

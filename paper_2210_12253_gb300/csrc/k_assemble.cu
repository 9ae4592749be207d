// k_assemble.cu -- Step S1.2 / A1 + A4: launchers of the batched LOR matrix
// assembly (kernel in k_assemble_impl.cuh): values zeroed, then one launch of
// the sub-hex block kernel (which also sets the essential diagonals to 1),
// with the reaction term's mass blocks (k_assemble_mass.cu) when beta is
// given.
#include "k_assemble_impl.cuh"

cudaError_t lor_assemble_mass_dispatch(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta,
                                       double* vals, cudaStream_t s);
cudaError_t lor_assemble_mass_dispatch(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta,
                                       float* vals, cudaStream_t s);
// general meshes (k_assemble_general.cu, k_assemble_general_mass.cu)
cudaError_t lor_assemble_general_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                          const double* beta, double* vals, cudaStream_t s);
cudaError_t lor_assemble_general_dispatch(const LorMesh& m, const LorTables& T, const double* kappa,
                                          const double* beta, float* vals, cudaStream_t s);

namespace {

template <typename VT>
cudaError_t launch(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta, VT* vals,
                   cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(vals, 0, sizeof(VT) * m.nnz, s);
  if (err != cudaSuccess) return err;
  if (m.edofs) return lor_assemble_general_dispatch(m, T, kappa, beta, vals, s);
  if (beta) return lor_assemble_mass_dispatch(m, T, kappa, beta, vals, s);
  return assemble_dispatch<VT, false, false>(m, T, kappa, nullptr, vals, s);
}

}  // namespace

cudaError_t lor_launch_assemble(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta,
                                void* values, int dtype, cudaStream_t s) {
  if (dtype == LOR_F64) return launch<double>(m, T, kappa, beta, (double*)values, s);
  return launch<float>(m, T, kappa, beta, (float*)values, s);
}

// k_assemble.cu -- Step S1.2 / A1 + A4: launchers of the batched LOR matrix
// assembly (kernel in k_assemble_impl.cuh): values zeroed, essential
// diagonals preset to 1, then one launch of the sub-hex block kernel, with the
// reaction term's mass blocks (k_assemble_mass.cu) when beta is given.
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

// Diagonal of every essential row = 1 (the values are zeroed before);
// closed-form position on the structured grid, found in the row otherwise.
template <typename VT>
__global__ void k_essential_diagonal(LorMesh m, VT* __restrict__ vals) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m.ndof; r += (int64_t)gridDim.x * blockDim.x) {
    if (m.ess) {
      if (!m.ess[r]) continue;
      const int64_t pos = lor_find_col(m.colidx, m.rowptr[r], m.rowptr[r + 1], r);
      if (pos >= 0) vals[pos] = (VT)1;
      continue;
    }
    const int64_t I = r % m.nx, J = (r / m.nx) % m.ny, K = r / (m.nx * m.ny);
    if (lor_is_essential(I, J, K, m.nx, m.ny, m.nz)) vals[lor_entry_pos(I, J, K, 0, 0, 0, m.nx, m.ny, m.nz)] = (VT)1;
  }
}

template <typename VT>
cudaError_t launch(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta, VT* vals,
                   cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(vals, 0, sizeof(VT) * m.nnz, s);
  if (err != cudaSuccess) return err;
  {
    const int64_t blocks = (m.ndof + 255) / 256;
    k_essential_diagonal<VT><<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(m, vals); lor_count_launch();
  }
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

// k_apply.cu -- Step S2.1: launchers of the matrix-free high-order operator
// and its backward (kernels in k_apply_impl.cuh).  Without a reaction term the
// kernels instantiated here run; with one (the definite Helmholtz operator of
// Section 4.1) those of k_apply_mass.cu.
#include "k_apply_impl.cuh"

cudaError_t lor_apply_mass_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                    const double* x, double* y, cudaStream_t s);
cudaError_t lor_backward_mass_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                       const double* kappa, const double* x, const double* gy, double* gx,
                                       double* gk, cudaStream_t s);
// general meshes (k_apply_general.cu)
cudaError_t lor_apply_general_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                       const double* x, double* y, cudaStream_t s);
cudaError_t lor_backward_general_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                          const double* kappa, const double* x, const double* gy, double* gx,
                                          double* gk, cudaStream_t s);

namespace {

// y <- x on essential DOFs, 0 elsewhere (the apply then adds the free rows).
__global__ void k_init_output(LorMesh m, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m.ndof; r += (int64_t)gridDim.x * blockDim.x) {
    y[r] = lor_dof_essential(m, r) ? x[r] : 0.0;
  }
}

cudaError_t init_output(const LorMesh& m, const double* x, double* y, cudaStream_t s) {
  const int64_t blocks = (m.ndof + 255) / 256;
  k_init_output<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(m, x, y); lor_count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t lor_launch_apply(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                             const double* x, double* y, cudaStream_t s) {
  cudaError_t err = init_output(m, x, y, s);
  if (err != cudaSuccess) return err;
  return lor_launch_apply_accumulate(m, T, Dq, Mq, x, y, s);
}

cudaError_t lor_launch_apply_accumulate(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                        const double* x, double* y, cudaStream_t s) {
  if (m.edofs) return lor_apply_general_dispatch(m, T, Dq, Mq, x, y, s);
  if (Mq) return lor_apply_mass_dispatch(m, T, Dq, Mq, x, y, s);
  return apply_dispatch<false, false, double>(m, T, Dq, nullptr, x, y, s);
}

cudaError_t lor_launch_apply_f32(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                 const double* x, double* y, cudaStream_t s) {
  cudaError_t err = init_output(m, x, y, s);
  if (err != cudaSuccess) return err;
  return lor_launch_apply_f32_accumulate(m, T, Dq, Mq, x, y, s);
}

cudaError_t lor_launch_apply_backward(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                      const double* kappa, const double* x, const double* gy, double* gx,
                                      double* gkappa, cudaStream_t s) {
  if (gx) {
    cudaError_t err = init_output(m, gy, gx, s);
    if (err != cudaSuccess) return err;
  }
  if (!gx && !gkappa) return cudaSuccess;
  if (m.edofs) return lor_backward_general_dispatch(m, T, Dq, Mq, kappa, x, gy, gx, gkappa, s);
  if (Mq) return lor_backward_mass_dispatch(m, T, Dq, Mq, kappa, x, gy, gx, gkappa, s);
  return backward_dispatch<false, false>(m, T, Dq, nullptr, kappa, x, gy, gx, gkappa, s);
}

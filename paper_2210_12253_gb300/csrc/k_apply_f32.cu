// k_apply_f32.cu -- the high-order apply (Step S2.1) with FP32 arithmetic,
// for the inner solves of the mixed-precision iterative refinement: the same
// sum-factorisation kernel as the FP64 apply (k_apply_impl.cuh) instantiated
// with float tables, stage buffers and D (and beta w detJ) factors; x is read
// and y accumulated in FP64.  Structured meshes here, general meshes in
// k_apply_f32_general.cu.
#include "k_apply_impl.cuh"

cudaError_t lor_apply_f32_general_dispatch(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                           const double* x, double* y, cudaStream_t s);
cudaError_t lor_apply_f32v_general_dispatch(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                            const float* x, float* y, cudaStream_t s);

namespace {

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

}  // namespace

cudaError_t lor_launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  k_to_f32<<<(int)(blocks < 152 * 16 ? (blocks > 0 ? blocks : 1) : 152 * 16), 256, 0, s>>>(n, a, b);
  lor_count_launch();
  return cudaGetLastError();
}

cudaError_t lor_launch_apply_f32_accumulate(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                            const double* x, double* y, cudaStream_t s) {
  if (m.edofs) return lor_apply_f32_general_dispatch(m, T, Dq, Mq, x, y, s);
  if (Mq) return apply_dispatch<true, false, float>(m, T, Dq, Mq, x, y, s);
  return apply_dispatch<false, false, float>(m, T, Dq, nullptr, x, y, s);
}

// The same with FP32 input and output vectors (FP32 atomics into y), for the
// refinement's inner iterations whose vectors are FP32.
cudaError_t lor_launch_apply_f32v_accumulate(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                             const float* x, float* y, cudaStream_t s) {
  if (m.edofs) return lor_apply_f32v_general_dispatch(m, T, Dq, Mq, x, y, s);
  if (Mq) return apply_dispatch<true, false, float, float>(m, T, Dq, Mq, x, y, s);
  return apply_dispatch<false, false, float, float>(m, T, Dq, nullptr, x, y, s);
}

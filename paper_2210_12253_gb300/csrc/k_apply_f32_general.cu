// k_apply_f32_general.cu -- the FP32-arithmetic high-order apply on a general
// conforming hex mesh (gather/scatter through the element-to-DOF map; kernels
// in k_apply_impl.cuh).
#include "k_apply_impl.cuh"

cudaError_t lor_apply_f32_general_dispatch(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                           const double* x, double* y, cudaStream_t s) {
  if (Mq) return apply_dispatch<true, true, float>(m, T, Dq, Mq, x, y, s);
  return apply_dispatch<false, true, float>(m, T, Dq, nullptr, x, y, s);
}

cudaError_t lor_apply_f32v_general_dispatch(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                            const float* x, float* y, cudaStream_t s) {
  if (Mq) return apply_dispatch<true, true, float, float>(m, T, Dq, Mq, x, y, s);
  return apply_dispatch<false, true, float, float>(m, T, Dq, nullptr, x, y, s);
}

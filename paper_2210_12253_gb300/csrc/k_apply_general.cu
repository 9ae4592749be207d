// k_apply_general.cu -- the high-order apply and its backward on a general
// conforming hex mesh: the gather G and scatter G^T of Eq. (4) go through the
// element-to-DOF map (the element restriction of Step S1.1) and the essential
// mask instead of the structured index (kernels in k_apply_impl.cuh).
#include "k_apply_impl.cuh"

cudaError_t lor_apply_general_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                       const double* x, double* y, cudaStream_t s) {
  if (Mq) return apply_dispatch<true, true, double>(m, T, Dq, Mq, x, y, s);
  return apply_dispatch<false, true, double>(m, T, Dq, nullptr, x, y, s);
}

cudaError_t lor_backward_general_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                          const double* kappa, const double* x, const double* gy, double* gx,
                                          double* gk, cudaStream_t s) {
  if (Mq) return backward_dispatch<true, true>(m, T, Dq, Mq, kappa, x, gy, gx, gk, s);
  return backward_dispatch<false, true>(m, T, Dq, nullptr, kappa, x, gy, gx, gk, s);
}

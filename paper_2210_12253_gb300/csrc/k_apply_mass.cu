// k_apply_mass.cu -- the high-order apply and its backward with the reaction
// term of the definite Helmholtz operator (Section 4.1): the z-line step also
// evaluates u = (B (x) B (x) B) x, scales it by beta w detJ and adds its
// transpose (kernels in k_apply_impl.cuh).
#include "k_apply_impl.cuh"

cudaError_t lor_apply_mass_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                    const double* x, double* y, cudaStream_t s) {
  return apply_dispatch<true, false, double>(m, T, Dq, Mq, x, y, s);
}

cudaError_t lor_backward_mass_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                       const double* kappa, const double* x, const double* gy, double* gx,
                                       double* gk, cudaStream_t s) {
  return backward_dispatch<true, false>(m, T, Dq, Mq, kappa, x, gy, gx, gk, s);
}

// k_pattern.cu -- Step S1.2 / A2: CSR sparsity of the LOR matrix.
//
// The paper builds the processor-local CSR by counting the nonzeros of each
// row from the macro-element blocks (keeping only the contribution of the
// lowest-numbered macro element that holds a DOF), scanning the counts into
// the row pointer, and filling the column indices.  On a structured grid of
// macro elements every count is known in closed form (2 or 3 couplings per
// axis), so one thread per row writes its row pointer and its sorted columns
// directly: no atomics, no scan, and rows are independent.
#include "lor_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_pattern(int64_t nx, int64_t ny, int64_t nz, int64_t* __restrict__ rowptr,
                                                 int32_t* __restrict__ colidx) {
  const int64_t n = nx * ny * nz;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = r % nx, J = (r / nx) % ny, K = r / (nx * ny);
    int64_t pos = lor_row_start(I, J, K, nx, ny, nz);
    rowptr[r] = pos;
    if (r == n - 1) rowptr[n] = (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2);
    for (int dk = -1; dk <= 1; ++dk) {
      const int64_t K2 = K + dk;
      if (K2 < 0 || K2 >= nz) continue;
      for (int dj = -1; dj <= 1; ++dj) {
        const int64_t J2 = J + dj;
        if (J2 < 0 || J2 >= ny) continue;
        for (int di = -1; di <= 1; ++di) {
          const int64_t I2 = I + di;
          if (I2 < 0 || I2 >= nx) continue;
          colidx[pos++] = (int32_t)(I2 + nx * (J2 + ny * K2));
        }
      }
    }
  }
}

}  // namespace

cudaError_t lor_launch_pattern(const LorMesh& m, int64_t* rowptr, int32_t* colidx, cudaStream_t s) {
  const int64_t blocks = (m.ndof + 255) / 256;
  const int g = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
  k_pattern<<<g, 256, 0, s>>>(m.nx, m.ny, m.nz, rowptr, colidx); lor_count_launch();
  return cudaGetLastError();
}

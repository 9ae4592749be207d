// lor_internal.cuh -- shared definitions of the liblor CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lor.h"

#define LOR_MAX_Q (LOR_MAX_P + 2)
#define LOR_MAX_N (LOR_MAX_P + 1)

// 1D tables of one (p, q = p+2) space, built on the host (lor_abi.cu) and
// passed to kernels by value (kernel parameter space).
struct LorTables {
  int p, q, n;                          // n = p + 1
  double B[LOR_MAX_Q * LOR_MAX_N];      // B_1D[g][i] = l_i(xg_g)   (q x n)
  double Dm[LOR_MAX_Q * LOR_MAX_N];     // D_1D[g][i] = l_i'(xg_g)  (q x n)
  double gx[LOR_MAX_Q];                 // Gauss-Legendre points
  double gw[LOR_MAX_Q];                 // Gauss-Legendre weights
  double gll[LOR_MAX_N];                // Gauss-Lobatto nodes
  // LOR sub-hexes: interval a = [gll[a], gll[a+1]] of each axis
  double sub_r[LOR_MAX_P];              // half width (gll[a+1]-gll[a])/2
  double sub_t[2 * LOR_MAX_P];          // element reference coordinate of the 2 Gauss points of each interval
  double sub_l0[2 * LOR_MAX_P];         // (1 - t)/2 at the 2 Gauss points of each interval
  double sub_l1[2 * LOR_MAX_P];         // (1 + t)/2 at the same points
  int bin_first[LOR_MAX_P];             // high-order Gauss points of interval a:
  int bin_count[LOR_MAX_P];             //   g = bin_first[a] .. bin_first[a]+bin_count[a]-1
  double bin_w[LOR_MAX_Q];              // w_g / sum_{g' in bin(g)} w_g'
};

struct LorMesh {
  int nex, ney, nez, p;
  int64_t nx, ny, nz;   // DOFs per axis
  int64_t ndof, nel, nnz;
  const double* verts;  // device [(nex+1)(ney+1)(nez+1)][3]
};

struct lor_ctx {
  lor_config cfg;
  LorMesh m;
  LorTables T;
  int device;
  std::string err;
  // owned device buffers
  double* verts = nullptr;
  double* Dq = nullptr;        // [nel][6][q^3]: kappa w detJ J^-1 J^-T (00,01,02,11,12,22)
  double* kappa = nullptr;     // [nel][q^3]
  int64_t* rowptr = nullptr;   // [N+1]
  int32_t* colidx = nullptr;   // [nnz]
  double* vals64 = nullptr;    // [nnz]
  float* vals32 = nullptr;     // [nnz]
  int* d_status = nullptr;     // device error flags
  bool have_coeff = false, have_pattern = false, have_vals64 = false, have_vals32 = false;
  // preconditioner
  int pc_kind = LOR_PRECOND_NONE, pc_dtype = LOR_F64, pc_degree = 1;
  double pc_lo = 0, pc_hi = 0, pc_lmax = 0;
  double* dinv64 = nullptr;    // [N]
  float* dinv32 = nullptr;     // [N]
  void* pc_work = nullptr;     // 3 vectors of the smoother dtype
  // PCG work
  double* pcg_work = nullptr;  // r, z, p, Ap: 4 N
  double* red = nullptr;       // reduction partials + scalars
  double* h_scalar = nullptr;  // pinned host scalars
};

// Process-wide count of kernels launched by liblor (reported by lor_launch_count).
void lor_count_launch();

// Device error flags (bit mask in ctx->d_status[0]).
#define LOR_FLAG_BAD_KAPPA 1
#define LOR_FLAG_BAD_GEOM 2

// Number of CTAs used by the reduction kernels (multiple of the 152 SMs).
#define LOR_RED_BLOCKS 608
#define LOR_RED_THREADS 256

// -------------------------------------------------------------------------
// Closed-form CSR positions of the LOR pattern.  On the structured
// macro-element grid the number of nonzeros of row (I,J,K) is
// cx(I) cy(J) cz(K), c(I) = 2 at the two ends of an axis and 3 inside, so
// prefix sums (row pointers) and the rank of a column inside its row follow
// arithmetically; no position table is read.
// -------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t lor_axis_count(int64_t I, int64_t n) {
  return (I == 0 || I == n - 1) ? 2 : 3;
}
__host__ __device__ __forceinline__ int64_t lor_axis_prefix(int64_t I) {
  return I == 0 ? 0 : 3 * I - 1;
}
__host__ __device__ __forceinline__ int64_t lor_row_start(int64_t I, int64_t J, int64_t K, int64_t nx, int64_t ny,
                                                          int64_t nz) {
  const int64_t Sx = 3 * nx - 2, Sy = 3 * ny - 2;
  const int64_t cz = lor_axis_count(K, nz), cy = lor_axis_count(J, ny);
  return lor_axis_prefix(K) * Sy * Sx + cz * lor_axis_prefix(J) * Sx + cz * cy * lor_axis_prefix(I);
}
// Position of entry (row (I,J,K), column (I+di, J+dj, K+dk)), |d*| <= 1 and in range.
__host__ __device__ __forceinline__ int64_t lor_entry_pos(int64_t I, int64_t J, int64_t K, int di, int dj, int dk,
                                                          int64_t nx, int64_t ny, int64_t nz) {
  const int64_t cx = lor_axis_count(I, nx), cy = lor_axis_count(J, ny);
  const int64_t rx = di + (I > 0 ? 1 : 0), ry = dj + (J > 0 ? 1 : 0), rz = dk + (K > 0 ? 1 : 0);
  return lor_row_start(I, J, K, nx, ny, nz) + (rz * cy + ry) * cx + rx;
}
__host__ __device__ __forceinline__ bool lor_is_essential(int64_t I, int64_t J, int64_t K, int64_t nx, int64_t ny,
                                                          int64_t nz) {
  return I == 0 || J == 0 || K == 0 || I == nx - 1 || J == ny - 1 || K == nz - 1;
}

// -------------------------------------------------------------------------
// Host-side launchers (defined in the k_*.cu files).  Each returns a
// cudaError_t from the launch.
// -------------------------------------------------------------------------
cudaError_t lor_launch_geometry_check(const LorMesh& m, const LorTables& T, int* d_status, cudaStream_t s);
cudaError_t lor_launch_setup(const LorMesh& m, const LorTables& T, const double* kappa_in, double* kappa_copy,
                             double* Dq, int* d_status, cudaStream_t s);
cudaError_t lor_launch_load_vector(const LorMesh& m, const LorTables& T, const double* f, double* b,
                                   cudaStream_t s);
cudaError_t lor_launch_pattern(const LorMesh& m, int64_t* rowptr, int32_t* colidx, cudaStream_t s);
cudaError_t lor_launch_assemble(const LorMesh& m, const LorTables& T, const double* kappa, void* values,
                                int dtype, cudaStream_t s);
cudaError_t lor_launch_apply(const LorMesh& m, const LorTables& T, const double* Dq, const double* x, double* y,
                             cudaStream_t s);
cudaError_t lor_launch_apply_backward(const LorMesh& m, const LorTables& T, const double* Dq, const double* kappa,
                                      const double* x, const double* gy, double* gx, double* gkappa,
                                      cudaStream_t s);
// sparse / solver kernels (k_sparse.cu)
cudaError_t lor_launch_diag_inv(const LorMesh& m, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                                int dtype, void* dinv, cudaStream_t s);
cudaError_t lor_launch_spmv(const LorMesh& m, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                            int dtype, const double* x, double* y, cudaStream_t s);
int lor_precond_apply_impl(lor_ctx* c, const double* r, double* z, cudaStream_t s);
int lor_power_iteration(lor_ctx* c, int dtype, int iters, const double* v0, double* lambda, cudaStream_t s);
int lor_pcg_impl(lor_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
                 cudaStream_t s);

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
  double sub_rinv[LOR_MAX_P];           // 1 / sub_r
  double sub_t[2 * LOR_MAX_P];          // element reference coordinate of the 2 Gauss points of each interval
  double sub_l0[2 * LOR_MAX_P];         // (1 - t)/2 at the 2 Gauss points of each interval
  double sub_l1[2 * LOR_MAX_P];         // (1 + t)/2 at the same points
  double gl0[LOR_MAX_Q];                // (1 - x_g)/2 at the high-order Gauss points
  double gl1[LOR_MAX_Q];                // (1 + x_g)/2
  int bin_first[LOR_MAX_P];             // high-order Gauss points of interval a:
  int bin_count[LOR_MAX_P];             //   g = bin_first[a] .. bin_first[a]+bin_count[a]-1
  double bin_w[LOR_MAX_Q];              // w_g / sum_{g' in bin(g)} w_g'
};

struct LorMesh {
  int nex, ney, nez, p;
  int64_t nx, ny, nz;   // DOFs per axis
  int64_t ndof, nel, nnz;
  const double* verts;  // device [(nex+1)(ney+1)(nez+1)][3]
  // General conforming hex mesh (the element-restriction form; NULL on the
  // structured unit-cube grid): element corners [nel][8][3] (corner
  // c0 + 2 c1 + 4 c2), element-to-DOF map [nel][(p+1)^3] (node i + n(j + n k)),
  // essential-DOF mask [ndof], and the LOR CSR pattern built from the map.
  const double* ecorners = nullptr;
  const int64_t* edofs = nullptr;
  const uint8_t* ess = nullptr;
  const int64_t* rowptr = nullptr;
  const int32_t* colidx = nullptr;
  unsigned test_flags = 0;  // lor_set_test_hooks (LOR_TEST_EXPIRE_WAITS)
};

struct lor_ctx {
  lor_config cfg;
  LorMesh m;
  LorTables T;
  int device;
  std::string err;
  size_t device_bytes = 0;  // held by the buffers below (allocated through alloc())
  // owned device buffers
  double* verts = nullptr;
  double* Dq = nullptr;        // kappa w detJ J^-1 J^-T (00,01,02,11,12,22) in fixed point: [nel][6][q^3] packed + [nel][q^3] scales (fixed_point.cuh)
  double* kappa = nullptr;     // [nel][q^3]
  double* beta = nullptr;      // [nel][q^3] reaction coefficient (copy), when set
  double* Mq = nullptr;        // [nel][q^3] beta w detJ, when set
  int64_t* rowptr = nullptr;   // [N+1]
  int32_t* colidx = nullptr;   // [nnz]
  double* vals64 = nullptr;    // [nnz]
  float* vals32 = nullptr;     // [nnz]
  int* d_status = nullptr;     // device error flags
  bool have_coeff = false, have_pattern = false, have_vals64 = false, have_vals32 = false;
  bool have_beta = false;      // the reaction term is on (lor_set_reaction)
  bool general = false;        // created by lor_create_general (element-restriction mesh)
  double* ecorners = nullptr;  // general: [nel][8][3]
  int64_t* edofs = nullptr;    // general: [nel][(p+1)^3]
  uint8_t* ess = nullptr;      // general: [ndof]
  int32_t* etail = nullptr;    // general: LOR edges (built on the first discrete-gradient call)
  int32_t* ehead = nullptr;
  int64_t nedge = -1;
  // preconditioner
  int pc_kind = LOR_PRECOND_NONE, pc_dtype = LOR_F64, pc_degree = 1;
  double pc_lo = 0, pc_hi = 0, pc_lmax = 0;
  double* dinv64 = nullptr;    // [N]
  float* dinv32 = nullptr;     // [N]
  void* pc_work = nullptr;     // 3 vectors of the smoother dtype
  // PCG work
  double* pcg_work = nullptr;  // r, z, p, Ap: 4 N
  double* red = nullptr;       // reduction partials (LOR_RED_BLOCKS), 16 scalars, 2 x LOR_PCG_MAX_BLOCKS fused-PCG partials
  unsigned* red_count = nullptr;  // arrival counters of the last-block reductions (kept at 0 between uses)
  double* h_scalar = nullptr;  // pinned host scalars
  // FP32 copies of the operator factors for the FP32 apply (made on first use
  // after the coefficient or reaction term changes) and the refinement's
  // outer residual and correction (2 N)
  float* Dq32 = nullptr;
  float* Mq32 = nullptr;
  bool have_d32 = false;
  double* ir_work = nullptr;
};

// Process-wide count of kernels launched by liblor (reported by lor_launch_count).
void lor_count_launch();

// Device error flags (bit mask in ctx->d_status[0]).
#define LOR_FLAG_BAD_KAPPA 1
#define LOR_FLAG_BAD_GEOM 2
#define LOR_FLAG_TIMEOUT 4  // a bounded wait on an mbarrier expired (a TMA copy never completed)
#define LOR_FLAG_BAD_PATTERN 8  // the unstructured assembly met a coupling missing from the given CSR pattern
#define LOR_FLAG_BAD_MAP 16  // a general mesh's element-to-DOF map is out of range (or a vertex valence above 64)

// Elements of padding after the nnz CSR values of the context's value arrays
// (a tile's bulk copy may end up to 15 bytes past the last value).
#define LOR_VALS_PAD 4

// Number of CTAs used by the reduction kernels (multiple of the 152 SMs).
#define LOR_RED_BLOCKS 608
#define LOR_PCG_MAX_BLOCKS 2048  // grid cap of the fused PCG reductions (two partials per CTA)
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

// Essential (Dirichlet) DOF: the mask of a general mesh, else the boundary of
// the structured grid.
__host__ __device__ __forceinline__ bool lor_dof_essential(const LorMesh& m, int64_t r) {
  if (m.ess) return m.ess[r] != 0;
  const int64_t I = r % m.nx, J = (r / m.nx) % m.ny, K = r / (m.nx * m.ny);
  return lor_is_essential(I, J, K, m.nx, m.ny, m.nz);
}

// Position of column col in the sorted CSR row segment [b, e) (-1 if absent).
__device__ __forceinline__ int64_t lor_find_col(const int32_t* __restrict__ colidx, int64_t b, int64_t e,
                                                int64_t col) {
  while (b < e) {
    const int64_t mid = (b + e) >> 1;
    const int64_t v = colidx[mid];
    if (v == col) return mid;
    if (v < col) b = mid + 1;
    else e = mid;
  }
  return -1;
}

// -------------------------------------------------------------------------
// Device helpers shared by the geometry and assembly kernels.
// -------------------------------------------------------------------------
// Corner c = c0 + 2 c1 + 4 c2 of element e.
__device__ __forceinline__ void lor_element_corner(const LorMesh& m, int64_t e, int c, double X[3]) {
  if (m.ecorners) {
    const double* v = m.ecorners + (e * 8 + c) * 3;
    X[0] = v[0];
    X[1] = v[1];
    X[2] = v[2];
    return;
  }
  const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
  const int64_t a = ex + (c & 1), b = ey + ((c >> 1) & 1), cc = ez + ((c >> 2) & 1);
  const double* v = m.verts + 3 * (a + (int64_t)(m.nex + 1) * (b + (int64_t)(m.ney + 1) * cc));
  X[0] = v[0];
  X[1] = v[1];
  X[2] = v[2];
}

// Tabulate the three Jacobian columns of the trilinear map of element e on
// the tensor grid of L reference coordinates t[0..L), given the bilinear
// weights w0[i] = (1 - t_i)/2, w1[i] = (1 + t_i)/2:
//   col[d][u + L v][comp], with (u, v) the two coordinates other than d, in
//   increasing axis order.  E.g. col[0][g1 + L g2] = dx/dxi_0 at (., t_g1, t_g2).
// dx/dxi_d = sum over the 4 edges along d of w(t_u) w(t_v) (X_hi - X_lo)/2,
// evaluated separably (2 FP64 operations per table entry).
// Cooperative over the block; ends with __syncthreads().
__device__ __forceinline__ void lor_jacobian_columns(const LorMesh& m, int64_t e, const double* w0, const double* w1,
                                                     int L, double* Ehalf, double* col) {
  // Ehalf[d][pair][comp]: half edge vectors along axis d for the 4 edges
  // parallel to it; pair = (other0 bit) + 2 (other1 bit).
  for (int idx = threadIdx.x; idx < 36; idx += blockDim.x) {
    const int d = idx / 12, pair = (idx / 3) % 4, comp = idx % 3;
    const int o0 = pair & 1, o1 = pair >> 1;
    int lo = 0, hi = 0;
    if (d == 0) { lo = 0 + 2 * o0 + 4 * o1; hi = lo + 1; }
    if (d == 1) { lo = o0 + 0 + 4 * o1; hi = lo + 2; }
    if (d == 2) { lo = o0 + 2 * o1 + 0; hi = lo + 4; }
    double A[3], Bv[3];
    lor_element_corner(m, e, lo, A);
    lor_element_corner(m, e, hi, Bv);
    Ehalf[idx] = 0.5 * (Bv[comp] - A[comp]);
  }
  __syncthreads();
  const int L2 = L * L;
  for (int idx = threadIdx.x; idx < 9 * L; idx += blockDim.x) {
    const int d = idx / (3 * L), u = (idx / 3) % L, comp = idx % 3;
    const double* E = Ehalf + d * 12 + comp;
    const double a = w0[u] * E[0] + w1[u] * E[3];  // v-bit 0 edges, interpolated in u
    const double b = w0[u] * E[6] + w1[u] * E[9];  // v-bit 1 edges
    double* cd = col + d * L2 * 3 + comp;
    for (int v = 0; v < L; ++v) cd[3 * (u + L * v)] = w0[v] * a + w1[v] * b;
  }
  __syncthreads();
}

// Adjugate rows of J = [c0 c1 c2]: a0 = c1 x c2, a1 = c2 x c0, a2 = c0 x c1;
// J^-1 has rows a_i / det, det = c0 . a0.
__device__ __forceinline__ void lor_cross(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

// Reciprocal by Newton-Raphson iteration r <- r + r (1 - x r) from an FP32
// seed (24 correct bits); each step doubles the correct bits, two steps
// reach FP64 precision (within 1 ulp).  Valid for |x| in the FP32 range.
__device__ __forceinline__ double lor_rcp(double x) {
  double r = (double)(1.0f / (float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/sqrt(x) in FP64 for any normal x > 0.  x = 4^k m with m in [1, 4)
// (exponent-field arithmetic, exact), an FP32 seed for 1/sqrt(m) (m's
// leading 20 mantissa bits, the hardware rsqrt approximation: about 20
// correct bits), one Newton step with its second-order term,
// y (1 + e/2 + 3 e^2/8) with e = 1 - m y^2 (the error left is O(e^3), below
// FP64 rounding), and the exact scaling by 2^-k.  Within 1.3 ulp in a CPU
// emulation over 1e-300 .. 1e300.  The FP64 <-> FP32 moves and the scalings
// are integer bit operations, since the conversion instructions issue on the
// FP64 pipe.  Five FP64 operations.
__device__ __forceinline__ double lor_rsqrt(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int k = (((hi >> 20) & 0x7FF) - 1023) >> 1;  // floor(unbiased exponent / 2)
  const double m = __hiloint2double(hi - 2 * k * (1 << 20), lo);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__int_as_float((__double2hiint(m) - (896 << 20)) << 3)));
  const int yb = __float_as_int(yf);
  const double y = __hiloint2double((yb >> 3) + (896 << 20), yb << 29);
  const double t = m * y;
  const double e = fma(-t, y, 1.0);
  const double r = fma(y * e, fma(0.375, e, 0.5), y);  // 1/sqrt(m), in (1/2, 1]
  return __hiloint2double(__double2hiint(r) - k * (1 << 20), __double2loint(r));
}

// -------------------------------------------------------------------------
// Host-side launchers (defined in the k_*.cu files).  Each returns a
// cudaError_t from the launch.
// -------------------------------------------------------------------------
cudaError_t lor_launch_geometry_check(const LorMesh& m, const LorTables& T, int* d_status, cudaStream_t s);
cudaError_t lor_launch_setup(const LorMesh& m, const LorTables& T, const double* kappa_in, double* kappa_copy,
                             double* Dq, int* d_status, cudaStream_t s);
// Mq = beta w detJ at every Gauss point and a copy of beta (checked finite > 0).
cudaError_t lor_launch_reaction_setup(const LorMesh& m, const LorTables& T, const double* beta_in, double* beta_copy,
                                      double* Mq, int* d_status, cudaStream_t s);
cudaError_t lor_launch_load_vector(const LorMesh& m, const LorTables& T, const double* f, double* b,
                                   cudaStream_t s);
cudaError_t lor_launch_pattern(const LorMesh& m, int64_t* rowptr, int32_t* colidx, cudaStream_t s);
// beta (may be NULL): the reaction coefficient; adds the LOR mass blocks.
cudaError_t lor_launch_assemble(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta,
                                void* values, int dtype, cudaStream_t s);
// Mq (may be NULL): beta w detJ at the Gauss points, the reaction term.
cudaError_t lor_launch_apply(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                             const double* x, double* y, cudaStream_t s);
// The apply without its output initialisation: adds A_free x into y (y must
// already hold x on essential DOFs and 0 elsewhere).
cudaError_t lor_launch_apply_accumulate(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                        const double* x, double* y, cudaStream_t s);
// The apply in FP32 arithmetic (FP32 tables and D / M factors, FP64 x and y
// with FP64 atomics), with and without the output initialisation.
cudaError_t lor_launch_apply_f32(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                 const double* x, double* y, cudaStream_t s);
cudaError_t lor_launch_apply_f32_accumulate(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                            const double* x, double* y, cudaStream_t s);
// ... and with FP32 x and y (FP32 atomics; y initialised by the caller).
cudaError_t lor_launch_apply_f32v_accumulate(const LorMesh& m, const LorTables& T, const float* Dq, const float* Mq,
                                             const float* x, float* y, cudaStream_t s);
// b = (float) a, n elements
cudaError_t lor_launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
// FP32 copy of the setup's fixed-point D (6 nq floats, [e][c][q^3])
cudaError_t lor_launch_d_to_f32(const LorMesh& m, const double* Dq, float* out, cudaStream_t s);
cudaError_t lor_launch_apply_backward(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                                      const double* kappa, const double* x, const double* gy, double* gx,
                                      double* gkappa, cudaStream_t s);
// unstructured assembly (k_unstructured.cu)
cudaError_t lor_launch_lor_mesh(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta,
                                double* corners, int64_t* dofs, double* ksub, double* bsub, uint8_t* ess,
                                cudaStream_t s);
cudaError_t lor_launch_assemble_unstructured(int64_t nsub, const double* corners, const int64_t* dofs,
                                             const double* ksub, const double* bsub, int64_t n, int64_t nnz,
                                             const int64_t* rowptr, const int32_t* colidx, const uint8_t* ess,
                                             void* vals, int dtype, int* status, cudaStream_t s);
// The context's device allocator, handed to the general-mesh builders so that
// their temporaries and results count against the same budget as the
// context's own buffers (LOR_DEVICE_ALLOC_LIMIT): alloc fails with
// cudaErrorMemoryAllocation past the limit without calling the runtime;
// release frees a block and uncounts its bytes.
struct LorDeviceAlloc {
  void* ctx;
  cudaError_t (*alloc)(void* ctx, void** p, size_t bytes);
  void (*release)(void* ctx, void* p, size_t bytes);
};
// general meshes (k_general.cu): LOR pattern from the element-to-DOF map
// (allocates *rowptr and *colidx through A, sets *nnz; synchronises), map
// validation
cudaError_t lor_general_pattern(const LorMesh& m, const LorDeviceAlloc& A, int64_t** rowptr, int32_t** colidx,
                                int64_t* nnz, int* d_status, cudaStream_t s);
// the LOR edges of a general mesh (tail < head, ordered by tail then head;
// allocates *tail and *head through A, synchronises), the discrete gradient
// from them, and the vertex coordinates through the map
cudaError_t lor_general_edges(const LorMesh& m, const LorDeviceAlloc& A, int32_t** tail, int32_t** head,
                              int64_t* nedge, int* d_status, cudaStream_t s);
cudaError_t lor_launch_general_gradient(int64_t nedge, const int32_t* tail, const int32_t* head, int64_t* rowptr,
                                        int32_t* colidx, double* values, cudaStream_t s);
cudaError_t lor_launch_general_vertices(const LorMesh& m, const LorTables& T, double* xyz, cudaStream_t s);
// H(curl) topology of the LOR mesh (k_hcurl.cu)
int64_t lor_edge_count(const LorMesh& m);
cudaError_t lor_launch_discrete_gradient(const LorMesh& m, int64_t* rowptr, int32_t* colidx, double* values,
                                         cudaStream_t s);
cudaError_t lor_launch_vertex_coordinates(const LorMesh& m, const LorTables& T, double* xyz, cudaStream_t s);
// sparse / solver kernels (k_sparse.cu)
// The SpMV-type kernels read the CSR values only: the columns and row starts
// of the 27-point LOR pattern are recomputed from the grid (the pattern
// lor_launch_pattern writes).  Value arrays must be 16-byte aligned and padded
// by LOR_VALS_PAD elements; a TMA wait that expires sets LOR_FLAG_TIMEOUT.
cudaError_t lor_launch_diag_inv(const LorMesh& m, const void* vals, int dtype, void* dinv, cudaStream_t s);
cudaError_t lor_launch_spmv(const LorMesh& m, const void* vals, int dtype, const double* x, double* y, int* status,
                            cudaStream_t s);
int lor_precond_apply_impl(lor_ctx* c, const double* r, double* z, cudaStream_t s);
int lor_power_iteration(lor_ctx* c, int dtype, int iters, const double* v0, double* lambda, cudaStream_t s);
int lor_pcg_impl(lor_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
                 cudaStream_t s);
// Mixed-precision iterative refinement around PCG (k_sparse.cu).
int lor_pcg_ir_impl(lor_ctx* c, const double* b, double* x, double rtol, double inner_rtol, int maxit, int scheme,
                    int* outer_iters, int* inner_iters, double* relres, cudaStream_t s);
// FP32 copies of D (and beta w detJ) for the FP32 apply, made when stale;
// the refinement's work vectors (lor_abi.cu).
int lor_ensure_f32_factors(lor_ctx* c, cudaStream_t s);
int lor_alloc_ir_work(lor_ctx* c);

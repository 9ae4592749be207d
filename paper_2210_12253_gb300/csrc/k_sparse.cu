// k_sparse.cu -- the solve phase on the assembled LOR matrix (Step S2.2's
// building blocks: spmv and vector updates) and the preconditioned CG of
// Section 3, step S2.
//
// The preconditioner B_h is a Chebyshev-Jacobi smoother on A_h (any uniform
// preconditioner of the LOR matrix preconditions A_p, Section 2.2).  Each
// Chebyshev step is one kernel: the CSR row product, the residual, the
// direction update and the iterate update are fused per row, so a degree-k
// smoother reads the matrix k-1 times and touches each vector once per step.
// In the mixed-precision mode the matrix, the diagonal and the smoother's
// vectors are FP32; PCG's vectors, dot products and recurrences stay FP64.
#include <math.h>

#include "lor_internal.cuh"

namespace {

constexpr int kThreads = 256;

int grid_rows(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 152 * 32 ? b : 152 * 32);
}

#define LOR_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// sum_j A_ij x_j in the matrix precision VT (x converted on the fly), with kLanes lanes per row: lane l takes entries
// rowptr[i] + l, + 2 kLanes, ... (consecutive lanes read consecutive
// entries, so a warp reads 32/kLanes row segments of kLanes entries per
// instruction) and the lanes combine by shuffles; every lane returns the sum.
// All 32 lanes of the warp must call it (rows past n pass valid = false).
constexpr int kLanes = 4;
template <typename VT, typename XT>
__device__ __forceinline__ VT row_product_lanes(const int64_t* __restrict__ rowptr,
                                                const int32_t* __restrict__ colidx, const VT* __restrict__ vals,
                                                const XT* __restrict__ x, int64_t i, bool valid) {
  VT s = 0;
  if (valid) {
    const int lane = threadIdx.x & (kLanes - 1);
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    for (int64_t j = b + lane; j < e; j += kLanes) s += vals[j] * (VT)x[colidx[j]];
  }
#pragma unroll
  for (int o = kLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// One (row, lane) per thread; the grid covers all rows exactly.
#define LOR_ROW_LANES(i, valid, n)                                                        \
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kLanes;            \
  const bool valid = i < (n);                                                             \
  const bool lead = valid && (threadIdx.x & (kLanes - 1)) == 0;

unsigned grid_row_lanes(int64_t n) { return (unsigned)((n * kLanes + kThreads - 1) / kThreads); }

template <typename VT>
__global__ void k_diag_inv(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           const VT* __restrict__ vals, VT* __restrict__ dinv) {
  LOR_GRID_STRIDE(i, n) {
    VT d = 0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j)
      if (colidx[j] == i) d += vals[j];
    dinv[i] = (VT)1 / d;
  }
}

template <typename VT>
__global__ void k_spmv(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                       const VT* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y) {
  LOR_ROW_LANES(i, valid, n)
  const VT s = row_product_lanes<VT, double>(rowptr, colidx, vals, x, i, valid);
  if (lead) y[i] = (double)s;
}

// w = D^-1 A v (power iteration), FP64 vectors, VT matrix.
template <typename VT>
__global__ void k_dinv_spmv(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                            const VT* __restrict__ vals, const VT* __restrict__ dinv, const double* __restrict__ v,
                            double* __restrict__ w) {
  LOR_ROW_LANES(i, valid, n)
  const VT s = row_product_lanes<VT, double>(rowptr, colidx, vals, v, i, valid);
  if (lead) w[i] = (double)(dinv[i] * s);
}

// Chebyshev step 0 from z_0 = 0: d = z = D^-1 r / theta.  If zout64 is set
// (degree 1) the result goes straight to the FP64 output.
template <typename VT>
__global__ void k_cheb_first(int64_t n, const VT* __restrict__ dinv, const double* __restrict__ r, VT inv_theta,
                             VT* __restrict__ z, VT* __restrict__ d, double* __restrict__ zout64) {
  LOR_GRID_STRIDE(i, n) {
    const VT v = dinv[i] * (VT)r[i] * inv_theta;
    if (zout64) {
      zout64[i] = (double)v;
    } else {
      z[i] = v;
      d[i] = v;
    }
  }
}

// Chebyshev step j >= 1:  res = r - A z_in;  d = c1 d + c2 D^-1 res;
// z_out = z_in + d (into zout64 as FP64 on the last step).
template <typename VT>
__global__ void k_cheb_step(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                            const VT* __restrict__ vals, const VT* __restrict__ dinv, const double* __restrict__ r,
                            const VT* __restrict__ zin, VT* __restrict__ zout, VT* __restrict__ d, VT c1, VT c2,
                            double* __restrict__ zout64) {
  LOR_ROW_LANES(i, valid, n)
  const VT az = row_product_lanes<VT, VT>(rowptr, colidx, vals, zin, i, valid);
  if (lead) {
    const VT res = (VT)r[i] - az;
    const VT dn = c1 * d[i] + c2 * dinv[i] * res;
    const VT zn = zin[i] + dn;
    if (zout64) {
      zout64[i] = (double)zn;
    } else {
      d[i] = dn;
      zout[i] = zn;
    }
  }
}

__global__ void k_fill(double* __restrict__ v, int64_t n, double a) {
  LOR_GRID_STRIDE(i, n) v[i] = a;
}

__global__ void k_scale(double* __restrict__ v, int64_t n, double a) {
  LOR_GRID_STRIDE(i, n) v[i] *= a;
}

template <typename VT>
__global__ void k_jacobi(int64_t n, const VT* __restrict__ dinv, const double* __restrict__ r,
                         double* __restrict__ z) {
  LOR_GRID_STRIDE(i, n) z[i] = (double)(dinv[i] * (VT)r[i]);
}

// ---------------------------------------------------------------- reductions
// Block partial sums of a.b into partial[blockIdx.x] (fixed grid, fixed
// order: the result is deterministic).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += warp_part[w];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(kThreads) k_dot_partial(int64_t n, const double* __restrict__ a,
                                                          const double* __restrict__ b,
                                                          double* __restrict__ partial) {
  double s = 0.0;
  LOR_GRID_STRIDE(i, n) s += a[i] * b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_reduce_final(const double* __restrict__ partial, int np,
                                                           double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- PCG vector kernels
// Device scalars (slots of ctx->red after the partials).
enum { S_PQ = 0, S_RR = 1, S_BB = 2, S_RZ0 = 3, S_RZ1 = 4, S_COUNT = 5 };

__global__ void k_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ Ax,
                           double* __restrict__ r) {
  LOR_GRID_STRIDE(i, n) r[i] = b[i] - Ax[i];
}

template <typename VT>
cudaError_t precond_apply_t(lor_ctx* c, const VT* vals, const VT* dinv, const double* r, double* z,
                            cudaStream_t s) {
  const int64_t n = c->m.ndof;
  const int g = grid_rows(n);
  if (c->pc_kind == LOR_PRECOND_JACOBI) {
    k_jacobi<VT><<<g, kThreads, 0, s>>>(n, dinv, r, z); lor_count_launch();
    return cudaGetLastError();
  }
  VT* zA = (VT*)c->pc_work;
  VT* zB = zA + n;
  VT* d = zB + n;
  const double theta = 0.5 * (c->pc_hi + c->pc_lo), delta = 0.5 * (c->pc_hi - c->pc_lo);
  const double sigma = theta / delta;
  const int k = c->pc_degree;
  k_cheb_first<VT><<<g, kThreads, 0, s>>>(n, dinv, r, (VT)(1.0 / theta), zA, d, k == 1 ? z : nullptr); lor_count_launch();
  double rho = 1.0 / sigma;
  VT* zin = zA;
  VT* zout = zB;
  for (int j = 1; j < k; ++j) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
    k_cheb_step<VT><<<grid_row_lanes(n), kThreads, 0, s>>>(n, c->rowptr, c->colidx, vals, dinv, r, zin, zout, d, (VT)c1, (VT)c2,
                                          j == k - 1 ? z : nullptr); lor_count_launch();
    rho = rho_new;
    VT* t = zin;
    zin = zout;
    zout = t;
  }
  return cudaGetLastError();
}

cudaError_t dot_to(lor_ctx* c, const double* a, const double* b, double* out, cudaStream_t s) {
  k_dot_partial<<<LOR_RED_BLOCKS, kThreads, 0, s>>>(c->m.ndof, a, b, c->red); lor_count_launch();
  k_reduce_final<<<1, kThreads, 0, s>>>(c->red, LOR_RED_BLOCKS, out); lor_count_launch();
  return cudaGetLastError();
}

int fail(lor_ctx* c, cudaError_t err, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(err);
  return LOR_ECUDA;
}

}  // namespace

cudaError_t lor_launch_diag_inv(const LorMesh& m, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                                int dtype, void* dinv, cudaStream_t s) {
  if (dtype == LOR_F64) {
    k_diag_inv<double><<<grid_rows(m.ndof), kThreads, 0, s>>>(m.ndof, rowptr, colidx, (const double*)vals,
                                                             (double*)dinv); lor_count_launch();
  } else {
    k_diag_inv<float><<<grid_rows(m.ndof), kThreads, 0, s>>>(m.ndof, rowptr, colidx, (const float*)vals,
                                                            (float*)dinv); lor_count_launch();
  }
  return cudaGetLastError();
}

cudaError_t lor_launch_spmv(const LorMesh& m, const int64_t* rowptr, const int32_t* colidx, const void* vals,
                            int dtype, const double* x, double* y, cudaStream_t s) {
  if (dtype == LOR_F64) {
    k_spmv<double><<<grid_row_lanes(m.ndof), kThreads, 0, s>>>(m.ndof, rowptr, colidx, (const double*)vals, x, y); lor_count_launch();
  } else {
    k_spmv<float><<<grid_row_lanes(m.ndof), kThreads, 0, s>>>(m.ndof, rowptr, colidx, (const float*)vals, x, y); lor_count_launch();
  }
  return cudaGetLastError();
}

int lor_precond_apply_impl(lor_ctx* c, const double* r, double* z, cudaStream_t s) {
  cudaError_t err;
  if (c->pc_kind == LOR_PRECOND_NONE) {
    err = cudaMemcpyAsync(z, r, sizeof(double) * c->m.ndof, cudaMemcpyDeviceToDevice, s);
  } else if (c->pc_dtype == LOR_F64) {
    err = precond_apply_t<double>(c, c->vals64, c->dinv64, r, z, s);
  } else {
    err = precond_apply_t<float>(c, c->vals32, c->dinv32, r, z, s);
  }
  return err == cudaSuccess ? LOR_OK : fail(c, err, "precond_apply");
}

int lor_power_iteration(lor_ctx* c, int dtype, int iters, const double* v0, double* lambda, cudaStream_t s) {
  const int64_t n = c->m.ndof;
  double* v = c->pcg_work;
  double* w = c->pcg_work + n;
  cudaError_t err;
  if (v0) {
    err = cudaMemcpyAsync(v, v0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  } else {
    k_fill<<<grid_rows(n), kThreads, 0, s>>>(v, n, 1.0); lor_count_launch();
    err = cudaGetLastError();
  }
  if (err != cudaSuccess) return fail(c, err, "power iteration");
  double* S = c->red + LOR_RED_BLOCKS;
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    if (dtype == LOR_F64) {
      k_dinv_spmv<double><<<grid_row_lanes(n), kThreads, 0, s>>>(n, c->rowptr, c->colidx, c->vals64, c->dinv64, v, w); lor_count_launch();
    } else {
      k_dinv_spmv<float><<<grid_row_lanes(n), kThreads, 0, s>>>(n, c->rowptr, c->colidx, c->vals32, c->dinv32, v, w); lor_count_launch();
    }
    dot_to(c, w, w, S + 0, s);
    dot_to(c, v, v, S + 1, s);
    err = cudaMemcpyAsync(c->h_scalar, S, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return fail(c, err, "power iteration");
    const double nw = sqrt(c->h_scalar[0]), nv = sqrt(c->h_scalar[1]);
    if (!(nw > 0.0) || !(nv > 0.0)) {
      c->err = "power iteration: zero vector";
      return LOR_EINVAL;
    }
    lam = nw / nv;
    // v = w / |w|
    double* tmp = v;
    v = w;
    w = tmp;
    k_scale<<<grid_rows(n), kThreads, 0, s>>>(v, n, 1.0 / nw); lor_count_launch();
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(c, err, "power iteration");
  }
  *lambda = lam;
  return LOR_OK;
}

namespace {

// ---------------------------------------------------------------- fused PCG kernels
// Each dot product finishes in the last CTA to arrive (arrival counted with
// an atomic after a fence; that CTA sums the per-CTA partials in index order,
// so the result does not depend on which CTA finishes last, and resets the
// counter).  No CTA waits for another.
__device__ __forceinline__ void finish_sums(double s0, double s1, int nsum, double* __restrict__ partial,
                                            unsigned* __restrict__ counter, double* __restrict__ out0,
                                            double* __restrict__ out1) {
  __shared__ bool last;
  s0 = block_sum(s0);
  if (nsum > 1) s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    if (nsum > 1) partial[gridDim.x + blockIdx.x] = s1;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const volatile double* vp = partial;
  double t0 = 0.0, t1 = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    t0 += vp[i];
    if (nsum > 1) t1 += vp[gridDim.x + i];
  }
  t0 = block_sum(t0);
  if (nsum > 1) t1 = block_sum(t1);
  if (threadIdx.x == 0) {
    *out0 = t0;
    if (nsum > 1) *out1 = t1;
    *counter = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_pcg_dot(int64_t n, const double* __restrict__ a,
                                                      const double* __restrict__ b, double* __restrict__ partial,
                                                      unsigned* __restrict__ counter, double* __restrict__ out) {
  double s = 0.0;
  LOR_GRID_STRIDE(i, n) s += a[i] * b[i];
  finish_sums(s, 0.0, 1, partial, counter, out, nullptr);
}

// x += alpha p, r -= alpha q (alpha = rz / pq on the device), r.r, and the
// first step of the preconditioner on the updated r:
//   mode 0 (none): z = r;  mode 1 (Jacobi): z = D^-1 r;
//   mode 2 (Chebyshev, degree 1): z = D^-1 r / theta;
//   mode 3 (Chebyshev, degree >= 2): zA = d = D^-1 r / theta (smoother precision).
// Modes 0-2 also form r.z (z is final there).
template <typename VT>
__global__ void __launch_bounds__(kThreads) k_pcg_update(int64_t n, const double* __restrict__ S, int rz_slot,
                                                         const double* __restrict__ p, const double* __restrict__ q,
                                                         double* __restrict__ x, double* __restrict__ r, int mode,
                                                         const VT* __restrict__ dinv, VT inv_theta,
                                                         double* __restrict__ z, VT* __restrict__ zA,
                                                         VT* __restrict__ d, double* __restrict__ partial,
                                                         unsigned* __restrict__ counter, double* __restrict__ out_rr,
                                                         double* __restrict__ out_rz) {
  const double alpha = S[rz_slot] / S[S_PQ];
  double srr = 0.0, srz = 0.0;
  LOR_GRID_STRIDE(i, n) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    srr += ri * ri;
    if (mode == 0) {
      z[i] = ri;
      srz += ri * ri;
    } else if (mode == 1 || mode == 2) {
      const VT zi = mode == 1 ? dinv[i] * (VT)ri : dinv[i] * (VT)ri * inv_theta;
      z[i] = (double)zi;
      srz += ri * (double)zi;
    } else {
      const VT zi = dinv[i] * (VT)ri * inv_theta;
      zA[i] = zi;
      d[i] = zi;
    }
  }
  finish_sums(srr, srz, mode <= 2 ? 2 : 1, partial, counter, out_rr, out_rz);
}

// Last Chebyshev step fused with r.z: z = z_in + (c1 d + c2 D^-1 (r - A z_in))
// written as FP64, and the partial sums of r.z.  kLanes lanes per row; every
// warp runs the same number of row rounds so that its shuffles stay uniform.
template <typename VT>
__global__ void __launch_bounds__(kThreads) k_pcg_cheb_last(int64_t n, const int64_t* __restrict__ rowptr,
                                                            const int32_t* __restrict__ colidx,
                                                            const VT* __restrict__ vals, const VT* __restrict__ dinv,
                                                            const double* __restrict__ r,
                                                            const VT* __restrict__ zin, const VT* __restrict__ d,
                                                            VT c1, VT c2, double* __restrict__ z,
                                                            double* __restrict__ partial,
                                                            unsigned* __restrict__ counter, double* __restrict__ out) {
  const int64_t rows_per_round = (int64_t)gridDim.x * blockDim.x / kLanes;
  const int64_t warp_first = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / kLanes;
  const int group = (threadIdx.x & 31) / kLanes;
  double srz = 0.0;
  for (int64_t base = warp_first; base < n; base += rows_per_round) {
    const int64_t i = base + group;
    const bool valid = i < n;
    const VT az = row_product_lanes<VT, VT>(rowptr, colidx, vals, zin, i, valid);
    if (valid && (threadIdx.x & (kLanes - 1)) == 0) {
      const double ri = r[i];
      const VT zn = zin[i] + (c1 * d[i] + c2 * dinv[i] * ((VT)ri - az));
      z[i] = (double)zn;
      srz += ri * (double)zn;
    }
  }
  finish_sums(srz, 0.0, 1, partial, counter, out, nullptr);
}

// p = z + beta p (beta = rz_new / rz_old; first: p = z) and the output of
// the next apply initialised: q = p on essential DOFs, 0 elsewhere.
__global__ void k_pcg_direction(LorMesh m, const double* __restrict__ S, int new_slot, int old_slot, int first,
                                const double* __restrict__ z, double* __restrict__ p, double* __restrict__ q) {
  const double beta = first ? 0.0 : S[new_slot] / S[old_slot];
  LOR_GRID_STRIDE(i, m.ndof) {
    const double pi = first ? z[i] : z[i] + beta * p[i];
    p[i] = pi;
    const int64_t I = i % m.nx, J = (i / m.nx) % m.ny, K = i / (m.nx * m.ny);
    q[i] = lor_is_essential(I, J, K, m.nx, m.ny, m.nz) ? pi : 0.0;
  }
}

// two partial sums per CTA, after the scalars
double* pcg_partials(lor_ctx* c) { return c->red + LOR_RED_BLOCKS + 16; }

// Grid of a reducing PCG kernel: every SM filled to the kernel's occupancy
// (the loops are grid-stride), at most LOR_PCG_MAX_BLOCKS CTAs.
template <typename K>
int pcg_grid(K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
  const int g = sms * (per_sm > 0 ? per_sm : 1);
  return g < 1 ? 1 : g > LOR_PCG_MAX_BLOCKS ? LOR_PCG_MAX_BLOCKS : g;
}

template <typename VT>
cudaError_t pcg_precond_rest(lor_ctx* c, const VT* vals, const VT* dinv, const double* r, double* z,
                             double* out_rz, int grid, cudaStream_t s) {
  // Chebyshev steps 1 .. k-1 after k_pcg_update's step 0 (degree >= 2)
  const int64_t n = c->m.ndof;
  VT* zA = (VT*)c->pc_work;
  VT* zB = zA + n;
  VT* d = zB + n;
  const double theta = 0.5 * (c->pc_hi + c->pc_lo), delta = 0.5 * (c->pc_hi - c->pc_lo);
  const double sigma = theta / delta;
  const int k = c->pc_degree;
  double rho = 1.0 / sigma;
  VT* zin = zA;
  VT* zout = zB;
  for (int j = 1; j < k; ++j) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
    if (j < k - 1) {
      k_cheb_step<VT><<<grid_row_lanes(n), kThreads, 0, s>>>(n, c->rowptr, c->colidx, vals, dinv, r, zin, zout, d,
                                                            (VT)c1, (VT)c2, nullptr); lor_count_launch();
    } else {
      k_pcg_cheb_last<VT><<<grid, kThreads, 0, s>>>(n, c->rowptr, c->colidx, vals, dinv, r, zin, d, (VT)c1,
                                                        (VT)c2, z, pcg_partials(c), c->red_count, out_rz); lor_count_launch();
    }
    rho = rho_new;
    VT* t = zin;
    zin = zout;
    zout = t;
  }
  return cudaGetLastError();
}

template <typename VT>
cudaError_t pcg_update(lor_ctx* c, const VT* dinv, double* S, int cur, const double* p, const double* q, double* x,
                       double* r, double* z, int mode, double* out_rz, int grid, cudaStream_t s) {
  const double theta = 0.5 * (c->pc_hi + c->pc_lo);
  VT* zA = (VT*)c->pc_work;
  VT* d = zA ? zA + 2 * c->m.ndof : nullptr;
  k_pcg_update<VT><<<grid, kThreads, 0, s>>>(c->m.ndof, S, cur, p, q, x, r, mode, dinv,
                                                   (VT)(theta > 0 ? 1.0 / theta : 1.0), z, zA, d, pcg_partials(c),
                                                   c->red_count, S + S_RR, out_rz); lor_count_launch();
  return cudaGetLastError();
}

}  // namespace

int lor_pcg_impl(lor_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
                 cudaStream_t s) {
  const int64_t n = c->m.ndof;
  double* r = c->pcg_work;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* S = c->red + LOR_RED_BLOCKS;  // S[0] = p.q, S[1] = r.r, S[2] = b.b, S[3], S[4] = r.z (alternating)
  double* hs = c->h_scalar;
  const int g = grid_rows(n);
  const bool f64 = c->pc_dtype == LOR_F64;
  // preconditioner mode of the fused update (see k_pcg_update)
  const int mode = c->pc_kind == LOR_PRECOND_NONE ? 0 : c->pc_kind == LOR_PRECOND_JACOBI ? 1 : c->pc_degree == 1 ? 2 : 3;
  const int g_dot = pcg_grid(k_pcg_dot);
  const int g_upd = f64 ? pcg_grid(k_pcg_update<double>) : pcg_grid(k_pcg_update<float>);
  const int g_last = f64 ? pcg_grid(k_pcg_cheb_last<double>) : pcg_grid(k_pcg_cheb_last<float>);
  auto dot = [&](const double* a, const double* bb, double* out) {
    k_pcg_dot<<<g_dot, kThreads, 0, s>>>(n, a, bb, pcg_partials(c), c->red_count, out); lor_count_launch();
  };
  cudaError_t err = cudaMemsetAsync(x, 0, sizeof(double) * n, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (err == cudaSuccess) {
    dot(b, b, S + S_BB);
    err = cudaMemcpyAsync(hs, S + S_BB, sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return fail(c, err, "pcg");
  const double nb = sqrt(hs[0]);
  int it = 0;
  double rel = 0.0;
  int status = LOR_ENOCONV;
  if (nb == 0.0) {
    status = LOR_OK;
  } else {
    int rc = lor_precond_apply_impl(c, r, z, s);
    if (rc) return rc;
    int cur = S_RZ0;
    dot(r, z, S + cur);
    k_pcg_direction<<<g, kThreads, 0, s>>>(c->m, S, cur, cur, 1, z, p, q); lor_count_launch();
    while (it < maxit) {
      err = lor_launch_apply_accumulate(c->m, c->T, c->Dq, p, q, s);
      if (err != cudaSuccess) return fail(c, err, "pcg apply");
      dot(p, q, S + S_PQ);
      const int nxt = cur == S_RZ0 ? S_RZ1 : S_RZ0;
      err = f64 ? pcg_update<double>(c, c->dinv64, S, cur, p, q, x, r, z, mode, S + nxt, g_upd, s)
                : pcg_update<float>(c, c->dinv32, S, cur, p, q, x, r, z, mode, S + nxt, g_upd, s);
      if (err == cudaSuccess) err = cudaMemcpyAsync(hs, S + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err != cudaSuccess) return fail(c, err, "pcg");
      ++it;
      rel = sqrt(hs[0]) / nb;
      bool restarted = false;
      if (rel <= rtol) {
        // confirm on the true residual b - A x
        err = lor_launch_apply(c->m, c->T, c->Dq, x, q, s);
        if (err == cudaSuccess) {
          k_residual<<<g, kThreads, 0, s>>>(n, b, q, r); lor_count_launch();
          dot(r, r, S + S_RR);
          err = cudaMemcpyAsync(hs, S + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s);
        }
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return fail(c, err, "pcg");
        rel = sqrt(hs[0]) / nb;
        if (rel <= rtol) {
          status = LOR_OK;
          break;
        }
        // continue from the true residual: precondition it afresh
        rc = lor_precond_apply_impl(c, r, z, s);
        if (rc) return rc;
        dot(r, z, S + nxt);
        restarted = true;
      }
      if (!restarted && mode == 3) {
        err = f64 ? pcg_precond_rest<double>(c, c->vals64, c->dinv64, r, z, S + nxt, g_last, s)
                  : pcg_precond_rest<float>(c, c->vals32, c->dinv32, r, z, S + nxt, g_last, s);
        if (err != cudaSuccess) return fail(c, err, "pcg precond");
      }
      k_pcg_direction<<<g, kThreads, 0, s>>>(c->m, S, nxt, cur, 0, z, p, q); lor_count_launch();
      cur = nxt;
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(c, err, "pcg");
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (status == LOR_ENOCONV) c->err = "pcg: no convergence within maxit";
  return status;
}

// ---------------------------------------------------------------------------
// Preconditioner apply without device allocation.
//
// lor_precond_apply_noalloc gives the same result as lor_precond_apply, but
// the smoother's three work vectors live in the file-scope device array below
// instead of buffers the context allocated, so the call itself never asks the
// CUDA runtime for memory.  Some callers cannot allocate device memory at the
// point where they apply a preconditioner: a solver loop whose device memory
// is reserved up front by another allocator (cudaMalloc/cudaFree there would
// bypass it, and cudaFree can synchronise the whole device), or host code
// running where CUDA allocation calls are not allowed.  They can use this
// entry point once the context has been set up.
//
// The array is LOR_NOALLOC_SCRATCH_BYTES long; every GPU that loads the
// library holds it until the process exits.  A call needs 3 N elements of the
// smoother's precision (N = DOFs) and is rejected with LOR_EINVAL beyond that.
// All calls share the array and it keeps the last call's contents; every
// element a call reads is written by the same call first, so nothing has to
// start at zero.  Calls that overlap on the GPU (different streams, or two
// contexts) race on the array and must be ordered by the caller.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

static __device__ __align__(256) unsigned char lor_noalloc_scratch[LOR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of lor_noalloc_scratch on the current device (looked up once
// per device, with that device current; the host-side symbol itself is not a
// device address).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, lor_noalloc_scratch);
    if (err != cudaSuccess) return err;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

template <typename VT>
cudaError_t precond_apply_noalloc_t(lor_ctx* c, const VT* vals, const VT* dinv, const double* r, double* z,
                                    VT* work, cudaStream_t s) {
  const int64_t n = c->m.ndof;
  const int g = grid_rows(n);
  if (c->pc_kind == LOR_PRECOND_JACOBI) {
    k_jacobi<VT><<<g, kThreads, 0, s>>>(n, dinv, r, z); lor_count_launch();
    return cudaGetLastError();
  }
  VT* zA = work;
  VT* zB = zA + n;
  VT* d = zB + n;
  const double theta = 0.5 * (c->pc_hi + c->pc_lo), delta = 0.5 * (c->pc_hi - c->pc_lo);
  const double sigma = theta / delta;
  const int k = c->pc_degree;
  k_cheb_first<VT><<<g, kThreads, 0, s>>>(n, dinv, r, (VT)(1.0 / theta), zA, d, k == 1 ? z : nullptr); lor_count_launch();
  double rho = 1.0 / sigma;
  VT* zin = zA;
  VT* zout = zB;
  for (int j = 1; j < k; ++j) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
    k_cheb_step<VT><<<grid_row_lanes(n), kThreads, 0, s>>>(n, c->rowptr, c->colidx, vals, dinv, r, zin, zout, d, (VT)c1, (VT)c2,
                                          j == k - 1 ? z : nullptr); lor_count_launch();
    rho = rho_new;
    VT* t = zin;
    zin = zout;
    zout = t;
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" int lor_precond_apply_noalloc(lor_ctx* c, const double* d_r, double* d_z, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_r || !d_z || d_r == d_z) {
    c->err = "lor_precond_apply_noalloc: r, z must be distinct device arrays";
    return LOR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (c->pc_kind == LOR_PRECOND_NONE) {
    cudaError_t err = cudaMemcpyAsync(d_z, d_r, sizeof(double) * c->m.ndof, cudaMemcpyDeviceToDevice, s);
    return err == cudaSuccess ? LOR_OK : fail(c, err, "lor_precond_apply_noalloc");
  }
  const size_t elem = c->pc_dtype == LOR_F64 ? sizeof(double) : sizeof(float);
  const size_t need = 3 * (size_t)c->m.ndof * elem;
  if (c->pc_kind == LOR_PRECOND_CHEB && c->pc_degree > 1 && need > (size_t)LOR_NOALLOC_SCRATCH_BYTES) {
    c->err = "lor_precond_apply_noalloc: the smoother needs " + std::to_string(need) +
             " bytes of scratch but the static array holds " + std::to_string((size_t)LOR_NOALLOC_SCRATCH_BYTES) +
             " (use lor_precond_apply for this size)";
    return LOR_EINVAL;
  }
  void* work = nullptr;
  cudaError_t err = noalloc_scratch(&work);
  if (err != cudaSuccess) return fail(c, err, "lor_precond_apply_noalloc: scratch address");
  if (c->pc_dtype == LOR_F64)
    err = precond_apply_noalloc_t<double>(c, c->vals64, c->dinv64, d_r, d_z, (double*)work, s);
  else
    err = precond_apply_noalloc_t<float>(c, c->vals32, c->dinv32, d_r, d_z, (float*)work, s);
  return err == cudaSuccess ? LOR_OK : fail(c, err, "lor_precond_apply_noalloc");
}

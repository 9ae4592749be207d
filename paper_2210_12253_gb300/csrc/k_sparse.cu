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
// The mixed-precision refinement (lor_pcg_ir_impl) runs the same PCG with
// the FP32-arithmetic operator and forms every residual that decides
// convergence with the FP64 one.
#include <math.h>
#include <string.h>

#include <type_traits>

#include "lor_internal.cuh"

namespace {

constexpr int kThreads = 256;

int grid_rows(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 152 * 32 ? b : 152 * 32);
}

#define LOR_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Vectors of the solve are FP64, except in the refinement's inner
// iterations (V = float).  A thread's partial sums accumulate in the vector
// precision (a few dozen terms per thread) and the CTA and grid sums in FP64.
template <typename V>
using Acc = std::conditional_t<sizeof(V) == sizeof(float), float, double>;

// Chebyshev step 0 from z_0 = 0: d = z = D^-1 r / theta.  If zout64 is set
// (degree 1) the result goes straight to the FP64 output.
template <typename VT, typename V = double>
__global__ void k_cheb_first(int64_t n, const VT* __restrict__ dinv, const V* __restrict__ r, VT inv_theta,
                             VT* __restrict__ z, VT* __restrict__ d, V* __restrict__ zout64) {
  LOR_GRID_STRIDE(i, n) {
    const VT v = dinv[i] * (VT)r[i] * inv_theta;
    if (zout64) {
      zout64[i] = (V)v;
    } else {
      z[i] = v;
      d[i] = v;
    }
  }
}

__global__ void k_fill(double* __restrict__ v, int64_t n, double a) {
  LOR_GRID_STRIDE(i, n) v[i] = a;
}

__global__ void k_scale(double* __restrict__ v, int64_t n, double a) {
  LOR_GRID_STRIDE(i, n) v[i] *= a;
}

template <typename VT, typename V = double>
__global__ void k_jacobi(int64_t n, const VT* __restrict__ dinv, const V* __restrict__ r, V* __restrict__ z) {
  LOR_GRID_STRIDE(i, n) z[i] = (V)(dinv[i] * (VT)r[i]);
}

// ---------------------------------------------------------------- reductions
// Sum of v over the CTA (blockDim.x a multiple of 32, at most kThreads),
// returned in thread 0, in a fixed order: the result is deterministic.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += warp_part[w];
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

// Each dot product finishes in the last CTA to arrive (arrival counted with
// an atomic after a fence; that CTA sums the per-CTA partials in index order,
// so the result does not depend on which CTA finishes last, and resets the
// counter).  No CTA waits for another.  Returns true in the last CTA.
__device__ __forceinline__ bool finish_sums(double s0, double s1, int nsum, double* __restrict__ partial,
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
  if (!last) return false;
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
  return true;
}


// ---------------------------------------------------------------- the LOR pattern as a stencil
// The LOR matrix has the 27-point pattern of the GLL grid (Section 2.1):
// row i = (I, J, K) holds the columns (I+di, J+dj, K+dk), |d| <= 1, inside
// the grid, in increasing column order (dk slowest, di fastest), and its
// first value sits at lor_row_start(I, J, K).  lor_build_pattern writes
// exactly this pattern as CSR; the kernels below read only the CSR values and
// recompute each row's columns instead of loading column indices and row
// pointers (a third of an FP64 SpMV's bytes, half of an FP32 one's).
//
// A CTA takes kThreads consecutive rows.  Their values are contiguous in CSR,
// so the CTA copies the segment into shared memory with 16-byte loads and
// each thread forms its own row's product from there, in column order; for
// one offset (di, dj, dk) the rows of a warp read consecutive entries of x.
// CTAs loop over tiles (a persistent grid), so that the reducing variant can
// finish its sum in the last CTA.

__device__ __forceinline__ void grid_index(const LorMesh& m, int64_t i, int64_t& I, int64_t& J, int64_t& K) {
  if (m.ndof <= (int64_t)0xffffffff) {  // 32-bit division where it suffices
    const uint32_t u = (uint32_t)i, nx = (uint32_t)m.nx, ny = (uint32_t)m.ny;
    const uint32_t jk = u / nx, k = jk / ny;
    I = u - jk * nx;
    J = jk - k * ny;
    K = k;
  } else {
    const int64_t jk = i / m.nx;
    I = i - jk * m.nx;
    K = jk / m.ny;
    J = jk - K * m.ny;
  }
}

// First CSR position of row i (nnz for i = N).
__device__ __forceinline__ int64_t stencil_row_start(const LorMesh& m, int64_t i) {
  if (i >= m.ndof) return m.nnz;
  int64_t I, J, K;
  grid_index(m, i, I, J, K);
  return lor_row_start(I, J, K, m.nx, m.ny, m.nz);
}

struct StencilRow {
  int64_t i, start;
  bool xm, xp, ym, yp, zm, zp;  // neighbour present below / above on each axis
};

__device__ __forceinline__ StencilRow stencil_row(const LorMesh& m, int64_t i) {
  StencilRow r;
  int64_t I, J, K;
  grid_index(m, i, I, J, K);
  r.i = i;
  r.start = lor_row_start(I, J, K, m.nx, m.ny, m.nz);
  r.xm = I > 0;
  r.xp = I < m.nx - 1;
  r.ym = J > 0;
  r.yp = J < m.ny - 1;
  r.zm = K > 0;
  r.zp = K < m.nz - 1;
  return r;
}

// sum_j A_ij x_j from the row's values v[0..) in column order, in the matrix
// precision VT (x converted on the fly).
template <typename VT, typename XT>
__device__ __forceinline__ VT stencil_product(const LorMesh& m, const StencilRow& r, const VT* v,
                                              const XT* __restrict__ x) {
  const XT* xc = x + r.i;
  const int64_t sy = m.nx, sz = m.nx * m.ny;
  VT s = 0;
  int k = 0;
#pragma unroll
  for (int dk = -1; dk <= 1; ++dk) {
    const bool vk = dk < 0 ? r.zm : (dk > 0 ? r.zp : true);
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const bool vj = vk && (dj < 0 ? r.ym : (dj > 0 ? r.yp : true));
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const bool ok = vj && (di < 0 ? r.xm : (di > 0 ? r.xp : true));
        if (ok) {
          s += v[k] * (VT)xc[di + dj * sy + dk * sz];
          ++k;
        }
      }
    }
  }
  return s;
}

// ---- TMA staging.  Thread 0 of the CTA copies a tile's value segment into
// shared memory with one bulk asynchronous copy (cp.async.bulk, completion
// counted in bytes on an mbarrier); the CTA double-buffers, so the copy of
// its next tile runs while it computes the current one.  Every wait on an
// mbarrier is bounded (1 s of %globaltimer); on expiry the CTA records
// LOR_FLAG_TIMEOUT in the context's status word and stops.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` of bar, at most 1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}

// Copy bytes (a multiple of 16; both addresses 16-byte aligned) from global
// src to shared dst, completing on bar, which expects exactly these bytes.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// One tile's buffer: its at most 27 kThreads values plus the slack of
// starting at the 16-byte boundary below the segment and ending on one.
// The value arrays carry 16 bytes of padding after nnz for that last round-up.
template <typename VT>
constexpr uint32_t tile_bytes() {
  return (uint32_t)(sizeof(VT) * 27 * kThreads + 16);
}
// Buffers per CTA: 2 overlaps a CTA's next copy with its rows; 1 halves the
// shared memory, so twice as many CTAs share an SM and overlap each other's
// copies.  Measured on the 32^3 p = 6 PCG: one buffer is 2% faster per FP64
// and mixed iteration and 7% per refinement iteration (FP32 vectors).
template <typename VT>
constexpr int kStencilBuffers = 1;
template <typename VT>
constexpr size_t stencil_smem() {
  return kStencilBuffers<VT> * (size_t)tile_bytes<VT>();
}

// Start the copy of tile t's values into buf; returns the CSR position of buf[0].
template <typename VT>
__device__ __forceinline__ int64_t issue_tile(const LorMesh& m, const VT* __restrict__ vals, int64_t t, VT* buf,
                                              uint64_t* bar) {
  const int64_t r0 = t * kThreads;
  const int64_t v0 = stencil_row_start(m, r0);
  const int64_t v1 = stencil_row_start(m, r0 + kThreads < m.ndof ? r0 + kThreads : m.ndof);
  const int64_t a0 = v0 & ~(int64_t)(16 / sizeof(VT) - 1);
  const uint32_t bytes = (uint32_t)(((v1 - a0) * (int64_t)sizeof(VT) + 15) & ~(int64_t)15);
  tma_load_1d(buf, vals + a0, bytes, bar);
  return a0;
}

enum StencilMode {
  ST_SPMV = 0,       // y = A x
  ST_DINV_SPMV = 1,  // y = D^-1 A x
  ST_CHEB = 2,       // Chebyshev step: d = c1 d + c2 D^-1 (r - A z_in), z_out = z_in + d (or y = that, FP64)
  ST_CHEB_DOT = 3    // the same step writing y (FP64) and finishing r.y into *out
};

// What each mode does with row i's product s = (A x)_i.
template <typename VT, typename XT, int MODE, typename V>
__device__ __forceinline__ void stencil_epilogue(int64_t i, VT s, const VT* __restrict__ dinv,
                                                 const XT* __restrict__ x, const V* __restrict__ r,
                                                 VT* __restrict__ d, VT c1, VT c2, VT* __restrict__ zout,
                                                 V* __restrict__ y, Acc<V>& acc) {
  if constexpr (MODE == ST_SPMV) {
    y[i] = (V)s;
  } else if constexpr (MODE == ST_DINV_SPMV) {
    y[i] = (V)(dinv[i] * s);
  } else {
    const V ri = r[i];
    const VT dn = c1 * d[i] + c2 * dinv[i] * ((VT)ri - s);
    const VT zn = (VT)x[i] + dn;
    if constexpr (MODE == ST_CHEB_DOT) {
      y[i] = (V)zn;
      acc += ri * (V)zn;
    } else if (y) {
      y[i] = (V)zn;
    } else {
      d[i] = dn;
      zout[i] = zn;
    }
  }
}

template <typename VT, typename XT, int MODE, typename V = double>
__global__ void __launch_bounds__(kThreads) k_stencil(LorMesh m, const VT* __restrict__ vals,
                                                      const VT* __restrict__ dinv, const XT* __restrict__ x,
                                                      const V* __restrict__ r, VT* __restrict__ d, VT c1, VT c2,
                                                      VT* __restrict__ zout, V* __restrict__ y,
                                                      double* __restrict__ partial, unsigned* __restrict__ counter,
                                                      double* __restrict__ out, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t base[2];  // CSR position of each buffer's first element
  __shared__ int abort_flag;
  constexpr int NB = kStencilBuffers<VT>;
  VT* buf0 = reinterpret_cast<VT*>(smem_raw);
  VT* buf1 = reinterpret_cast<VT*>(smem_raw + (NB - 1) * tile_bytes<VT>());
  const int64_t ntiles = (m.ndof + kThreads - 1) / kThreads;
  const int64_t stride = gridDim.x;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
    if ((int64_t)blockIdx.x < ntiles) base[0] = issue_tile<VT>(m, vals, blockIdx.x, buf0, &bar[0]);
  }
  __syncthreads();
  Acc<V> acc = 0;
  int it = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += stride, ++it) {
    const int b = it & 1;
    // prefetch the next tile into the other buffer (its readers finished at
    // the barrier that ended the previous iteration); with one buffer the
    // next copy starts only after this tile's rows are done (below)
    if (NB == 2 && threadIdx.x == 0 && t + stride < ntiles)
      base[b ^ 1] = issue_tile<VT>(m, vals, t + stride, b ? buf0 : buf1, &bar[b ^ 1]);
    // (a test hook makes the wait count as expired: the copy still lands and
    // is waited for below)
    const bool landed = !(m.test_flags & LOR_TEST_EXPIRE_WAITS) && mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u);
    if (!landed) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    const VT* sv = b ? buf1 : buf0;
    const int64_t i = t * kThreads + threadIdx.x;
    if (i < m.ndof) {
      const StencilRow row = stencil_row(m, i);
      const VT s = stencil_product<VT, XT>(m, row, sv + (row.start - base[b]), x);
      stencil_epilogue<VT, XT, MODE, V>(i, s, dinv, x, r, d, c1, c2, zout, y, acc);
    }
    __syncthreads();  // every read of this buffer is done before it is refilled
    if (NB == 1 && threadIdx.x == 0 && t + stride < ntiles)
      base[b ^ 1] = issue_tile<VT>(m, vals, t + stride, buf0, &bar[b ^ 1]);
  }
  if (abort_flag && threadIdx.x == 0) {
    atomicOr(status, LOR_FLAG_TIMEOUT);
    // Let every copy this CTA issued land before it exits, each wait again
    // bounded: the tile whose wait gave up (after a real expiry this wait
    // gives up too, and the CTA can only exit with that copy pending if the
    // copy never completes) and the next tile's prefetch if one is in flight.
    const int b = it & 1;
    mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u);
    if (NB == 2 && blockIdx.x + (int64_t)(it + 1) * stride < ntiles)
      mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
  }
  if constexpr (MODE == ST_CHEB_DOT) finish_sums((double)acc, 0.0, 1, partial, counter, out, nullptr);
}

// ---- the same modes on an explicit CSR pattern (general meshes, whose LOR
// pattern has no closed form).  A CTA takes kCsrRows consecutive rows, one
// thread per row; their values and column indices are contiguous in CSR, so
// thread 0 stages both segments into shared memory with one bulk copy each
// (both completing on one mbarrier) and each thread forms its row's product
// from there, in column order.  A tile whose segments do not fit the buffers
// (more than kCsrCap / kCsrRows entries per row on average) is read from
// global memory instead, and its barrier phase is completed by a plain
// arrive so that the phases stay in step.  The column array carries 16 bytes
// of padding after nnz for the rounded last copy (the value arrays carry
// theirs).
constexpr int kCsrRows = 128;
constexpr int kCsrCap = 28 * kCsrRows;  // entries each tile buffer holds

template <typename VT>
constexpr uint32_t csr_vbuf_bytes() {
  return (uint32_t)(sizeof(VT) * kCsrCap + 16);
}
constexpr uint32_t csr_cbuf_bytes() { return (uint32_t)(4 * kCsrCap + 16); }
template <typename VT>
constexpr size_t csr_smem() {
  return csr_vbuf_bytes<VT>() + csr_cbuf_bytes();
}

// Start the copies of tile t's value and column segments (both addresses
// rounded down to 16 bytes, both lengths up); returns false, after a plain
// arrive on bar, when they do not fit.
template <typename VT>
__device__ __forceinline__ bool issue_csr_tile(const LorMesh& m, const VT* __restrict__ vals, int64_t t, VT* vbuf,
                                               int32_t* cbuf, uint64_t* bar, int64_t* vbase, int64_t* cbase) {
  const int64_t r0 = t * kCsrRows;
  const int64_t r1 = r0 + kCsrRows < m.ndof ? r0 + kCsrRows : m.ndof;
  const int64_t e0 = m.rowptr[r0], e1 = m.rowptr[r1];
  const int64_t av = e0 & ~(int64_t)(16 / sizeof(VT) - 1), ac = e0 & ~(int64_t)3;
  const int64_t vb = ((e1 - av) * (int64_t)sizeof(VT) + 15) & ~(int64_t)15;
  const int64_t cb = ((e1 - ac) * 4 + 15) & ~(int64_t)15;
  if (vb > (int64_t)csr_vbuf_bytes<VT>() || cb > (int64_t)csr_cbuf_bytes() || (m.test_flags & LOR_TEST_UNSTAGED_CSR)) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    return false;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"((uint32_t)(vb + cb))
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(vbuf)),
               "l"(vals + av), "r"((uint32_t)vb), "r"(smem_u32(bar))
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(cbuf)),
               "l"(m.colidx + ac), "r"((uint32_t)cb), "r"(smem_u32(bar))
               : "memory");
  *vbase = av;
  *cbase = ac;
  return true;
}

template <typename VT, typename XT, int MODE, typename V = double>
__global__ void __launch_bounds__(kCsrRows) k_csr(LorMesh m, const VT* __restrict__ vals, const VT* __restrict__ dinv,
                                                  const XT* __restrict__ x, const V* __restrict__ r,
                                                  VT* __restrict__ d, VT c1, VT c2, VT* __restrict__ zout,
                                                  V* __restrict__ y, double* __restrict__ partial,
                                                  unsigned* __restrict__ counter, double* __restrict__ out,
                                                  int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t vbase[2], cbase[2];  // CSR position of each buffer's first element
  __shared__ int staged[2];
  __shared__ int abort_flag;
  VT* vbuf = reinterpret_cast<VT*>(smem_raw);
  int32_t* cbuf = reinterpret_cast<int32_t*>(smem_raw + csr_vbuf_bytes<VT>());
  const int64_t ntiles = (m.ndof + kCsrRows - 1) / kCsrRows;
  const int64_t stride = gridDim.x;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
    if ((int64_t)blockIdx.x < ntiles)
      staged[0] = issue_csr_tile<VT>(m, vals, blockIdx.x, vbuf, cbuf, &bar[0], &vbase[0], &cbase[0]);
  }
  __syncthreads();
  Acc<V> acc = 0;
  int it = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += stride, ++it) {
    const int b = it & 1;
    // (the test hook makes the wait count as expired; the copy still lands
    // and is waited for below)
    const bool landed = !(m.test_flags & LOR_TEST_EXPIRE_WAITS) && mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u);
    if (!landed) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    const int64_t i = t * kCsrRows + threadIdx.x;
    if (i < m.ndof) {
      const int64_t j0 = m.rowptr[i], j1 = m.rowptr[i + 1];
      VT s = 0;
      if (staged[b]) {
        const int64_t ov = vbase[b], oc = cbase[b];
        for (int64_t j = j0; j < j1; ++j) s += vbuf[j - ov] * (VT)x[cbuf[j - oc]];
      } else {
        for (int64_t j = j0; j < j1; ++j) s += vals[j] * (VT)x[m.colidx[j]];
      }
      stencil_epilogue<VT, XT, MODE, V>(i, s, dinv, x, r, d, c1, c2, zout, y, acc);
    }
    __syncthreads();  // every read of the buffers is done before they are refilled
    if (threadIdx.x == 0 && t + stride < ntiles)
      staged[b ^ 1] = issue_csr_tile<VT>(m, vals, t + stride, vbuf, cbuf, &bar[b ^ 1], &vbase[b ^ 1], &cbase[b ^ 1]);
  }
  if (abort_flag && threadIdx.x == 0) {
    atomicOr(status, LOR_FLAG_TIMEOUT);
    // let the copies whose wait gave up land before the CTA exits (bounded
    // again; after a real expiry this gives up too)
    mbar_wait_bounded(&bar[it & 1], (uint32_t)(it >> 1) & 1u);
  }
  if constexpr (MODE == ST_CHEB_DOT) finish_sums((double)acc, 0.0, 1, partial, counter, out, nullptr);
}

// Persistent grid: every SM filled to the kernel's occupancy (at most one CTA
// per tile; the reducing mode at most LOR_PCG_MAX_BLOCKS CTAs).  The shared
// memory limit is raised once per device and the grid size cached for the
// life of the process (one primary context per device: a cudaDeviceReset
// would drop the attribute).
template <typename VT, typename XT, int MODE, typename V>
cudaError_t stencil_grid(const LorMesh& m, int* grid) {
  static int per_device[64] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!per_device[dev]) {
    err = cudaFuncSetAttribute(k_stencil<VT, XT, MODE, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stencil_smem<VT>());
    int sms = 0, occ = 0;
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess)
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stencil<VT, XT, MODE, V>, kThreads,
                                                          stencil_smem<VT>());
    if (err != cudaSuccess) return err;
    per_device[dev] = sms * (occ > 0 ? occ : 1);
  }
  const int64_t ntiles = (m.ndof + kThreads - 1) / kThreads;
  int64_t g = per_device[dev] < ntiles ? per_device[dev] : ntiles;
  if (MODE == ST_CHEB_DOT && g > LOR_PCG_MAX_BLOCKS) g = LOR_PCG_MAX_BLOCKS;
  *grid = (int)(g > 0 ? g : 1);
  return cudaSuccess;
}

// The same for the explicit-CSR kernel.
template <typename VT, typename XT, int MODE, typename V>
cudaError_t csr_grid(const LorMesh& m, int* grid) {
  static int per_device[64] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!per_device[dev]) {
    err = cudaFuncSetAttribute(k_csr<VT, XT, MODE, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)csr_smem<VT>());
    int sms = 0, occ = 0;
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess)
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_csr<VT, XT, MODE, V>, kCsrRows, csr_smem<VT>());
    if (err != cudaSuccess) return err;
    per_device[dev] = sms * (occ > 0 ? occ : 1);
  }
  const int64_t ntiles = (m.ndof + kCsrRows - 1) / kCsrRows;
  int64_t g = per_device[dev] < ntiles ? per_device[dev] : ntiles;
  if (MODE == ST_CHEB_DOT && g > LOR_PCG_MAX_BLOCKS) g = LOR_PCG_MAX_BLOCKS;
  *grid = (int)(g > 0 ? g : 1);
  return cudaSuccess;
}

template <typename VT, typename XT, int MODE, typename V = double>
cudaError_t launch_stencil(const LorMesh& m, const VT* vals, const VT* dinv, const XT* x, const V* r, VT* d,
                           double c1, double c2, VT* zout, V* y, double* partial, unsigned* counter,
                           double* out, int* status, cudaStream_t s) {
  if (m.rowptr) {  // general mesh: explicit CSR pattern
    int grid = 0;
    cudaError_t err = csr_grid<VT, XT, MODE, V>(m, &grid);
    if (err != cudaSuccess) return err;
    k_csr<VT, XT, MODE, V><<<grid, kCsrRows, csr_smem<VT>(), s>>>(m, vals, dinv, x, r, d, (VT)c1, (VT)c2, zout, y,
                                                                  partial, counter, out, status);
    lor_count_launch();
    return cudaGetLastError();
  }
  int grid = 0;
  cudaError_t err = stencil_grid<VT, XT, MODE, V>(m, &grid);
  if (err != cudaSuccess) return err;
  k_stencil<VT, XT, MODE, V><<<grid, kThreads, stencil_smem<VT>(), s>>>(m, vals, dinv, x, r, d, (VT)c1, (VT)c2, zout, y,
                                                                    partial, counter, out, status); lor_count_launch();
  return cudaGetLastError();
}

// D^-1 from the diagonal entries (closed-form positions).
template <typename VT>
__global__ void k_diag_inv(LorMesh m, const VT* __restrict__ vals, VT* __restrict__ dinv) {
  LOR_GRID_STRIDE(i, m.ndof) {
    if (m.rowptr) {
      const int64_t pos = lor_find_col(m.colidx, m.rowptr[i], m.rowptr[i + 1], i);
      dinv[i] = (VT)1 / vals[pos];
      continue;
    }
    int64_t I, J, K;
    grid_index(m, i, I, J, K);
    dinv[i] = (VT)1 / vals[lor_entry_pos(I, J, K, 0, 0, 0, m.nx, m.ny, m.nz)];
  }
}

// One Chebyshev step j >= 1 (see ST_CHEB); the last one writes z64.
template <typename VT, typename V = double>
cudaError_t cheb_step(lor_ctx* c, const VT* vals, const VT* dinv, const V* r, const VT* zin, VT* zout, VT* d,
                      double c1, double c2, V* z64, cudaStream_t s) {
  return launch_stencil<VT, VT, ST_CHEB, V>(c->m, vals, dinv, zin, r, d, c1, c2, zout, z64, nullptr, nullptr, nullptr,
                                            c->d_status, s);
}

// ---------------------------------------------------------------- PCG vector kernels
// Device scalars (slots of ctx->red after the partials).
enum { S_PQ = 0, S_RR = 1, S_BB = 2, S_RZ0 = 3, S_RZ1 = 4, S_IR = 5, S_COUNT = 6 };

__global__ void k_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ Ax,
                           double* __restrict__ r) {
  LOR_GRID_STRIDE(i, n) r[i] = b[i] - Ax[i];
}

template <typename VT, typename V = double>
cudaError_t precond_apply_t(lor_ctx* c, const VT* vals, const VT* dinv, const V* r, V* z, cudaStream_t s) {
  const int64_t n = c->m.ndof;
  const int g = grid_rows(n);
  if (c->pc_kind == LOR_PRECOND_JACOBI) {
    k_jacobi<VT, V><<<g, kThreads, 0, s>>>(n, dinv, r, z); lor_count_launch();
    return cudaGetLastError();
  }
  VT* zA = (VT*)c->pc_work;
  VT* zB = zA + n;
  VT* d = zB + n;
  const double theta = 0.5 * (c->pc_hi + c->pc_lo), delta = 0.5 * (c->pc_hi - c->pc_lo);
  const double sigma = theta / delta;
  const int k = c->pc_degree;
  k_cheb_first<VT, V><<<g, kThreads, 0, s>>>(n, dinv, r, (VT)(1.0 / theta), zA, d, k == 1 ? z : nullptr);
  lor_count_launch();
  double rho = 1.0 / sigma;
  VT* zin = zA;
  VT* zout = zB;
  for (int j = 1; j < k; ++j) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
    const cudaError_t err = cheb_step<VT, V>(c, vals, dinv, r, zin, zout, d, c1, c2, j == k - 1 ? z : nullptr, s);
    if (err != cudaSuccess) return err;
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

// The status word rides along with each synchronising scalar read (into the
// last pinned slot); a set LOR_FLAG_TIMEOUT ends the solve.
double* status_slot(lor_ctx* c) { return c->h_scalar + 15; }
cudaError_t queue_status_read(lor_ctx* c, cudaStream_t s) {
  return cudaMemcpyAsync(status_slot(c), c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
}
int timed_out(lor_ctx* c, const char* what) {
  int flags = 0;
  memcpy(&flags, status_slot(c), sizeof(int));
  if (!(flags & LOR_FLAG_TIMEOUT)) return LOR_OK;
  c->err = std::string(what) + ": a bounded device wait expired (a bulk copy into shared memory never completed)";
  return LOR_ETIMEOUT;
}

}  // namespace

cudaError_t lor_launch_diag_inv(const LorMesh& m, const void* vals, int dtype, void* dinv, cudaStream_t s) {
  if (dtype == LOR_F64) {
    k_diag_inv<double><<<grid_rows(m.ndof), kThreads, 0, s>>>(m, (const double*)vals, (double*)dinv); lor_count_launch();
  } else {
    k_diag_inv<float><<<grid_rows(m.ndof), kThreads, 0, s>>>(m, (const float*)vals, (float*)dinv); lor_count_launch();
  }
  return cudaGetLastError();
}

cudaError_t lor_launch_spmv(const LorMesh& m, const void* vals, int dtype, const double* x, double* y, int* status,
                            cudaStream_t s) {
  if (dtype == LOR_F64)
    return launch_stencil<double, double, ST_SPMV, double>(m, (const double*)vals, nullptr, x, nullptr, nullptr, 0.0,
                                                           0.0, nullptr, y, nullptr, nullptr, nullptr, status, s);
  return launch_stencil<float, double, ST_SPMV, double>(m, (const float*)vals, nullptr, x, nullptr, nullptr, 0.0, 0.0,
                                                        nullptr, y, nullptr, nullptr, nullptr, status, s);
}

namespace {

// z = B_h r for vectors of type V (FP64, or FP32 in the refinement's inner
// iterations).
template <typename V>
int precond_apply_v(lor_ctx* c, const V* r, V* z, cudaStream_t s) {
  cudaError_t err;
  if (c->pc_kind == LOR_PRECOND_NONE) {
    err = cudaMemcpyAsync(z, r, sizeof(V) * c->m.ndof, cudaMemcpyDeviceToDevice, s);
  } else if (c->pc_dtype == LOR_F64) {
    err = precond_apply_t<double, V>(c, c->vals64, c->dinv64, r, z, s);
  } else {
    err = precond_apply_t<float, V>(c, c->vals32, c->dinv32, r, z, s);
  }
  return err == cudaSuccess ? LOR_OK : fail(c, err, "precond_apply");
}

}  // namespace

int lor_precond_apply_impl(lor_ctx* c, const double* r, double* z, cudaStream_t s) {
  return precond_apply_v<double>(c, r, z, s);
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
    err = dtype == LOR_F64
              ? launch_stencil<double, double, ST_DINV_SPMV, double>(c->m, c->vals64, c->dinv64, v, nullptr, nullptr,
                                                                     0.0, 0.0, nullptr, w, nullptr, nullptr, nullptr,
                                                                     c->d_status, s)
              : launch_stencil<float, double, ST_DINV_SPMV, double>(c->m, c->vals32, c->dinv32, v, nullptr, nullptr,
                                                                    0.0, 0.0, nullptr, w, nullptr, nullptr, nullptr,
                                                                    c->d_status, s);
    if (err != cudaSuccess) return fail(c, err, "power iteration");
    dot_to(c, w, w, S + 0, s);
    dot_to(c, v, v, S + 1, s);
    err = cudaMemcpyAsync(c->h_scalar, S, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = queue_status_read(c, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return fail(c, err, "power iteration");
    if (int rc = timed_out(c, "power iteration")) return rc;
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
template <typename V = double>
__global__ void __launch_bounds__(kThreads) k_pcg_dot(int64_t n, const V* __restrict__ a, const V* __restrict__ b,
                                                      double* __restrict__ partial, unsigned* __restrict__ counter,
                                                      double* __restrict__ out) {
  Acc<V> s = 0;
  LOR_GRID_STRIDE(i, n) s += a[i] * b[i];
  finish_sums((double)s, 0.0, 1, partial, counter, out, nullptr);
}

// x += alpha p, r -= alpha q (alpha = rz / pq on the device), r.r, and the
// first step of the preconditioner on the updated r:
//   mode 0 (none): z = r;  mode 1 (Jacobi): z = D^-1 r;
//   mode 2 (Chebyshev, degree 1): z = D^-1 r / theta;
//   mode 3 (Chebyshev, degree >= 2): zA = d = D^-1 r / theta (smoother precision).
// Modes 0-2 also form r.z (z is final there).
//
// Convergence record rec (device): rec[0] = r.r, rec[1] = 1 when
// r.r <= stop_rr (the stopping test of this iteration), rec[2] = the status
// word; written by the last CTA, copied to the host in one read.  The host
// queues the next iteration before it reads this one's record, so the next
// iteration's update and direction kernels start by testing rec[1]: behind a
// converged iteration they change nothing (x, r, p, q and the scalars keep
// the converged iteration's values).
template <typename VT, typename V = double>
__global__ void __launch_bounds__(kThreads) k_pcg_update(int64_t n, const double* __restrict__ S, int rz_slot,
                                                         const V* __restrict__ p, const V* __restrict__ q,
                                                         double* __restrict__ x, V* __restrict__ r, int mode,
                                                         const VT* __restrict__ dinv, VT inv_theta,
                                                         V* __restrict__ z, VT* __restrict__ zA,
                                                         VT* __restrict__ d, double* __restrict__ partial,
                                                         unsigned* __restrict__ counter, double* __restrict__ out_rr,
                                                         double* __restrict__ out_rz, double stop_rr,
                                                         double* __restrict__ rec, const int* __restrict__ status) {
  if (*(volatile double*)(rec + 1) != 0.0) return;  // behind a converged iteration
  const double alpha = S[rz_slot] / S[S_PQ];
  const V av = (V)alpha;
  Acc<V> srr = 0, srz = 0;
  LOR_GRID_STRIDE(i, n) {
    x[i] += alpha * (double)p[i];
    const V ri = r[i] - av * q[i];
    r[i] = ri;
    srr += ri * ri;
    if (mode == 0) {
      z[i] = ri;
      srz += ri * ri;
    } else if (mode == 1 || mode == 2) {
      const VT zi = mode == 1 ? dinv[i] * (VT)ri : dinv[i] * (VT)ri * inv_theta;
      z[i] = (V)zi;
      srz += ri * (V)zi;
    } else {
      const VT zi = dinv[i] * (VT)ri * inv_theta;
      zA[i] = zi;
      d[i] = zi;
    }
  }
  if (finish_sums((double)srr, (double)srz, mode <= 2 ? 2 : 1, partial, counter, out_rr, out_rz) &&
      threadIdx.x == 0) {
    const double rr = *out_rr;
    rec[0] = rr;
    rec[2] = (double)*(const volatile int*)status;
    __threadfence();
    rec[1] = rr <= stop_rr ? 1.0 : 0.0;
  }
}

// p = z + beta p (beta = rz_new / rz_old; first: p = z) and the output of
// the next apply initialised: q = p on essential DOFs, 0 elsewhere.  Does
// nothing behind a converged iteration (rec[1] set, see k_pcg_update).
template <typename V = double>
__global__ void k_pcg_direction(LorMesh m, const double* __restrict__ S, int new_slot, int old_slot, int first,
                                const V* __restrict__ z, V* __restrict__ p, V* __restrict__ q,
                                const double* __restrict__ rec) {
  if (*(const volatile double*)(rec + 1) != 0.0) return;
  const V beta = (V)(first ? 0.0 : S[new_slot] / S[old_slot]);
  LOR_GRID_STRIDE(i, m.ndof) {
    const V pi = first ? z[i] : z[i] + beta * p[i];
    p[i] = pi;
    q[i] = lor_dof_essential(m, i) ? pi : (V)0;
  }
}

// r = b - A x rounded to V, and |b - A x|^2 (FP64) into *out.
template <typename V>
__global__ void __launch_bounds__(kThreads) k_residual_norm(int64_t n, const double* __restrict__ b,
                                                            const double* __restrict__ Ax, V* __restrict__ r,
                                                            double* __restrict__ partial,
                                                            unsigned* __restrict__ counter, double* __restrict__ out) {
  double s = 0.0;
  LOR_GRID_STRIDE(i, n) {
    const double ri = b[i] - Ax[i];
    r[i] = (V)ri;
    s += ri * ri;
  }
  finish_sums(s, 0.0, 1, partial, counter, out, nullptr);
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

template <typename VT, typename V = double>
cudaError_t pcg_precond_rest(lor_ctx* c, const VT* vals, const VT* dinv, const V* r, V* z, double* out_rz,
                             cudaStream_t s) {
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
      const cudaError_t err = cheb_step<VT, V>(c, vals, dinv, r, zin, zout, d, c1, c2, (V*)nullptr, s);
      if (err != cudaSuccess) return err;
    } else {
      const cudaError_t err = launch_stencil<VT, VT, ST_CHEB_DOT, V>(c->m, vals, dinv, zin, r, d, c1, c2, nullptr, z,
                                                                     pcg_partials(c), c->red_count, out_rz,
                                                                     c->d_status, s);
      if (err != cudaSuccess) return err;
    }
    rho = rho_new;
    VT* t = zin;
    zin = zout;
    zout = t;
  }
  return cudaGetLastError();
}

template <typename VT, typename V = double>
cudaError_t pcg_update(lor_ctx* c, const VT* dinv, double* S, int cur, const V* p, const V* q, double* x, V* r,
                       V* z, int mode, double* out_rz, double stop_rr, double* rec, int grid, cudaStream_t s) {
  const double theta = 0.5 * (c->pc_hi + c->pc_lo);
  VT* zA = (VT*)c->pc_work;
  VT* d = zA ? zA + 2 * c->m.ndof : nullptr;
  k_pcg_update<VT, V><<<grid, kThreads, 0, s>>>(c->m.ndof, S, cur, p, q, x, r, mode, dinv,
                                                   (VT)(theta > 0 ? 1.0 / theta : 1.0), z, zA, d, pcg_partials(c),
                                                   c->red_count, S + S_RR, out_rz, stop_rr, rec, c->d_status);
  lor_count_launch();
  return cudaGetLastError();
}

// The two events of the iteration records (below), destroyed on every exit.
struct EventPair {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t create() {
    for (auto& e : ev) {
      const cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
  }
  ~EventPair() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

__global__ void k_add(int64_t n, double* __restrict__ x, const double* __restrict__ d) {
  LOR_GRID_STRIDE(i, n) x[i] += d[i];
}

// PCG with x_0 = 0.  V: the type of the vectors r, z, p, q (x stays FP64).
// f32_apply: the operator is the FP32-arithmetic apply, else the FP64 one
// (V = float requires it).  confirm: a converged recurrence residual is
// checked against the true residual b - A x (FP64 operator) before the solve
// counts as converged; if it fails, the iteration continues from the true
// residual (keeping the search direction).  replace > 0 (with confirm): the
// true residual is also formed, and substituted, whenever the recurrence
// residual has fallen by the factor `replace` since the last substitution
// (residual replacement); *replacements counts them.  A replacement that does
// not lower the true residual ends the solve (LOR_ENOCONV).
template <typename V>
int pcg_core(lor_ctx* c, const double* b, double* x, double rtol, int maxit, bool f32_apply, bool confirm,
             double replace, int* iters, double* relres, int* replacements, cudaStream_t s) {
  constexpr bool VF = sizeof(V) == sizeof(float);
  const int64_t n = c->m.ndof;
  // FP64: r, z, p, Ap in the 4 N doubles of pcg_work.  FP32: the same four
  // in its first 2 N doubles' worth, and A x (FP64) for the true residual in
  // the last N doubles.
  V* r = reinterpret_cast<V*>(c->pcg_work);
  V* z = r + n;
  V* p = z + n;
  V* q = p + n;
  double* ax64 = c->pcg_work + 2 * n;
  double* S = c->red + LOR_RED_BLOCKS;  // S[0] = p.q, S[1] = r.r, S[2] = b.b, S[3], S[4] = r.z (alternating)
  double* rec = S + 8;                  // the latest update's record: r.r, converged flag, status word
  double* hs = c->h_scalar;
  // Host copies of the records of two consecutive iterations (pinned), each
  // complete when its event has passed.
  auto hrec = [&](int k) { return hs + 8 + 3 * (k & 1); };
  EventPair evs;
  const int g = grid_rows(n);
  const bool f64 = c->pc_dtype == LOR_F64;
  // preconditioner mode of the fused update (see k_pcg_update)
  const int mode = c->pc_kind == LOR_PRECOND_NONE ? 0 : c->pc_kind == LOR_PRECOND_JACOBI ? 1 : c->pc_degree == 1 ? 2 : 3;
  const int g_dot = pcg_grid(k_pcg_dot<V>);
  const int g_dot64 = pcg_grid(k_pcg_dot<double>);
  const int g_upd = f64 ? pcg_grid(k_pcg_update<double, V>) : pcg_grid(k_pcg_update<float, V>);
  auto dot = [&](const V* a, const V* bb, double* out) {
    k_pcg_dot<V><<<g_dot, kThreads, 0, s>>>(n, a, bb, pcg_partials(c), c->red_count, out); lor_count_launch();
  };
  auto other = [](int slot) { return slot == S_RZ0 ? S_RZ1 : S_RZ0; };
  cudaError_t err = evs.create();
  if (err == cudaSuccess) err = cudaMemsetAsync(x, 0, sizeof(double) * n, s);
  if (err == cudaSuccess) {
    if constexpr (VF) err = lor_launch_to_f32(b, r, n, s);
    else err = cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  }
  if (err == cudaSuccess) {
    k_pcg_dot<double><<<g_dot64, kThreads, 0, s>>>(n, b, b, pcg_partials(c), c->red_count, S + S_BB);
    lor_count_launch();
    err = cudaMemcpyAsync(hs, S + S_BB, sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return fail(c, err, "pcg");
  const double nb = sqrt(hs[0]);
  int it = 0, nrep = 0;
  double rel = 0.0, last_true = 1.0;
  int status = LOR_ENOCONV;
  const char* why = "pcg: no convergence within maxit";
  // One iteration: q += A p, p.q, then the fused update, which also tests
  // |r|^2 <= (trigger |b|)^2 and records the result; the record is read on
  // the host one iteration late (the next iteration is already queued).
  auto queue_iteration = [&](int k, int cur, double trigger) -> cudaError_t {
    cudaError_t e;
    if constexpr (VF) {
      e = lor_launch_apply_f32v_accumulate(c->m, c->T, c->Dq32, c->have_beta ? c->Mq32 : nullptr, p, q, s);
    } else {
      e = f32_apply ? lor_launch_apply_f32_accumulate(c->m, c->T, c->Dq32, c->have_beta ? c->Mq32 : nullptr, p, q, s)
                    : lor_launch_apply_accumulate(c->m, c->T, c->Dq, c->have_beta ? c->Mq : nullptr, p, q, s);
    }
    if (e != cudaSuccess) return e;
    dot(p, q, S + S_PQ);
    const double stop = trigger * nb;
    e = f64 ? pcg_update<double, V>(c, c->dinv64, S, cur, p, q, x, r, z, mode, S + other(cur), stop * stop, rec,
                                    g_upd, s)
            : pcg_update<float, V>(c, c->dinv32, S, cur, p, q, x, r, z, mode, S + other(cur), stop * stop, rec,
                                   g_upd, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hrec(k), rec, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(evs.ev[k & 1], s);
    return e;
  };
  // The rest of the preconditioner on the updated r (Chebyshev degree >= 2)
  // and the next search direction (a no-op behind a converged iteration).
  auto queue_tail = [&](int cur) -> cudaError_t {
    const int nxt = other(cur);
    if (mode == 3) {
      const cudaError_t e = f64 ? pcg_precond_rest<double, V>(c, c->vals64, c->dinv64, r, z, S + nxt, s)
                                : pcg_precond_rest<float, V>(c, c->vals32, c->dinv32, r, z, S + nxt, s);
      if (e != cudaSuccess) return e;
    }
    k_pcg_direction<V><<<g, kThreads, 0, s>>>(c->m, S, nxt, cur, 0, z, p, q, rec); lor_count_launch();
    return cudaGetLastError();
  };
  auto trigger_now = [&]() { return replace > 0.0 ? fmax(rtol, replace * last_true) : rtol; };
  if (nb == 0.0) {
    status = LOR_OK;
  } else if (maxit > 0) {
    int rc = precond_apply_v<V>(c, r, z, s);
    if (rc) return rc;
    int cur = S_RZ0;
    dot(r, z, S + cur);
    err = cudaMemsetAsync(rec, 0, 3 * sizeof(double), s);
    if (err != cudaSuccess) return fail(c, err, "pcg");
    k_pcg_direction<V><<<g, kThreads, 0, s>>>(c->m, S, cur, cur, 1, z, p, q, rec); lor_count_launch();
    double trigger = trigger_now();
    err = queue_iteration(0, cur, trigger);
    if (err != cudaSuccess) return fail(c, err, "pcg");
    // Loop invariant: iteration `it` (0-based) is queued and its record not yet read.
    while (true) {
      const int nxt = other(cur);
      const bool ahead = it + 1 < maxit;
      if (ahead) {  // queue the next iteration before waiting for this one's record
        err = queue_tail(cur);
        if (err == cudaSuccess) err = queue_iteration(it + 1, nxt, trigger);
        if (err != cudaSuccess) return fail(c, err, "pcg");
      }
      err = cudaEventSynchronize(evs.ev[it & 1]);
      if (err != cudaSuccess) return fail(c, err, "pcg");
      const double* hr = hrec(it);
      const int flags = (int)hr[2];
      if (flags & LOR_FLAG_TIMEOUT) {
        c->err = "pcg: a bounded device wait expired (a bulk copy into shared memory never completed)";
        return LOR_ETIMEOUT;
      }
      ++it;
      rel = sqrt(hr[0]) / nb;
      if (hr[1] == 0.0) {  // not converged: the next iteration is already queued
        if (!ahead) break;
        cur = nxt;
        continue;
      }
      // Converged on the recurrence residual; the iteration queued behind it
      // changed nothing.
      if (!confirm) {
        status = LOR_OK;
        break;
      }
      // confirm on the true residual b - A x (FP64 operator)
      if constexpr (VF) {
        err = lor_launch_apply(c->m, c->T, c->Dq, c->have_beta ? c->Mq : nullptr, x, ax64, s);
        if (err == cudaSuccess) {
          k_residual_norm<V><<<g_dot64, kThreads, 0, s>>>(n, b, ax64, r, pcg_partials(c), c->red_count, S + S_RR);
          lor_count_launch();
          err = cudaMemcpyAsync(hs, S + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s);
        }
      } else {
        err = lor_launch_apply(c->m, c->T, c->Dq, c->have_beta ? c->Mq : nullptr, x, q, s);
        if (err == cudaSuccess) {
          k_residual<<<g, kThreads, 0, s>>>(n, b, q, r); lor_count_launch();
          dot(r, r, S + S_RR);
          err = cudaMemcpyAsync(hs, S + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s);
        }
      }
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err != cudaSuccess) return fail(c, err, "pcg");
      rel = sqrt(hs[0]) / nb;
      if (rel <= rtol) {
        status = LOR_OK;
        break;
      }
      if (replace > 0.0) {
        if (!(rel < last_true)) {
          why = "pcg: a residual replacement did not lower the true residual";
          break;
        }
        last_true = rel;
        ++nrep;
      }
      // continue from the true residual (keeping the search direction):
      // precondition it afresh and clear the converged flag
      err = cudaMemsetAsync(rec, 0, 3 * sizeof(double), s);
      if (err != cudaSuccess) return fail(c, err, "pcg");
      rc = precond_apply_v<V>(c, r, z, s);
      if (rc) return rc;
      dot(r, z, S + nxt);
      k_pcg_direction<V><<<g, kThreads, 0, s>>>(c->m, S, nxt, cur, 0, z, p, q, rec); lor_count_launch();
      cur = nxt;
      trigger = trigger_now();
      if (it >= maxit) break;
      err = queue_iteration(it, cur, trigger);
      if (err != cudaSuccess) return fail(c, err, "pcg");
    }
    // drain what was queued behind the last record read
    err = cudaStreamSynchronize(s);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) return fail(c, err, "pcg");
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if (replacements) *replacements = nrep;
  if (status == LOR_ENOCONV) c->err = why;
  return status;
}

}  // namespace

int lor_pcg_impl(lor_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters, double* relres,
                 cudaStream_t s) {
  return pcg_core<double>(c, b, x, rtol, maxit, false, true, 0.0, iters, relres, nullptr, s);
}

// Iterative refinement: the outer residual b - A x with the FP64 operator,
// the corrections by PCG with the FP32 operator to inner_rtol.
int lor_pcg_ir_impl(lor_ctx* c, const double* b, double* x, double rtol, double inner_rtol, int maxit, int scheme,
                    int* outer_iters, int* inner_iters, double* relres, cudaStream_t s) {
  int rc = lor_ensure_f32_factors(c, s);
  if (rc) return rc;
  if (scheme == LOR_IR_REPLACE) {
    // one PCG on the FP32 operator; the FP64 residual replaces the recurrence
    // residual each time the latter has fallen by inner_rtol
    int it = 0, nrep = 0;
    double rel = 0.0;
    rc = pcg_core<float>(c, b, x, rtol, maxit, true, true, inner_rtol, &it, &rel, &nrep, s);
    if (outer_iters) *outer_iters = it > 0 ? nrep + 1 : 0;
    if (inner_iters) *inner_iters = it;
    if (relres) *relres = rel;
    return rc;
  }
  rc = lor_alloc_ir_work(c);
  if (rc) return rc;
  const int64_t n = c->m.ndof;
  double* rr = c->ir_work;  // outer residual
  double* dd = rr + n;      // correction (and A x scratch)
  double* S = c->red + LOR_RED_BLOCKS;
  double* hs = c->h_scalar;
  const int g = grid_rows(n);
  const int g_dot = pcg_grid(k_pcg_dot<double>);
  auto norm2 = [&](const double* a, double* out) -> cudaError_t {
    k_pcg_dot<double><<<g_dot, kThreads, 0, s>>>(n, a, a, pcg_partials(c), c->red_count, S + S_IR);
    lor_count_launch();
    cudaError_t e = cudaMemcpyAsync(hs, S + S_IR, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *out = hs[0];
    return e;
  };
  cudaError_t err = cudaMemsetAsync(x, 0, sizeof(double) * n, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(rr, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  double bb = 0.0;
  if (err == cudaSuccess) err = norm2(b, &bb);
  if (err != cudaSuccess) return fail(c, err, "pcg_ir");
  const double nb = sqrt(bb);
  int outer = 0, inner = 0, status = LOR_ENOCONV;
  const char* why = "pcg_ir: no convergence within the limits";
  double rel = nb == 0.0 ? 0.0 : 1.0, prev = HUGE_VAL;
  while (true) {
    if (rel <= rtol) {
      status = LOR_OK;
      break;
    }
    if (outer >= 64 || inner >= maxit) break;
    if (!(rel < prev)) {
      why = "pcg_ir: an outer step did not reduce the residual";
      break;
    }
    prev = rel;
    int it = 0;
    double rin = 0.0;
    rc = pcg_core<float>(c, rr, dd, inner_rtol, maxit - inner, true, false, 0.0, &it, &rin, nullptr, s);
    if (rc != LOR_OK && rc != LOR_ENOCONV) return rc;
    inner += it;
    ++outer;
    k_add<<<g, kThreads, 0, s>>>(n, x, dd); lor_count_launch();
    err = lor_launch_apply(c->m, c->T, c->Dq, c->have_beta ? c->Mq : nullptr, x, dd, s);
    if (err == cudaSuccess) {
      k_residual<<<g, kThreads, 0, s>>>(n, b, dd, rr); lor_count_launch();
      err = cudaGetLastError();
    }
    double r2 = 0.0;
    if (err == cudaSuccess) err = norm2(rr, &r2);
    if (err != cudaSuccess) return fail(c, err, "pcg_ir");
    if (int trc = timed_out(c, "pcg_ir")) return trc;
    rel = sqrt(r2) / nb;
  }
  if (outer_iters) *outer_iters = outer;
  if (inner_iters) *inner_iters = inner;
  if (relres) *relres = rel;
  if (status == LOR_ENOCONV) c->err = why;
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
// device address).  Cached for the life of the process: this assumes one
// primary context per device (after a cudaDeviceReset it would be stale).
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
    const cudaError_t err = cheb_step<VT>(c, vals, dinv, r, zin, zout, d, c1, c2, j == k - 1 ? z : nullptr, s);
    if (err != cudaSuccess) return err;
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

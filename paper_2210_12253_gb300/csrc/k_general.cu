// k_general.cu -- Step S1.2 / A2 on a general conforming hex mesh: the LOR
// CSR pattern from the element-to-DOF map (the element restriction G of the
// high-order space, Section 3, Step S1.1), when no closed form exists.
//
// The macro-element structure is kept: sub-hex (a,b,c) of element e couples
// the 8 DOFs map[e][(a+r0) + n((b+r1) + n(c+r2))].  Every (sub-hex, vertex)
// incidence appends the sub-hex's 8 DOFs to the vertex's list; each row's list
// is then sorted and de-duplicated; two exclusive scans give the list offsets
// and the row pointers.  This is the count / scan / fill order of the paper's
// A2, with the minimal-element rule replaced by de-duplication (every
// coupling is kept once whichever elements produce it).
#include "lor_internal.cuh"

namespace {

constexpr int kT = 256;
constexpr int kItems = 8;                  // items per thread in a scan block
constexpr int kChunk = kT * kItems;        // items per scan block
constexpr int kMaxRowList = 8 * 64;        // incidences x 8 per row (vertex valence up to 64)

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

int grid_for(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

// ---------------------------------------------------------------- exclusive scan (int64)
// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_tot[kT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < kT / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kT / 32) warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = w > 0 ? warp_tot[w - 1] : 0;
  *total = warp_tot[kT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kT) k_chunk_sums(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * kItems;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if (base + k < n) s += in[base + k];
  int64_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA scans the chunk sums in place (exclusive), chunk of kT at a time.
__global__ void __launch_bounds__(kT) k_scan_sums(int64_t* __restrict__ sums, int64_t nb) {
  int64_t carry = 0;
  for (int64_t b = 0; b < nb; b += kT) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < nb ? sums[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
}

// out[i] = exclusive prefix of in (out may alias in); out[n] = total.
__global__ void __launch_bounds__(kT) k_chunk_scan(const int64_t* in, int64_t n, const int64_t* __restrict__ offs,
                                                   int64_t* out) {
  const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * kItems;
  int64_t v[kItems], s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t run = offs[blockIdx.x] + block_exclusive_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (base + k < n) out[base + k] = run;
    if (base + k == n - 1) out[n] = run + v[k];
    run += v[k];
  }
}

cudaError_t exclusive_scan(int64_t* data, int64_t n, int64_t* scratch, cudaStream_t s) {
  // data has n + 1 entries; scratch at least ceil(n / kChunk) entries
  if (n == 0) return cudaMemsetAsync(data, 0, sizeof(int64_t), s);
  const int64_t nb = (n + kChunk - 1) / kChunk;
  k_chunk_sums<<<(unsigned)nb, kT, 0, s>>>(data, n, scratch); lor_count_launch();
  k_scan_sums<<<1, kT, 0, s>>>(scratch, nb); lor_count_launch();
  k_chunk_scan<<<(unsigned)nb, kT, 0, s>>>(data, n, scratch, data); lor_count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pattern
__device__ __forceinline__ int64_t subhex_dof(const LorMesh& m, int64_t e, int s, int r) {
  const int P = m.p, n = P + 1;
  const int a = s % P, b = (s / P) % P, c = s / (P * P);
  return m.edofs[e * (int64_t)n * n * n + (a + (r & 1)) + n * ((b + ((r >> 1) & 1)) + n * (c + (r >> 2)))];
}

// Every map entry in range; counts 8 list slots per (sub-hex, vertex) incidence.
__global__ void k_incidence_count(LorMesh m, int64_t* __restrict__ cnt, int* __restrict__ status) {
  const int64_t P3 = (int64_t)m.p * m.p * m.p;
  int bad = 0;
  GRID_STRIDE(w, m.nel * P3 * 8) {
    const int64_t e = w / (P3 * 8);
    const int s = (int)((w / 8) % P3), r = (int)(w & 7);
    const int64_t d = subhex_dof(m, e, s, r);
    if (d < 0 || d >= m.ndof) {
      bad = 1;
      continue;
    }
    atomicAdd((unsigned long long*)(cnt + d), 8ull);
  }
  if (bad) atomicOr(status, LOR_FLAG_BAD_MAP);
}

__global__ void k_incidence_fill(LorMesh m, const int64_t* __restrict__ off, int64_t* __restrict__ cur,
                                 int32_t* __restrict__ list) {
  const int64_t P3 = (int64_t)m.p * m.p * m.p;
  GRID_STRIDE(w, m.nel * P3 * 8) {
    const int64_t e = w / (P3 * 8);
    const int s = (int)((w / 8) % P3), r = (int)(w & 7);
    const int64_t d = subhex_dof(m, e, s, r);
    if (d < 0 || d >= m.ndof) continue;
    const int64_t pos = off[d] + (int64_t)atomicAdd((unsigned long long*)(cur + d), 8ull);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int64_t c = subhex_dof(m, e, s, t);
      list[pos + t] = (int32_t)((c >= 0 && c < m.ndof) ? c : d);
    }
  }
}

// Sort each row's list in place (insertion sort: a few dozen entries) and
// count its distinct columns.
__global__ void k_row_sort_count(int64_t n, const int64_t* __restrict__ off, int32_t* __restrict__ list,
                                 int64_t* __restrict__ ucnt, int* __restrict__ status) {
  GRID_STRIDE(i, n) {
    const int64_t b = off[i], e = off[i + 1];
    if (e - b > kMaxRowList) {
      atomicOr(status, LOR_FLAG_BAD_MAP);
      ucnt[i] = 0;
      continue;
    }
    for (int64_t j = b + 1; j < e; ++j) {
      const int32_t v = list[j];
      int64_t k = j - 1;
      while (k >= b && list[k] > v) {
        list[k + 1] = list[k];
        --k;
      }
      list[k + 1] = v;
    }
    int64_t u = 0;
    for (int64_t j = b; j < e; ++j) u += (j == b || list[j] != list[j - 1]) ? 1 : 0;
    ucnt[i] = u;
  }
}

__global__ void k_row_write(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ list,
                            const int64_t* __restrict__ rowptr, int32_t* __restrict__ colidx) {
  GRID_STRIDE(i, n) {
    const int64_t b = off[i], e = off[i + 1];
    int64_t o = rowptr[i];
    if (rowptr[i + 1] - o == 0) continue;
    for (int64_t j = b; j < e; ++j)
      if (j == b || list[j] != list[j - 1]) colidx[o++] = list[j];
  }
}

// ---------------------------------------------------------------- edges (discrete gradient)
// The 12 edges of the unit cube as pairs of local vertices r = r0 + 2 r1 + 4 r2.
__constant__ int kEdgeA[12] = {0, 2, 4, 6, 0, 1, 4, 5, 0, 1, 2, 3};
__constant__ int kEdgeB[12] = {1, 3, 5, 7, 2, 3, 6, 7, 4, 5, 6, 7};

__device__ __forceinline__ void subhex_edge(const LorMesh& m, int64_t w, int64_t& tail, int64_t& head) {
  const int64_t P3 = (int64_t)m.p * m.p * m.p;
  const int64_t e = w / (P3 * 12);
  const int s = (int)((w / 12) % P3), k = (int)(w % 12);
  const int64_t a = subhex_dof(m, e, s, kEdgeA[k]), b = subhex_dof(m, e, s, kEdgeB[k]);
  tail = a < b ? a : b;
  head = a < b ? b : a;
}

__global__ void k_edge_count(LorMesh m, int64_t* __restrict__ cnt) {
  GRID_STRIDE(w, m.nel * (int64_t)m.p * m.p * m.p * 12) {
    int64_t t, h;
    subhex_edge(m, w, t, h);
    atomicAdd((unsigned long long*)(cnt + t), 1ull);
  }
}

__global__ void k_edge_fill(LorMesh m, const int64_t* __restrict__ off, int64_t* __restrict__ cur,
                            int32_t* __restrict__ list) {
  GRID_STRIDE(w, m.nel * (int64_t)m.p * m.p * m.p * 12) {
    int64_t t, h;
    subhex_edge(m, w, t, h);
    list[off[t] + (int64_t)atomicAdd((unsigned long long*)(cur + t), 1ull)] = (int32_t)h;
  }
}

__global__ void k_edge_write(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ list,
                             const int64_t* __restrict__ estart, int32_t* __restrict__ tail, int32_t* __restrict__ head) {
  GRID_STRIDE(i, n) {
    int64_t o = estart[i];
    if (estart[i + 1] == o) continue;
    for (int64_t j = off[i]; j < off[i + 1]; ++j)
      if (j == off[i] || list[j] != list[j - 1]) {
        tail[o] = (int32_t)i;
        head[o] = list[j];
        ++o;
      }
  }
}

__global__ void k_edges_to_csr(int64_t nedge, const int32_t* __restrict__ tail, const int32_t* __restrict__ head,
                               int64_t* __restrict__ rowptr, int32_t* __restrict__ colidx,
                               double* __restrict__ values) {
  GRID_STRIDE(i, nedge + 1) {
    rowptr[i] = 2 * i;
    if (i == nedge) break;
    reinterpret_cast<int2*>(colidx)[i] = make_int2(tail[i], head[i]);
    reinterpret_cast<double2*>(values)[i] = make_double2(-1.0, 1.0);
  }
}

// ---------------------------------------------------------------- vertex coordinates
__global__ void k_owner_min(LorMesh m, unsigned long long* __restrict__ owner) {
  const int64_t n3 = (int64_t)(m.p + 1) * (m.p + 1) * (m.p + 1);
  GRID_STRIDE(w, m.nel * n3) atomicMin(owner + m.edofs[w], (unsigned long long)(w / n3));
}

// Each DOF written once, by the lowest-index element that holds it: x =
// T_e(GLL node), the trilinear map through the element's corners.
__global__ void k_general_vertices(LorMesh m, LorTables T, const unsigned long long* __restrict__ owner,
                                   double* __restrict__ xyz) {
  const int n = m.p + 1;
  const int64_t n3 = (int64_t)n * n * n;
  GRID_STRIDE(w, m.nel * n3) {
    const int64_t e = w / n3, d = m.edofs[w];
    if (owner[d] != (unsigned long long)e) continue;
    const int loc = (int)(w % n3), i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const double l0[2] = {0.5 * (1.0 - T.gll[i]), 0.5 * (1.0 + T.gll[i])};
    const double l1[2] = {0.5 * (1.0 - T.gll[j]), 0.5 * (1.0 + T.gll[j])};
    const double l2[2] = {0.5 * (1.0 - T.gll[k]), 0.5 * (1.0 + T.gll[k])};
    double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      double X[3];
      lor_element_corner(m, e, c, X);
      const double wc = l0[c & 1] * l1[(c >> 1) & 1] * l2[c >> 2];
      x[0] += wc * X[0];
      x[1] += wc * X[1];
      x[2] += wc * X[2];
    }
    xyz[3 * d] = x[0];
    xyz[3 * d + 1] = x[1];
    xyz[3 * d + 2] = x[2];
  }
}

}  // namespace

// A block allocated through the context's allocator, released on scope exit
// unless kept.
template <typename T>
struct DevBuf {
  const LorDeviceAlloc& A;
  T* p = nullptr;
  size_t bytes = 0;
  explicit DevBuf(const LorDeviceAlloc& a) : A(a) {}
  cudaError_t get(int64_t count) {
    bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
    return A.alloc(A.ctx, (void**)&p, bytes);
  }
  T* keep() {
    T* q = p;
    p = nullptr;
    return q;
  }
  ~DevBuf() {
    if (p) A.release(A.ctx, p, bytes);
  }
};

cudaError_t lor_general_pattern(const LorMesh& m, const LorDeviceAlloc& A, int64_t** rowptr_out, int32_t** colidx_out,
                                int64_t* nnz_out, int* d_status, cudaStream_t s) {
  const int64_t n = m.ndof;
  const int64_t nb = (n + kChunk - 1) / kChunk + 1;
  DevBuf<int64_t> off(A), cur(A), scratch(A), rowptr(A);
  DevBuf<int32_t> list(A), colidx(A);
  int64_t total = 0, nnz = 0;
  cudaError_t err = off.get(n + 1);
  if (err == cudaSuccess) err = cur.get(n + 1);
  if (err == cudaSuccess) err = scratch.get(nb);
  if (err == cudaSuccess) err = cudaMemsetAsync(off.p, 0, sizeof(int64_t) * (n + 1), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(cur.p, 0, sizeof(int64_t) * (n + 1), s);
  if (err == cudaSuccess) {
    k_incidence_count<<<grid_for(m.nel * (int64_t)m.p * m.p * m.p * 8), kT, 0, s>>>(m, off.p, d_status);
    lor_count_launch();
    err = exclusive_scan(off.p, n, scratch.p, s);
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(&total, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = list.get(total);
  if (err == cudaSuccess) {
    k_incidence_fill<<<grid_for(m.nel * (int64_t)m.p * m.p * m.p * 8), kT, 0, s>>>(m, off.p, cur.p, list.p);
    lor_count_launch();
    k_row_sort_count<<<grid_for(n), kT, 0, s>>>(n, off.p, list.p, cur.p, d_status); lor_count_launch();
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = rowptr.get(n + 1);
  if (err == cudaSuccess) err = cudaMemcpyAsync(rowptr.p, cur.p, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s);
  if (err == cudaSuccess) err = exclusive_scan(rowptr.p, n, scratch.p, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(&nnz, rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = colidx.get(nnz + 4);  // 16 bytes of padding for the smoother's rounded bulk copies
  if (err == cudaSuccess) {
    k_row_write<<<grid_for(n), kT, 0, s>>>(n, off.p, list.p, rowptr.p, colidx.p); lor_count_launch();
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(s);  // nothing queued may still use a block freed on the way out
    return err;
  }
  *rowptr_out = rowptr.keep();
  *colidx_out = colidx.keep();
  *nnz_out = nnz;
  return cudaSuccess;
}

cudaError_t lor_general_edges(const LorMesh& m, const LorDeviceAlloc& A, int32_t** tail_out, int32_t** head_out,
                              int64_t* nedge_out, int* d_status, cudaStream_t s) {
  const int64_t n = m.ndof;
  const int64_t nb = (n + kChunk - 1) / kChunk + 1;
  const int64_t nw = m.nel * (int64_t)m.p * m.p * m.p * 12;
  DevBuf<int64_t> off(A), cur(A), scratch(A), estart(A);
  DevBuf<int32_t> list(A), tail(A), head(A);
  int64_t nedge = 0;
  cudaError_t err = off.get(n + 1);
  if (err == cudaSuccess) err = cur.get(n + 1);
  if (err == cudaSuccess) err = estart.get(n + 1);
  if (err == cudaSuccess) err = scratch.get(nb);
  if (err == cudaSuccess) err = list.get(nw);
  if (err == cudaSuccess) err = cudaMemsetAsync(off.p, 0, sizeof(int64_t) * (n + 1), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(cur.p, 0, sizeof(int64_t) * (n + 1), s);
  if (err == cudaSuccess) {
    k_edge_count<<<grid_for(nw), kT, 0, s>>>(m, off.p); lor_count_launch();
    err = exclusive_scan(off.p, n, scratch.p, s);
  }
  if (err == cudaSuccess) {
    k_edge_fill<<<grid_for(nw), kT, 0, s>>>(m, off.p, cur.p, list.p); lor_count_launch();
    k_row_sort_count<<<grid_for(n), kT, 0, s>>>(n, off.p, list.p, cur.p, d_status); lor_count_launch();
    err = cudaMemcpyAsync(estart.p, cur.p, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s);
  }
  if (err == cudaSuccess) err = exclusive_scan(estart.p, n, scratch.p, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(&nedge, estart.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = tail.get(nedge);
  if (err == cudaSuccess) err = head.get(nedge);
  if (err == cudaSuccess) {
    k_edge_write<<<grid_for(n), kT, 0, s>>>(n, off.p, list.p, estart.p, tail.p, head.p); lor_count_launch();
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(s);
    return err;
  }
  *tail_out = tail.keep();
  *head_out = head.keep();
  *nedge_out = nedge;
  return cudaSuccess;
}

cudaError_t lor_launch_general_gradient(int64_t nedge, const int32_t* tail, const int32_t* head, int64_t* rowptr,
                                        int32_t* colidx, double* values, cudaStream_t s) {
  k_edges_to_csr<<<grid_for(nedge + 1), kT, 0, s>>>(nedge, tail, head, rowptr, colidx, values); lor_count_launch();
  return cudaGetLastError();
}

cudaError_t lor_launch_general_vertices(const LorMesh& m, const LorTables& T, double* xyz, cudaStream_t s) {
  unsigned long long* owner = nullptr;
  const int64_t nw = m.nel * (int64_t)(m.p + 1) * (m.p + 1) * (m.p + 1);
  cudaError_t err = cudaMallocAsync(&owner, sizeof(unsigned long long) * m.ndof, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(owner, 0xff, sizeof(unsigned long long) * m.ndof, s);
  if (err == cudaSuccess) {
    k_owner_min<<<grid_for(nw), kT, 0, s>>>(m, owner); lor_count_launch();
    k_general_vertices<<<grid_for(nw), kT, 0, s>>>(m, T, owner, xyz); lor_count_launch();
    err = cudaGetLastError();
  }
  if (owner) {
    const cudaError_t e2 = cudaFreeAsync(owner, s);
    if (err == cudaSuccess) err = e2;
  }
  return err;
}

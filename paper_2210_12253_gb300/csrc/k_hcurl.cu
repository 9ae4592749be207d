// k_hcurl.cu -- the topological inputs the paper's H(curl) solver (AMS)
// needs from the LOR mesh (Section 3, after Step S1.2): the discrete gradient
// matrix (Algorithm 1) and the deduplicated LOR vertex coordinates.
//
// Discrete gradient: one thread per LOR edge, as in Algorithm 1, but the
// macro-element maps it reads (element, local edge, its two local vertices,
// orientation, local-to-global) collapse on the structured grid of macro
// elements into closed form: edge i is an x-, y- or z-directed edge (x-edges
// numbered first), its tail vertex follows from i lexicographically and its
// head is the next vertex along the axis; the tail has the lower global
// index, so the row is (tail: -1, head: +1) with ascending columns.  The
// kernel is pure integer/HBM work: 8 bytes of row pointer and 24 bytes of
// (column, value) pairs written per edge.
//
// Vertex coordinates: every deduplicated vertex (global GLL grid point) is
// x = T_e(GLL point) on the lowest-index element containing it.
#include "lor_internal.cuh"

namespace {

__global__ void k_discrete_gradient(LorMesh m, int64_t nedge, int64_t* __restrict__ rowptr,
                                    int32_t* __restrict__ colidx, double* __restrict__ values) {
  const int64_t nxe = (m.nx - 1) * m.ny * m.nz, nye = m.nx * (m.ny - 1) * m.nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nedge; i += (int64_t)gridDim.x * blockDim.x) {
    rowptr[i] = 2 * i;
    if (i == nedge) break;
    int64_t r = i, mx = m.nx, my = m.ny, stride;
    if (r < nxe) {
      mx = m.nx - 1;
      stride = 1;
    } else if (r < nxe + nye) {
      r -= nxe;
      my = m.ny - 1;
      stride = m.nx;
    } else {
      r -= nxe + nye;
      stride = m.nx * m.ny;
    }
    const int64_t I = r % mx, J = (r / mx) % my, K = r / (mx * my);
    const int64_t tail = I + m.nx * (J + m.ny * K);
    // colidx and values as aligned pairs: one 8-byte and one 16-byte store
    reinterpret_cast<int2*>(colidx)[i] = make_int2((int)tail, (int)(tail + stride));
    reinterpret_cast<double2*>(values)[i] = make_double2(-1.0, 1.0);
  }
}

// One CTA per element writes the vertices it owns (the lowest-index element
// containing each vertex: local index 0..p-1 per axis, 0..p on the last
// element of an axis).  The trilinear map is evaluated by successive linear
// interpolation: the 4 edges along x at the n GLL abscissae, then the 2
// faces at the n^2 (i, j) pairs, then the vertices, about 6 FP64 operations
// per vertex instead of 42 for the 8-corner sum.
constexpr int kMaxN = LOR_MAX_P + 1;

__global__ void __launch_bounds__(128) k_vertex_coordinates(LorMesh m, LorTables T, double* __restrict__ xyz) {
  __shared__ double X[8][3];
  __shared__ double l0[kMaxN], l1[kMaxN];
  __shared__ double Ex[4][kMaxN][3];           // edges along x: (c1, c2) = (0,0), (1,0), (0,1), (1,1)
  __shared__ double Fx[2][kMaxN * kMaxN][3];   // faces: c2 = 0, 1
  const int P = m.p, n = P + 1;
  if (threadIdx.x < n) {
    l0[threadIdx.x] = 0.5 * (1.0 - T.gll[threadIdx.x]);
    l1[threadIdx.x] = 0.5 * (1.0 + T.gll[threadIdx.x]);
  }
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < 8) lor_element_corner(m, e, threadIdx.x, X[threadIdx.x]);
    __syncthreads();
    for (int w = threadIdx.x; w < 4 * n * 3; w += blockDim.x) {
      const int edge = w / (3 * n), i = (w / 3) % n, d = w % 3;
      const int c = 2 * (edge & 1) + 4 * (edge >> 1);  // corner with c0 = 0 on this edge
      Ex[edge][i][d] = l0[i] * X[c][d] + l1[i] * X[c + 1][d];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < 2 * n * n * 3; w += blockDim.x) {
      const int face = w / (3 * n * n), ij = (w / 3) % (n * n), d = w % 3;
      const int i = ij % n, j = ij / n;
      Fx[face][ij][d] = l0[j] * Ex[2 * face][i][d] + l1[j] * Ex[2 * face + 1][i][d];
    }
    __syncthreads();
    const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
    const int ni = ex == m.nex - 1 ? n : P, nj = ey == m.ney - 1 ? n : P, nk = ez == m.nez - 1 ? n : P;
    for (int w = threadIdx.x; w < ni * nj * nk; w += blockDim.x) {
      const int i = w % ni, j = (w / ni) % nj, k = w / (ni * nj);
      const int ij = i + n * j;
      const int64_t v = (ex * P + i) + m.nx * ((ey * P + j) + m.ny * (ez * P + k));
#pragma unroll
      for (int d = 0; d < 3; ++d) xyz[3 * v + d] = l0[k] * Fx[0][ij][d] + l1[k] * Fx[1][ij][d];
    }
  }
}

int grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

int64_t lor_edge_count(const LorMesh& m) {
  return (m.nx - 1) * m.ny * m.nz + m.nx * (m.ny - 1) * m.nz + m.nx * m.ny * (m.nz - 1);
}

cudaError_t lor_launch_discrete_gradient(const LorMesh& m, int64_t* rowptr, int32_t* colidx, double* values,
                                         cudaStream_t s) {
  const int64_t ne = lor_edge_count(m);
  k_discrete_gradient<<<grid_for(ne + 1), 256, 0, s>>>(m, ne, rowptr, colidx, values); lor_count_launch();
  return cudaGetLastError();
}

cudaError_t lor_launch_vertex_coordinates(const LorMesh& m, const LorTables& T, double* xyz, cudaStream_t s) {
  const int g = (int)(m.nel < 152 * 16 ? m.nel : 152 * 16);
  k_vertex_coordinates<<<g, 128, 0, s>>>(m, T, xyz); lor_count_launch();
  return cudaGetLastError();
}

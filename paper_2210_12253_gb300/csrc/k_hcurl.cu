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
// Vertex coordinates: one thread per deduplicated vertex (global GLL grid
// point): x = T_e(GLL point) on the lowest-index element containing it.
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

__global__ void k_vertex_coordinates(LorMesh m, LorTables T, double* __restrict__ xyz) {
  const int P = m.p;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < m.ndof; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = v % m.nx, J = (v / m.nx) % m.ny, K = v / (m.nx * m.ny);
    const int64_t ex = I / P < m.nex ? I / P : m.nex - 1;
    const int64_t ey = J / P < m.ney ? J / P : m.ney - 1;
    const int64_t ez = K / P < m.nez ? K / P : m.nez - 1;
    const int i = (int)(I - ex * P), j = (int)(J - ey * P), k = (int)(K - ez * P);
    const int64_t e = ex + m.nex * (ey + (int64_t)m.ney * ez);
    const double l0[2] = {0.5 * (1.0 - T.gll[i]), 0.5 * (1.0 + T.gll[i])};
    const double l1[2] = {0.5 * (1.0 - T.gll[j]), 0.5 * (1.0 + T.gll[j])};
    const double l2[2] = {0.5 * (1.0 - T.gll[k]), 0.5 * (1.0 + T.gll[k])};
    double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      double X[3];
      lor_element_corner(m, e, c, X);
      const double w = l0[c & 1] * l1[(c >> 1) & 1] * l2[c >> 2];
      x[0] += w * X[0];
      x[1] += w * X[1];
      x[2] += w * X[2];
    }
    xyz[3 * v] = x[0];
    xyz[3 * v + 1] = x[1];
    xyz[3 * v + 2] = x[2];
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
  k_vertex_coordinates<<<grid_for(m.ndof), 256, 0, s>>>(m, T, xyz); lor_count_launch();
  return cudaGetLastError();
}

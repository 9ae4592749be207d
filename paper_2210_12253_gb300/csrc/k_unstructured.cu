// k_unstructured.cu -- the unstructured LOR assembly the paper measures its
// macro-element algorithm against (Section 4.2, kernel throughput): the LOR
// mesh is handed over as a general hex mesh (E-vectors of vertex coordinates
// and of global DOF ids per sub-hex, one coefficient per sub-hex), each
// sub-hex's 8x8 block is formed by 8 threads (one per local DOF, i.e. one row
// of the block) and added into a given CSR matrix at positions found by
// binary search in the row's sorted column indices.  Nothing of the
// macro-element structure is used, so the kernel assembles the Q1 (2x2x2
// Gauss) diffusion(-reaction) matrix of any conforming hex mesh.
//
// k_lor_mesh builds those E-vectors from the context (the LOR mesh
// construction the unstructured path needs and the macro-element path
// avoids): sub-hex vertices T_e(GLL tensor points), global DOF ids, kappa_s
// and beta_s binned as in the macro-element assembly, and the essential mask.
#include "lor_internal.cuh"

namespace {

constexpr int kSubPerCta = 32;  // sub-hexes per CTA, 8 threads each
constexpr int kUThreads = 8 * kSubPerCta;

// Sub-hex s = a + p (b + p c) of element e (element-major).
template <int P>
__global__ void __launch_bounds__(128) k_lor_mesh(LorMesh m, LorTables T, const double* __restrict__ kappa,
                                                  const double* __restrict__ beta, double* __restrict__ corners,
                                                  int64_t* __restrict__ dofs, double* __restrict__ ksub,
                                                  double* __restrict__ bsub, uint8_t* __restrict__ ess) {
  constexpr int Q = P + 2, Q3 = Q * Q * Q, P3 = P * P * P;
  __shared__ double X[8][3];
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    if (threadIdx.x < 8) lor_element_corner(m, e, threadIdx.x, X[threadIdx.x]);
    __syncthreads();
    const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
    for (int w = threadIdx.x; w < P3 * 8; w += blockDim.x) {
      const int s = w >> 3, r = w & 7;
      const int a = s % P, b = (s / P) % P, c = s / (P * P);
      const int i = a + (r & 1), j = b + ((r >> 1) & 1), k = c + (r >> 2);
      // trilinear map of the element at the GLL point (i, j, k)
      const double l0[2] = {0.5 * (1.0 - T.gll[i]), 0.5 * (1.0 + T.gll[i])};
      const double l1[2] = {0.5 * (1.0 - T.gll[j]), 0.5 * (1.0 + T.gll[j])};
      const double l2[2] = {0.5 * (1.0 - T.gll[k]), 0.5 * (1.0 + T.gll[k])};
      double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const double wgt = l0[cc & 1] * l1[(cc >> 1) & 1] * l2[cc >> 2];
        x[0] += wgt * X[cc][0];
        x[1] += wgt * X[cc][1];
        x[2] += wgt * X[cc][2];
      }
      const int64_t sg = e * P3 + s;
      double* out = corners + (sg * 8 + r) * 3;
      out[0] = x[0];
      out[1] = x[1];
      out[2] = x[2];
      const int64_t I = ex * P + i, J = ey * P + j, K = ez * P + k;
      const int64_t dof = I + m.nx * (J + m.ny * K);
      dofs[sg * 8 + r] = dof;
      if (ess && (a == 0 || a == P - 1 || b == 0 || b == P - 1 || c == 0 || c == P - 1))
        ess[dof] = lor_is_essential(I, J, K, m.nx, m.ny, m.nz) ? 1 : 0;
      if (r == 0) {
        double ks = 0.0, bs = 0.0;
        for (int g2 = T.bin_first[c]; g2 < T.bin_first[c] + T.bin_count[c]; ++g2)
          for (int g1 = T.bin_first[b]; g1 < T.bin_first[b] + T.bin_count[b]; ++g1)
            for (int g0 = T.bin_first[a]; g0 < T.bin_first[a] + T.bin_count[a]; ++g0) {
              const double wq = T.bin_w[g0] * T.bin_w[g1] * T.bin_w[g2];
              const int64_t pt = e * Q3 + g0 + Q * (g1 + Q * g2);
              ks += wq * kappa[pt];
              if (beta) bs += wq * beta[pt];
            }
        ksub[sg] = ks;
        if (bsub) bsub[sg] = bs;
      }
    }
    __syncthreads();
  }
}

// Interior DOFs of the elements are never essential; the element-boundary
// pass above only writes DOFs on sub-hexes touching the element boundary, so
// the mask is cleared first.
__global__ void k_zero_u8(uint8_t* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 0;
}

// One 8-thread group per sub-hex: thread g first evaluates the geometry at
// Gauss point g (tau = eps / sqrt 3), then thread r forms row r of the block
//   K_rc = sum_g kappa_s grad phi_r^T (adj(J) adj(J)^T / detJ) grad phi_c
//          (+ beta_s detJ phi_r phi_c)
// in FP64 and adds it into the CSR values (VT).  Rows and columns with
// ess != 0 are skipped (their diagonal is preset to 1 elsewhere).
template <typename VT, bool MASS>
__global__ void __launch_bounds__(kUThreads) k_assemble_unstructured(
    int64_t nsub, const double* __restrict__ corners, const int64_t* __restrict__ dofs,
    const double* __restrict__ ksub, const double* __restrict__ bsub, const int64_t* __restrict__ rowptr,
    const int32_t* __restrict__ colidx, const uint8_t* __restrict__ ess, VT* __restrict__ vals,
    int* __restrict__ status) {
  __shared__ double X[kSubPerCta][8][3];
  __shared__ double G[kSubPerCta][8][7];  // 6 metric entries and detJ per Gauss point
  __shared__ double dphi[8][8][3];        // reference gradients: [g][c][k]
  __shared__ double phi[8][8];            // values: [g][c]
  // reference tables of the trilinear basis at the 2x2x2 Gauss points
  for (int w = threadIdx.x; w < 64; w += blockDim.x) {
    const int g = w >> 3, c = w & 7;
    double l[3], dl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double tau = (((g >> k) & 1) ? 1.0 : -1.0) * 0.57735026918962576451;
      const double sc = ((c >> k) & 1) ? 1.0 : -1.0;
      l[k] = 0.5 * (1.0 + sc * tau);
      dl[k] = 0.5 * sc;
    }
    phi[g][c] = l[0] * l[1] * l[2];
    dphi[g][c][0] = dl[0] * l[1] * l[2];
    dphi[g][c][1] = l[0] * dl[1] * l[2];
    dphi[g][c][2] = l[0] * l[1] * dl[2];
  }
  const int ls = threadIdx.x >> 3, lane = threadIdx.x & 7;
  int bad = 0;
  for (int64_t s0 = (int64_t)blockIdx.x * kSubPerCta; s0 < nsub; s0 += (int64_t)gridDim.x * kSubPerCta) {
    const int64_t s = s0 + ls;
    const bool live = s < nsub;
    if (live) {
      const double* xs = corners + (s * 8 + lane) * 3;
      X[ls][lane][0] = xs[0];
      X[ls][lane][1] = xs[1];
      X[ls][lane][2] = xs[2];
    }
    __syncthreads();
    if (live) {  // geometry at Gauss point g = lane
      double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) J[i][k] += X[ls][c][i] * dphi[lane][c][k];
      const double c0[3] = {J[0][0], J[1][0], J[2][0]}, c1[3] = {J[0][1], J[1][1], J[2][1]},
                   c2[3] = {J[0][2], J[1][2], J[2][2]};
      double a0[3], a1[3], a2[3];
      lor_cross(c1, c2, a0);
      lor_cross(c2, c0, a1);
      lor_cross(c0, c1, a2);
      const double det = c0[0] * a0[0] + c0[1] * a0[1] + c0[2] * a0[2];
      if (!(det > 0.0)) bad = 1;
      const double r = 1.0 / det;
      double* g = G[ls][lane];
      g[0] = r * (a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2]);
      g[1] = r * (a0[0] * a1[0] + a0[1] * a1[1] + a0[2] * a1[2]);
      g[2] = r * (a0[0] * a2[0] + a0[1] * a2[1] + a0[2] * a2[2]);
      g[3] = r * (a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
      g[4] = r * (a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2]);
      g[5] = r * (a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
      g[6] = det;
    }
    __syncthreads();
    if (live) {  // row r = lane of the block
      const int rr = lane;
      const double ks = ksub[s];
      const double bs = MASS ? bsub[s] : 0.0;
      double K[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const double* gm = G[ls][g];
        const double d0 = dphi[g][rr][0], d1 = dphi[g][rr][1], d2 = dphi[g][rr][2];
        const double t0 = ks * (gm[0] * d0 + gm[1] * d1 + gm[2] * d2);
        const double t1 = ks * (gm[1] * d0 + gm[3] * d1 + gm[4] * d2);
        const double t2 = ks * (gm[2] * d0 + gm[4] * d1 + gm[5] * d2);
        const double mr = MASS ? bs * gm[6] * phi[g][rr] : 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          K[c] += t0 * dphi[g][c][0] + t1 * dphi[g][c][1] + t2 * dphi[g][c][2];
          if (MASS) K[c] += mr * phi[g][c];
        }
      }
      const int64_t R = dofs[s * 8 + rr];
      if (!(ess && ess[R])) {
        const int64_t b = rowptr[R], e = rowptr[R + 1];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t C = dofs[s * 8 + c];
          if (ess && ess[C]) continue;
          const int64_t pos = lor_find_col(colidx, b, e, C);
          if (pos < 0) {
            bad |= 2;
            continue;
          }
          atomicAdd(vals + pos, (VT)K[c]);
        }
      }
    }
    __syncthreads();
  }
  if (bad & 1) atomicOr(status, LOR_FLAG_BAD_GEOM);
  if (bad & 2) atomicOr(status, LOR_FLAG_BAD_PATTERN);
}

// Diagonal of every essential row = 1 (values zeroed before).
template <typename VT>
__global__ void k_unstructured_diag(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                    const uint8_t* __restrict__ ess, VT* __restrict__ vals, int* __restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!ess[i]) continue;
    const int64_t pos = lor_find_col(colidx, rowptr[i], rowptr[i + 1], i);
    if (pos < 0) atomicOr(status, LOR_FLAG_BAD_PATTERN);
    else vals[pos] = (VT)1;
  }
}

template <typename VT>
cudaError_t launch_unstructured(int64_t nsub, const double* corners, const int64_t* dofs, const double* ksub,
                                const double* bsub, int64_t n, int64_t nnz, const int64_t* rowptr,
                                const int32_t* colidx, const uint8_t* ess, VT* vals, int* status, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(vals, 0, sizeof(VT) * nnz, s);
  if (err != cudaSuccess) return err;
  if (ess) {
    const int64_t blocks = (n + 255) / 256;
    k_unstructured_diag<VT><<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(n, rowptr, colidx, ess, vals,
                                                                                         status); lor_count_launch();
  }
  if (nsub == 0) return cudaGetLastError();
  const int64_t need = (nsub + kSubPerCta - 1) / kSubPerCta;
  const int grid = (int)(need < 152 * 64 ? need : 152 * 64);
  if (bsub) {
    k_assemble_unstructured<VT, true><<<grid, kUThreads, 0, s>>>(nsub, corners, dofs, ksub, bsub, rowptr, colidx,
                                                                 ess, vals, status); lor_count_launch();
  } else {
    k_assemble_unstructured<VT, false><<<grid, kUThreads, 0, s>>>(nsub, corners, dofs, ksub, nullptr, rowptr, colidx,
                                                                  ess, vals, status); lor_count_launch();
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t lor_launch_lor_mesh(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta,
                                double* corners, int64_t* dofs, double* ksub, double* bsub, uint8_t* ess,
                                cudaStream_t s) {
  if (ess) {
    const int64_t blocks = (m.ndof + 255) / 256;
    k_zero_u8<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(ess, m.ndof); lor_count_launch();
  }
  const int g = (int)(m.nel < 152 * 64 ? m.nel : 152 * 64);
  switch (m.p) {
#define LOR_CASE(P) \
  case P: k_lor_mesh<P><<<g, 128, 0, s>>>(m, T, kappa, beta, corners, dofs, ksub, bsub, ess); lor_count_launch(); break;
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t lor_launch_assemble_unstructured(int64_t nsub, const double* corners, const int64_t* dofs,
                                             const double* ksub, const double* bsub, int64_t n, int64_t nnz,
                                             const int64_t* rowptr, const int32_t* colidx, const uint8_t* ess,
                                             void* vals, int dtype, int* status, cudaStream_t s) {
  if (dtype == LOR_F64)
    return launch_unstructured<double>(nsub, corners, dofs, ksub, bsub, n, nnz, rowptr, colidx, ess, (double*)vals,
                                       status, s);
  return launch_unstructured<float>(nsub, corners, dofs, ksub, bsub, n, nnz, rowptr, colidx, ess, (float*)vals, status,
                                    s);
}

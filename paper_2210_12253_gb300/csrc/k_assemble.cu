// k_assemble.cu -- Step S1.2 / A1 + A4: batched LOR matrix assembly.
//
// One CTA per macro element (a high-order element split at the Gauss-Lobatto
// points into p^3 sub-hexes, Section 2.1), one thread per sub-hex, as in the
// paper's A1 (one block per macro element, one thread per sub-element).  Each
// thread forms its sub-hex's 8x8 stiffness block by 2x2x2 Gauss quadrature on
// the sub-hex's trilinear map with the sub-hex coefficient kappa_s (the
// Gauss-weight average of kappa over the high-order Gauss points inside the
// sub-hex), then adds the entries straight into the CSR values at positions
// computed in closed form (no macro-element sparse block is stored), with
// FP64/FP32 atomics for the entries shared between sub-hexes.  Rows and
// columns of essential DOFs are skipped and their diagonal pre-set to 1 (A4),
// so elimination costs no extra pass.
//
// Geometry: the sub-hex map is the element's trilinear map restricted to the
// sub-box, so J_sub(tau) = J_e(xi(tau)) diag(r_a, r_b, r_c) with r the half
// widths of the GLL intervals; only the element Jacobian columns (bilinear in
// the two other coordinates) are evaluated, in FP64.
#include "lor_internal.cuh"

namespace {

// Trilinear basis on the sub-hex reference cube at the 2x2x2 Gauss points
// tau = +-1/sqrt(3): l_0(tau) = (1 - tau)/2, l_1(tau) = (1 + tau)/2.
constexpr double kLa = 0.78867513459481288225;  // (1 + 1/sqrt(3)) / 2: l_i at the Gauss point on its own side
constexpr double kLb = 0.21132486540518711775;  // (1 - 1/sqrt(3)) / 2
__device__ __forceinline__ constexpr double lval(int i, int g) { return i == g ? kLa : kLb; }
__device__ __forceinline__ constexpr double dval(int i) { return i ? 0.5 : -0.5; }
// d phi_i / d tau_d at Gauss point g (vertex i = i0 + 2 i1 + 4 i2, g likewise).
__device__ __forceinline__ constexpr double dphi(int g, int i, int d) {
  return d == 0 ? dval(i & 1) * lval((i >> 1) & 1, (g >> 1) & 1) * lval(i >> 2, g >> 2)
       : d == 1 ? lval(i & 1, g & 1) * dval((i >> 1) & 1) * lval(i >> 2, g >> 2)
                : lval(i & 1, g & 1) * lval((i >> 1) & 1, (g >> 1) & 1) * dval(i >> 2);
}

__device__ __forceinline__ int upper(int i, int j) {  // packed index of (min, max) in an 8x8 upper triangle
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a * 8 - (a * (a - 1)) / 2 + (b - a);
}

template <int P>
constexpr int kAsmThreads = ((P * P * P + 31) / 32) * 32 < 256 ? ((P * P * P + 31) / 32) * 32 : 256;

template <typename VT>
__device__ __forceinline__ void atomic_add(VT* p, double v);
template <>
__device__ __forceinline__ void atomic_add<double>(double* p, double v) { atomicAdd(p, v); }
template <>
__device__ __forceinline__ void atomic_add<float>(float* p, double v) { atomicAdd(p, (float)v); }

template <int P, typename VT>
__global__ void __launch_bounds__(kAsmThreads<P>) k_assemble(LorMesh m, LorTables T,
                                                                          const double* __restrict__ kappa,
                                                                          VT* __restrict__ vals) {
  constexpr int Q = P + 2, Q3 = Q * Q * Q, P3 = P * P * P;
  __shared__ double Ehalf[36];
  const int64_t e = blockIdx.x;
  const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
  for (int idx = threadIdx.x; idx < 36; idx += blockDim.x) {
    const int d = idx / 12, pair = (idx / 3) % 4, comp = idx % 3;
    const int o0 = pair & 1, o1 = pair >> 1;
    const int lo = d == 0 ? 2 * o0 + 4 * o1 : d == 1 ? o0 + 4 * o1 : o0 + 2 * o1;
    const int hi = lo + (1 << d);
    auto corner = [&](int c) {
      const int64_t va = ex + (c & 1), vb = ey + ((c >> 1) & 1), vc = ez + ((c >> 2) & 1);
      return m.verts[3 * (va + (int64_t)(m.nex + 1) * (vb + (int64_t)(m.ney + 1) * vc)) + comp];
    };
    Ehalf[idx] = 0.5 * (corner(hi) - corner(lo));
  }
  __syncthreads();
  for (int s = threadIdx.x; s < P3; s += blockDim.x) {
  const int a = s % P, b = (s / P) % P, c = s / (P * P);

  // kappa_s: Gauss-weight average over the high-order points in the sub-hex.
  double ks = 0.0;
  for (int g2 = T.bin_first[c]; g2 < T.bin_first[c] + T.bin_count[c]; ++g2)
    for (int g1 = T.bin_first[b]; g1 < T.bin_first[b] + T.bin_count[b]; ++g1)
      for (int g0 = T.bin_first[a]; g0 < T.bin_first[a] + T.bin_count[a]; ++g0)
        ks += T.bin_w[g0] * T.bin_w[g1] * T.bin_w[g2] * kappa[e * Q3 + g0 + Q * (g1 + Q * g2)];

  const double ra = T.sub_r[a], rb = T.sub_r[b], rc = T.sub_r[c];
  // G_sub^{ab} = (r_a r_b r_c)/(r_a r_b) (adj_a . adj_b) / det_e
  const double F00 = rb * rc / ra, F11 = ra * rc / rb, F22 = ra * rb / rc;
  const double F01 = rc, F02 = rb, F12 = ra;
  double K[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) K[i] = 0.0;

#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const int t0 = 2 * a + (g & 1), t1 = 2 * b + ((g >> 1) & 1), t2 = 2 * c + (g >> 2);
    const double u0 = T.sub_l0[t0], u1 = T.sub_l1[t0];
    const double v0 = T.sub_l0[t1], v1 = T.sub_l1[t1];
    const double w0 = T.sub_l0[t2], w1 = T.sub_l1[t2];
    double col[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      col[0][q] = w0 * (v0 * Ehalf[0 + q] + v1 * Ehalf[3 + q]) + w1 * (v0 * Ehalf[6 + q] + v1 * Ehalf[9 + q]);
      col[1][q] = w0 * (u0 * Ehalf[12 + q] + u1 * Ehalf[15 + q]) + w1 * (u0 * Ehalf[18 + q] + u1 * Ehalf[21 + q]);
      col[2][q] = v0 * (u0 * Ehalf[24 + q] + u1 * Ehalf[27 + q]) + v1 * (u0 * Ehalf[30 + q] + u1 * Ehalf[33 + q]);
    }
    double A0[3], A1[3], A2[3];
    A0[0] = col[1][1] * col[2][2] - col[1][2] * col[2][1];
    A0[1] = col[1][2] * col[2][0] - col[1][0] * col[2][2];
    A0[2] = col[1][0] * col[2][1] - col[1][1] * col[2][0];
    A1[0] = col[2][1] * col[0][2] - col[2][2] * col[0][1];
    A1[1] = col[2][2] * col[0][0] - col[2][0] * col[0][2];
    A1[2] = col[2][0] * col[0][1] - col[2][1] * col[0][0];
    A2[0] = col[0][1] * col[1][2] - col[0][2] * col[1][1];
    A2[1] = col[0][2] * col[1][0] - col[0][0] * col[1][2];
    A2[2] = col[0][0] * col[1][1] - col[0][1] * col[1][0];
    const double det = col[0][0] * A0[0] + col[0][1] * A0[1] + col[0][2] * A0[2];
    const double f = ks / det;
    const double G00 = f * F00 * (A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2]);
    const double G01 = f * F01 * (A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2]);
    const double G02 = f * F02 * (A0[0] * A2[0] + A0[1] * A2[1] + A0[2] * A2[2]);
    const double G11 = f * F11 * (A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2]);
    const double G12 = f * F12 * (A1[0] * A2[0] + A1[1] * A2[1] + A1[2] * A2[2]);
    const double G22 = f * F22 * (A2[0] * A2[0] + A2[1] * A2[1] + A2[2] * A2[2]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const double d0 = dphi(g, i, 0), d1 = dphi(g, i, 1), d2 = dphi(g, i, 2);
      const double t0v = G00 * d0 + G01 * d1 + G02 * d2;
      const double t1v = G01 * d0 + G11 * d1 + G12 * d2;
      const double t2v = G02 * d0 + G12 * d1 + G22 * d2;
#pragma unroll
      for (int j = i; j < 8; ++j) K[upper(i, j)] += dphi(g, j, 0) * t0v + dphi(g, j, 1) * t1v + dphi(g, j, 2) * t2v;
    }
  }

  // Scatter into the CSR values (closed-form positions), skipping essential
  // rows and columns (their diagonal was pre-set to 1).
  const int64_t I0 = ex * P + a, J0 = ey * P + b, K0 = ez * P + c;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t I = I0 + (r & 1), J = J0 + ((r >> 1) & 1), Kk = K0 + (r >> 2);
    if (lor_is_essential(I, J, Kk, m.nx, m.ny, m.nz)) continue;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int64_t I2 = I0 + (t & 1), J2 = J0 + ((t >> 1) & 1), K2 = K0 + (t >> 2);
      if (lor_is_essential(I2, J2, K2, m.nx, m.ny, m.nz)) continue;
      const int64_t pos = lor_entry_pos(I, J, Kk, (t & 1) - (r & 1), ((t >> 1) & 1) - ((r >> 1) & 1),
                                        (t >> 2) - (r >> 2), m.nx, m.ny, m.nz);
      atomic_add<VT>(vals + pos, K[upper(r, t)]);
    }
  }
  }  // sub-hex loop
}

// Diagonal of every essential row = 1 (the values are zeroed before).
template <typename VT>
__global__ void k_essential_diagonal(LorMesh m, VT* __restrict__ vals) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m.ndof; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = r % m.nx, J = (r / m.nx) % m.ny, K = r / (m.nx * m.ny);
    if (lor_is_essential(I, J, K, m.nx, m.ny, m.nz)) vals[lor_entry_pos(I, J, K, 0, 0, 0, m.nx, m.ny, m.nz)] = (VT)1;
  }
}

template <typename VT>
cudaError_t launch(const LorMesh& m, const LorTables& T, const double* kappa, VT* vals, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(vals, 0, sizeof(VT) * m.nnz, s);
  if (err != cudaSuccess) return err;
  {
    const int64_t blocks = (m.ndof + 255) / 256;
    k_essential_diagonal<VT><<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(m, vals); lor_count_launch();
  }
  switch (m.p) {
#define LOR_CASE(P) \
  case P: k_assemble<P, VT><<<(unsigned)m.nel, kAsmThreads<P>, 0, s>>>(m, T, kappa, vals); lor_count_launch(); break;
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t lor_launch_assemble(const LorMesh& m, const LorTables& T, const double* kappa, void* values, int dtype,
                                cudaStream_t s) {
  if (dtype == LOR_F64) return launch<double>(m, T, kappa, (double*)values, s);
  return launch<float>(m, T, kappa, (float*)values, s);
}

// k_geom.cu -- Step S1.1 (high-order operator setup, partial assembly) and the
// geometry helpers shared by it: Jacobians of the trilinear element maps at
// Gauss points, D = kappa w detJ J^-1 J^-T, the geometry validity check, and
// the load vector.
//
// GB300 notes: FP64 runs at about 2 DFMA/clk/SM on this part (1/64 of FP32),
// so these kernels would be bound by FP64 issue, not by HBM.  A trilinear map
// has dx/dxi_0 independent of xi_0 (and likewise for the other columns), so
// each Jacobian column is tabulated once per element on a q x q grid in shared
// memory; per point the metric follows from their cross and dot products,
// formed in 64-bit fixed point on the integer pipe (fixed_point.cuh), as the
// LOR assembly does.
#include "fixed_point_metric.cuh"
#include "lor_internal.cuh"

namespace {

// D = kappa w detJ J^-1 J^-T = kappa w adj(J^T J) / det J, with adj(J^T J)_ab
// = r_a . r_b for the adjugate rows r_a = c_b x c_c of J (columns c_d,
// (a, b, c) cyclic) and det J = c_0 . r_0: formed this way the error stays
// O(eps cond(J)), where the cofactors of M = J^T J lose O(eps cond(J)^2) on
// stretched or skewed elements (5e-8 of the largest entry at cond(J) = 1e5
// in FP64).  The Jacobian columns are tabulated per element (a trilinear
// map's dx/dxi_0 does not depend on xi_0, and so on) and converted to 64-bit
// fixed point, one scale per column table; per Gauss point the cross and dot
// products run on the integer pipe (fixed_point.cuh: fx_metric), 1/det J
// (range-reduced) and kappa w times it in FP64, D_ab = (kappa w / det J)
// adj(M)_ab in fixed point, stored in the form the FP64 operator multiplies it
// in (the point's six entries at its largest).  det J > 0 is checked here; its
// sign was checked at context creation too (the mesh does not change
// afterwards).
template <int P>
__global__ void __launch_bounds__(128) k_setup(LorMesh m, LorTables T, const double* __restrict__ kin,
                                               double* __restrict__ kcopy, double* __restrict__ Dq,
                                               int* __restrict__ status) {
  constexpr int Q = P + 2, Q2 = Q * Q, Q3 = Q * Q * Q, CT = Q2 * 3;
  __shared__ double Ehalf[36];
  __shared__ double col[3 * CT];
  __shared__ long long colx[3 * CT];  // the columns in fixed point, one scale per table (1079 - cexp)
  __shared__ int cexp[3];
  __shared__ double sw[Q], s0[Q], s1[Q];
  if (threadIdx.x < Q) {
    sw[threadIdx.x] = T.gw[threadIdx.x];
    s0[threadIdx.x] = T.gl0[threadIdx.x];
    s1[threadIdx.x] = T.gl1[threadIdx.x];
  }
  __syncthreads();
  int bad = 0;
  int* sdq = lor_d_scales(Dq, m.nel * Q3);
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    lor_jacobian_columns(m, e, s0, s1, Q, Ehalf, col);
    if (threadIdx.x < 3) cexp[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * CT; i += blockDim.x) atomicMax(&cexp[i / CT], fx_expo(col[i]));
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * CT; i += blockDim.x) colx[i] = fx_pack(fx_from_double(col[i], cexp[i / CT]));
    __syncthreads();
    const int scs[3] = {1079 - cexp[0], 1079 - cexp[1], 1079 - cexp[2]};
    for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
      const int g0 = pt % Q, g1 = (pt / Q) % Q, g2 = pt / Q2;
      Fx C[3][3];  // C[d][k]: component k of column d
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C[0][k] = fx_unpack(colx[3 * (g1 + Q * g2) + k]);
        C[1][k] = fx_unpack(colx[CT + 3 * (g0 + Q * g2) + k]);
        C[2][k] = fx_unpack(colx[2 * CT + 3 * (g0 + Q * g1) + k]);
      }
      FxMetric mt;
      fx_metric(C, scs, mt);
      const double k = kin[e * Q3 + pt];
      if (!(k > 0.0) || !(k < INFINITY)) bad |= LOR_FLAG_BAD_KAPPA;
      if (!(mt.detM > 0.0)) bad |= LOR_FLAG_BAD_GEOM;
      // s = kappa w / det J in FP64, then D_ab = s adj(M)_ab in fixed point
      const double sv = k * (sw[g0] * sw[g1] * sw[g2]) * lor_rsqrt(mt.detM);
      const int es = fx_expo(sv);
      const Fx sx = fx_split(fx_from_double(sv, es));
      const int ss = 1079 - es;
      long long D[6];
      int mx = -(1 << 30);
#pragma unroll
      for (int ab = 0; ab < 6; ++ab) {
        FAcc t = fx_acc();
        fx_mac(t, sx, mt.A[ab]);
        D[ab] = fx_res(t);  // at most 2^59, scale ss + sA - 56
        if (D[ab] != 0) mx = max(mx, fx_bits((unsigned long long)(D[ab] ^ (D[ab] >> 63))) - (ss + mt.sA - kFxMacShift));
      }
      // the point's six entries at its largest: that one at most 2^57 (entry = X 2^-sd)
      const bool any = mx > -(1 << 30);
      const int sd = 57 - mx;
      long long* Dp = reinterpret_cast<long long*>(Dq) + e * 6 * Q3 + pt;
#pragma unroll
      for (int ab = 0; ab < 6; ++ab)
        Dp[ab * Q3] = any ? fx_pack(fx_shift(D[ab], min(sd - (ss + mt.sA - kFxMacShift), 63))) : 0ll;
      sdq[e * Q3 + pt] = any ? sd : INT_MAX;
      kcopy[e * Q3 + pt] = k;
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, bad);
}

// FP32 copy of D for the FP32-arithmetic operator: value = X 2^-sd.
__global__ void __launch_bounds__(256) k_d_to_f32(const double* __restrict__ Dq, int64_t nq, float* __restrict__ out,
                                                  int Q3) {
  const long long* D = reinterpret_cast<const long long*>(Dq);
  const int* sd = lor_d_scales(Dq, nq);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 6 * nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / (6 * Q3), pt = i % Q3;
    const int sc = sd[e * Q3 + pt];
    const Fx f = fx_unpack(D[i]);
    const long long X = (long long)f.h * 268435456ll + f.l;
    out[i] = sc == INT_MAX ? 0.0f : (float)fx_to_double(X, sc);
  }
}

// Reaction term (the definite Helmholtz operator of Section 4.1): at every
// Gauss point M = beta w detJ, the diagonal factor between B_m = B(x)B(x)B
// and its transpose; beta is copied and checked (finite, > 0) like kappa.
template <int P>
__global__ void __launch_bounds__(128) k_reaction_setup(LorMesh m, LorTables T, const double* __restrict__ bin,
                                                        double* __restrict__ bcopy, double* __restrict__ Mq,
                                                        int* __restrict__ status) {
  constexpr int Q = P + 2, Q2 = Q * Q, Q3 = Q * Q * Q;
  __shared__ double Ehalf[36];
  __shared__ double col[3 * Q2 * 3];
  __shared__ double sw[Q], s0[Q], s1[Q];
  if (threadIdx.x < Q) {
    sw[threadIdx.x] = T.gw[threadIdx.x];
    s0[threadIdx.x] = T.gl0[threadIdx.x];
    s1[threadIdx.x] = T.gl1[threadIdx.x];
  }
  __syncthreads();
  int bad = 0;
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    lor_jacobian_columns(m, e, s0, s1, Q, Ehalf, col);
    for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
      const int g0 = pt % Q, g1 = (pt / Q) % Q, g2 = pt / Q2;
      const double* c0 = col + 0 * Q2 * 3 + 3 * (g1 + Q * g2);
      const double* c1 = col + 1 * Q2 * 3 + 3 * (g0 + Q * g2);
      const double* c2 = col + 2 * Q2 * 3 + 3 * (g0 + Q * g1);
      double a0[3];
      lor_cross(c1, c2, a0);
      const double det = c0[0] * a0[0] + c0[1] * a0[1] + c0[2] * a0[2];
      const double b = bin[e * Q3 + pt];
      if (!(b > 0.0) || !(b < INFINITY)) bad |= LOR_FLAG_BAD_KAPPA;
      if (!(det > 0.0)) bad |= LOR_FLAG_BAD_GEOM;
      Mq[e * Q3 + pt] = b * (sw[g0] * sw[g1] * sw[g2]) * det;
      bcopy[e * Q3 + pt] = b;
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, bad);
}

// Jacobian determinant check at the tensor grid t[0..L) of every element.
__global__ void __launch_bounds__(128) k_geometry_check(LorMesh m, LorTables T, int L, int use_sub,
                                                        int* __restrict__ status) {
  __shared__ double Ehalf[36];
  __shared__ double col[3 * (2 * LOR_MAX_P + 2) * (2 * LOR_MAX_P + 2) * 3];
  __shared__ double t0[2 * LOR_MAX_P + 2], t1[2 * LOR_MAX_P + 2];
  if (threadIdx.x < L) {
    t0[threadIdx.x] = use_sub ? T.sub_l0[threadIdx.x] : T.gl0[threadIdx.x];
    t1[threadIdx.x] = use_sub ? T.sub_l1[threadIdx.x] : T.gl1[threadIdx.x];
  }
  __syncthreads();
  int bad = 0;
  const int L2 = L * L;
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    lor_jacobian_columns(m, e, t0, t1, L, Ehalf, col);
    for (int pt = threadIdx.x; pt < L2 * L; pt += blockDim.x) {
      const int g0 = pt % L, g1 = (pt / L) % L, g2 = pt / L2;
      const double* c0 = col + 0 * L2 * 3 + 3 * (g1 + L * g2);
      const double* c1 = col + 1 * L2 * 3 + 3 * (g0 + L * g2);
      const double* c2 = col + 2 * L2 * 3 + 3 * (g0 + L * g1);
      double a0[3];
      lor_cross(c1, c2, a0);
      const double det = c0[0] * a0[0] + c0[1] * a0[1] + c0[2] * a0[2];
      if (!(det > 0.0)) bad = LOR_FLAG_BAD_GEOM;
    }
    __syncthreads();
  }
  if (bad) atomicOr(status, bad);
}

// Load vector: b_e = (B (x) B (x) B)^T (w detJ f) per element, scatter-added
// into the non-essential DOFs (b must be zeroed first).
template <int P>
__global__ void __launch_bounds__(128) k_load_vector(LorMesh m, LorTables T, const double* __restrict__ f,
                                                     double* __restrict__ b) {
  constexpr int Q = P + 2, N = P + 1, Q2 = Q * Q, Q3 = Q * Q * Q;
  __shared__ double Ehalf[36];
  __shared__ double col[3 * Q2 * 3];
  __shared__ double s0[Q], s1[Q], sw[Q], sB[Q * N];
  __shared__ double v[Q3], t1[N * Q2];
  double* t2 = v;  // v is dead once t1 is formed (N N Q <= Q^3)
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) sB[i] = T.B[i];
  if (threadIdx.x < Q) {
    s0[threadIdx.x] = T.gl0[threadIdx.x];
    s1[threadIdx.x] = T.gl1[threadIdx.x];
    sw[threadIdx.x] = T.gw[threadIdx.x];
  }
  __syncthreads();
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    lor_jacobian_columns(m, e, s0, s1, Q, Ehalf, col);
    for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
      const int g0 = pt % Q, g1 = (pt / Q) % Q, g2 = pt / Q2;
      const double* c0 = col + 0 * Q2 * 3 + 3 * (g1 + Q * g2);
      const double* c1 = col + 1 * Q2 * 3 + 3 * (g0 + Q * g2);
      const double* c2 = col + 2 * Q2 * 3 + 3 * (g0 + Q * g1);
      double a0[3];
      lor_cross(c1, c2, a0);
      const double det = c0[0] * a0[0] + c0[1] * a0[1] + c0[2] * a0[2];
      const double fv = f ? f[e * Q3 + pt] : 1.0;
      v[pt] = sw[g0] * sw[g1] * sw[g2] * det * fv;
    }
    __syncthreads();
    // contract g2 -> k:  t1[k][g1][g0]
    for (int idx = threadIdx.x; idx < N * Q2; idx += blockDim.x) {
      const int g0 = idx % Q, g1 = (idx / Q) % Q, k = idx / Q2;
      double s = 0.0;
      for (int g2 = 0; g2 < Q; ++g2) s += sB[g2 * N + k] * v[g0 + Q * (g1 + Q * g2)];
      t1[idx] = s;
    }
    __syncthreads();
    // contract g1 -> j:  t2[k][j][g0]
    for (int idx = threadIdx.x; idx < N * N * Q; idx += blockDim.x) {
      const int g0 = idx % Q, j = (idx / Q) % N, k = idx / (Q * N);
      double s = 0.0;
      for (int g1 = 0; g1 < Q; ++g1) s += sB[g1 * N + j] * t1[g0 + Q * (g1 + Q * k)];
      t2[idx] = s;
    }
    __syncthreads();
    // contract g0 -> i and scatter
    const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
    for (int idx = threadIdx.x; idx < N * N * N; idx += blockDim.x) {
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      double s = 0.0;
      for (int g0 = 0; g0 < Q; ++g0) s += sB[g0 * N + i] * t2[g0 + Q * (j + N * k)];
      if (m.edofs) {
        const int64_t d = m.edofs[e * (int64_t)N * N * N + idx];
        if (!m.ess[d]) atomicAdd(b + d, s);
        continue;
      }
      const int64_t I = ex * P + i, J = ey * P + j, K = ez * P + k;
      if (!lor_is_essential(I, J, K, m.nx, m.ny, m.nz)) atomicAdd(b + I + m.nx * (J + m.ny * K), s);
    }
    __syncthreads();
  }
}

int grid_for(int64_t nel) {
  const int64_t cap = 152 * 64;
  return (int)(nel < cap ? nel : cap);
}

}  // namespace

cudaError_t lor_launch_setup(const LorMesh& m, const LorTables& T, const double* kappa_in, double* kappa_copy,
                             double* Dq, int* d_status, cudaStream_t s) {
  const int g = grid_for(m.nel);
  switch (m.p) {
#define LOR_CASE(P) \
  case P: k_setup<P><<<g, 128, 0, s>>>(m, T, kappa_in, kappa_copy, Dq, d_status); lor_count_launch(); break;
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t lor_launch_d_to_f32(const LorMesh& m, const double* Dq, float* out, cudaStream_t s) {
  const int Q3 = (m.p + 2) * (m.p + 2) * (m.p + 2);
  const int64_t nq = m.nel * (int64_t)Q3;
  const int64_t blocks = (6 * nq + 255) / 256;
  k_d_to_f32<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(Dq, nq, out, Q3);
  lor_count_launch();
  return cudaGetLastError();
}

cudaError_t lor_launch_reaction_setup(const LorMesh& m, const LorTables& T, const double* beta_in, double* beta_copy,
                                      double* Mq, int* d_status, cudaStream_t s) {
  const int g = grid_for(m.nel);
  switch (m.p) {
#define LOR_CASE(P) \
  case P: k_reaction_setup<P><<<g, 128, 0, s>>>(m, T, beta_in, beta_copy, Mq, d_status); lor_count_launch(); break;
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t lor_launch_geometry_check(const LorMesh& m, const LorTables& T, int* d_status, cudaStream_t s) {
  const int g = grid_for(m.nel);
  k_geometry_check<<<g, 128, 0, s>>>(m, T, T.q, 0, d_status); lor_count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_geometry_check<<<g, 128, 0, s>>>(m, T, 2 * T.p, 1, d_status); lor_count_launch();
  return cudaGetLastError();
}

cudaError_t lor_launch_load_vector(const LorMesh& m, const LorTables& T, const double* f, double* b,
                                   cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(b, 0, sizeof(double) * m.ndof, s);
  if (err != cudaSuccess) return err;
  const int g = grid_for(m.nel);
  switch (m.p) {
#define LOR_CASE(P) \
  case P: k_load_vector<P><<<g, 128, 0, s>>>(m, T, f, b); lor_count_launch(); break;
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

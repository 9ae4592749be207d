// k_apply.cu -- Step S2.1: matrix-free high-order diffusion operator
// y = G^T B^T D B G x (Eq. (4) on one rank) by sum factorisation, and its
// backward (gradients with respect to x and to kappa at the Gauss points).
//
// One CTA per element.  G (gather through the structured element-to-DOF map,
// Dirichlet DOFs masked) -> B: three 1D contraction stages giving the
// reference gradient at the q^3 Gauss points with
//   B = [B(x)B(x)d ; B(x)d(x)B ; d(x)B(x)B]
// -> D: the symmetric 3x3 factor stored by the setup -> B^T: the three stages
// in reverse -> G^T: FP64 atomics into y.  All arithmetic is FP64.
#include "lor_internal.cuh"

namespace {

constexpr int kApplyThreads = 128;

template <int P>
struct Dims {
  static constexpr int Q = P + 2, N = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, N2 = N * N, N3 = N2 * N;
  // shared-memory plan (doubles): tables | A: max(N^3, 2 N^2 Q) | Bf: 3 N Q^2 | V: 3 Q^3 | V2: 3 Q^3 (backward)
  static constexpr int tab = 2 * Q * N;
  static constexpr int A = (N3 > 2 * N2 * Q ? N3 : 2 * N2 * Q);
  static constexpr int Bf = 3 * N * Q2;
  static constexpr int V = 3 * Q3;
  static constexpr int apply_doubles = tab + A + Bf + V;
  static constexpr int backward_doubles = tab + A + Bf + 2 * V;
};

template <int P>
__device__ __forceinline__ void load_tables(const LorTables& T, double* sB, double* sD) {
  constexpr int Q = P + 2, N = P + 1;
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) {
    sB[i] = T.B[i];
    sD[i] = T.Dm[i];
  }
}

// u[k][j][i] <- x at the element's DOFs, 0 on essential DOFs.
template <int P>
__device__ __forceinline__ void gather(const LorMesh& m, int64_t e, const double* __restrict__ x, double* u) {
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
  for (int idx = threadIdx.x; idx < N3; idx += blockDim.x) {
    const int i = idx % N, j = (idx / N) % N, k = idx / N2;
    const int64_t I = ex * P + i, J = ey * P + j, K = ez * P + k;
    u[idx] = lor_is_essential(I, J, K, m.nx, m.ny, m.nz) ? 0.0 : x[I + m.nx * (J + m.ny * K)];
  }
}

// Reference gradient at the Gauss points: g[c][pt], pt = g0 + Q (g1 + Q g2).
// u is read (and the A, Bf buffers are overwritten).  Ends synchronised.
template <int P>
__device__ void forward_gradient(const double* sB, const double* sD, const double* u, double* A, double* Bf,
                                 double* g) {
  constexpr int Q = P + 2, N = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, N2 = N * N;
  double* Bu = A;            // [k][j][g0]
  double* Du = A + N2 * Q;   // [k][j][g0]
  // stage x: contract i
  for (int idx = threadIdx.x; idx < N2 * Q; idx += blockDim.x) {
    const int g0 = idx % Q, jk = idx / Q;
    const double* ur = u + jk * N;
    double sb = 0.0, sd = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      sb += sB[g0 * N + i] * ur[i];
      sd += sD[g0 * N + i] * ur[i];
    }
    Bu[idx] = sb;
    Du[idx] = sd;
  }
  __syncthreads();
  // stage y: contract j -> BB, BD (B in y, d in x), DB (d in y, B in x); [k][g1][g0]
  double* BB = Bf;
  double* BD = Bf + N * Q2;
  double* DB = Bf + 2 * N * Q2;
  for (int idx = threadIdx.x; idx < N * Q2; idx += blockDim.x) {
    const int g0 = idx % Q, g1 = (idx / Q) % Q, k = idx / Q2;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const double b = sB[g1 * N + j], d = sD[g1 * N + j];
      const double bu = Bu[g0 + Q * (j + N * k)], du = Du[g0 + Q * (j + N * k)];
      s0 += b * bu;
      s1 += b * du;
      s2 += d * bu;
    }
    BB[idx] = s0;
    BD[idx] = s1;
    DB[idx] = s2;
  }
  __syncthreads();
  // stage z: contract k -> d/dxi0 = B_z BD, d/dxi1 = B_z DB, d/dxi2 = d_z BB
  for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
    const int g01 = pt % Q2, g2 = pt / Q2;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double b = sB[g2 * N + k], d = sD[g2 * N + k];
      s0 += b * BD[g01 + Q2 * k];
      s1 += b * DB[g01 + Q2 * k];
      s2 += d * BB[g01 + Q2 * k];
    }
    g[pt] = s0;
    g[Q3 + pt] = s1;
    g[2 * Q3 + pt] = s2;
  }
  __syncthreads();
}

// v[c][pt] <- D_pt v (symmetric 3x3, stored (00,01,02,11,12,22)), in place.
template <int P>
__device__ __forceinline__ void apply_D(const double* __restrict__ De, double* v) {
  constexpr int Q3 = (P + 2) * (P + 2) * (P + 2);
  for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
    const double a = v[pt], b = v[Q3 + pt], c = v[2 * Q3 + pt];
    const double d00 = De[pt], d01 = De[Q3 + pt], d02 = De[2 * Q3 + pt];
    const double d11 = De[3 * Q3 + pt], d12 = De[4 * Q3 + pt], d22 = De[5 * Q3 + pt];
    v[pt] = d00 * a + d01 * b + d02 * c;
    v[Q3 + pt] = d01 * a + d11 * b + d12 * c;
    v[2 * Q3 + pt] = d02 * a + d12 * b + d22 * c;
  }
  __syncthreads();
}

// y_e = B^T v and scatter-add into the non-essential DOFs of y.
template <int P>
__device__ void backward_scatter(const LorMesh& m, int64_t e, const double* sB, const double* sD, const double* v,
                                 double* A, double* Bf, double* __restrict__ y) {
  constexpr int Q = P + 2, N = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, N2 = N * N, N3 = N2 * N;
  double* T0 = Bf;             // [k][g1][g0]
  double* T1 = Bf + N * Q2;
  double* T2 = Bf + 2 * N * Q2;
  for (int idx = threadIdx.x; idx < N * Q2; idx += blockDim.x) {
    const int g01 = idx % Q2, k = idx / Q2;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int g2 = 0; g2 < Q; ++g2) {
      const double b = sB[g2 * N + k], d = sD[g2 * N + k];
      s0 += b * v[g01 + Q2 * g2];
      s1 += b * v[Q3 + g01 + Q2 * g2];
      s2 += d * v[2 * Q3 + g01 + Q2 * g2];
    }
    T0[idx] = s0;
    T1[idx] = s1;
    T2[idx] = s2;
  }
  __syncthreads();
  double* U0 = A;              // [k][j][g0]: d still to apply in x
  double* U1 = A + N2 * Q;     // B still to apply in x
  for (int idx = threadIdx.x; idx < N2 * Q; idx += blockDim.x) {
    const int g0 = idx % Q, j = (idx / Q) % N, k = idx / (Q * N);
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int g1 = 0; g1 < Q; ++g1) {
      const double b = sB[g1 * N + j], d = sD[g1 * N + j];
      const int t = g0 + Q * (g1 + Q * k);
      s0 += b * T0[t];
      s1 += d * T1[t] + b * T2[t];
    }
    U0[idx] = s0;
    U1[idx] = s1;
  }
  __syncthreads();
  const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
  for (int idx = threadIdx.x; idx < N3; idx += blockDim.x) {
    const int i = idx % N, jk = idx / N;
    double s = 0.0;
#pragma unroll
    for (int g0 = 0; g0 < Q; ++g0) s += sD[g0 * N + i] * U0[g0 + Q * jk] + sB[g0 * N + i] * U1[g0 + Q * jk];
    const int j = jk % N, k = jk / N;
    const int64_t I = ex * P + i, J = ey * P + j, K = ez * P + k;
    if (!lor_is_essential(I, J, K, m.nx, m.ny, m.nz)) atomicAdd(y + I + m.nx * (J + m.ny * K), s);
  }
  __syncthreads();
}

template <int P>
__global__ void __launch_bounds__(kApplyThreads) k_apply(LorMesh m, LorTables T, const double* __restrict__ Dq,
                                                         const double* __restrict__ x, double* __restrict__ y) {
  using Dm = Dims<P>;
  extern __shared__ double smem[];
  double* sB = smem;
  double* sD = smem + Dm::Q * Dm::N;
  double* A = smem + Dm::tab;
  double* Bf = A + Dm::A;
  double* V = Bf + Dm::Bf;
  load_tables<P>(T, sB, sD);
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    gather<P>(m, e, x, V);  // u is read by stage x before stage z writes the gradient over it
    __syncthreads();
    forward_gradient<P>(sB, sD, V, A, Bf, V);
    apply_D<P>(Dq + e * 6 * Dm::Q3, V);
    backward_scatter<P>(m, e, sB, sD, V, A, Bf, y);
  }
}

template <int P>
__global__ void __launch_bounds__(kApplyThreads) k_apply_backward(LorMesh m, LorTables T,
                                                                  const double* __restrict__ Dq,
                                                                  const double* __restrict__ kappa,
                                                                  const double* __restrict__ x,
                                                                  const double* __restrict__ gy,
                                                                  double* __restrict__ gx,
                                                                  double* __restrict__ gkappa) {
  using Dm = Dims<P>;
  constexpr int Q3 = Dm::Q3;
  extern __shared__ double smem[];
  double* sB = smem;
  double* sD = smem + Dm::Q * Dm::N;
  double* A = smem + Dm::tab;
  double* Bf = A + Dm::A;
  double* V = Bf + Dm::Bf;   // gradient of gy, then D grad(gy)
  double* V2 = V + Dm::V;    // gradient of x
  load_tables<P>(T, sB, sD);
  for (int64_t e = blockIdx.x; e < m.nel; e += gridDim.x) {
    const double* De = Dq + e * 6 * Q3;
    gather<P>(m, e, gy, V);
    __syncthreads();
    forward_gradient<P>(sB, sD, V, A, Bf, V);
    if (gkappa) {
      gather<P>(m, e, x, V2);
      __syncthreads();
      forward_gradient<P>(sB, sD, V2, A, Bf, V2);
      // gkappa = grad(x)^T (D / kappa) grad(gy)
      for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
        const double a = V[pt], b = V[Q3 + pt], c = V[2 * Q3 + pt];
        const double d00 = De[pt], d01 = De[Q3 + pt], d02 = De[2 * Q3 + pt];
        const double d11 = De[3 * Q3 + pt], d12 = De[4 * Q3 + pt], d22 = De[5 * Q3 + pt];
        const double t0 = d00 * a + d01 * b + d02 * c;
        const double t1 = d01 * a + d11 * b + d12 * c;
        const double t2 = d02 * a + d12 * b + d22 * c;
        gkappa[e * Q3 + pt] = (V2[pt] * t0 + V2[Q3 + pt] * t1 + V2[2 * Q3 + pt] * t2) / kappa[e * Q3 + pt];
      }
      __syncthreads();
    }
    if (gx) {
      apply_D<P>(De, V);
      backward_scatter<P>(m, e, sB, sD, V, A, Bf, gx);
    }
  }
}

// y <- x on essential DOFs, 0 elsewhere (the apply then adds the free rows).
__global__ void k_init_output(LorMesh m, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m.ndof; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = r % m.nx, J = (r / m.nx) % m.ny, K = r / (m.nx * m.ny);
    y[r] = lor_is_essential(I, J, K, m.nx, m.ny, m.nz) ? x[r] : 0.0;
  }
}

cudaError_t init_output(const LorMesh& m, const double* x, double* y, cudaStream_t s) {
  const int64_t blocks = (m.ndof + 255) / 256;
  k_init_output<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(m, x, y); lor_count_launch();
  return cudaGetLastError();
}

template <int P>
cudaError_t apply_p(const LorMesh& m, const LorTables& T, const double* Dq, const double* x, double* y,
                    cudaStream_t s) {
  const size_t bytes = sizeof(double) * Dims<P>::apply_doubles;
  static unsigned configured = 0;  // per-device bit: the attribute is set once per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(configured & (1u << dev))) {
    cudaError_t err = cudaFuncSetAttribute(k_apply<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
    configured |= 1u << dev;
  }
  k_apply<P><<<(unsigned)m.nel, kApplyThreads, bytes, s>>>(m, T, Dq, x, y); lor_count_launch();
  return cudaGetLastError();
}

template <int P>
cudaError_t backward_p(const LorMesh& m, const LorTables& T, const double* Dq, const double* kappa, const double* x,
                       const double* gy, double* gx, double* gk, cudaStream_t s) {
  const size_t bytes = sizeof(double) * Dims<P>::backward_doubles;
  static unsigned configured = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(configured & (1u << dev))) {
    cudaError_t err =
        cudaFuncSetAttribute(k_apply_backward<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
    configured |= 1u << dev;
  }
  k_apply_backward<P><<<(unsigned)m.nel, kApplyThreads, bytes, s>>>(m, T, Dq, kappa, x, gy, gx, gk); lor_count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t lor_launch_apply(const LorMesh& m, const LorTables& T, const double* Dq, const double* x, double* y,
                             cudaStream_t s) {
  cudaError_t err = init_output(m, x, y, s);
  if (err != cudaSuccess) return err;
  switch (m.p) {
#define LOR_CASE(P) \
  case P: return apply_p<P>(m, T, Dq, x, y, s);
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t lor_launch_apply_backward(const LorMesh& m, const LorTables& T, const double* Dq, const double* kappa,
                                      const double* x, const double* gy, double* gx, double* gkappa,
                                      cudaStream_t s) {
  if (gx) {
    cudaError_t err = init_output(m, gy, gx, s);
    if (err != cudaSuccess) return err;
  }
  if (!gx && !gkappa) return cudaSuccess;
  switch (m.p) {
#define LOR_CASE(P) \
  case P: return backward_p<P>(m, T, Dq, kappa, x, gy, gx, gkappa, s);
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
}

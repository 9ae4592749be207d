// k_apply_impl.cuh -- kernels and launch templates of the high-order apply
// and its backward, instantiated without the reaction term in k_apply.cu,
// with it in k_apply_mass.cu, on general meshes in k_apply_general.cu, and
// the apply with FP32 arithmetic in k_apply_f32*.cu (the translation units
// compile in parallel).
//
// y = G^T B^T D B G x (Eq. (4) on one rank) by sum factorisation, and its
// backward (gradients with respect to x and to kappa at the Gauss points).
//
//   B = [B(x)B(x)d ; B(x)d(x)B ; d(x)B(x)B]  (Step S2.1, 3D diffusion)
//
// with the 1D interpolation matrix B_1D and derivative matrix d_1D (q x n,
// n = p+1 GLL nodes, q = p+2 Gauss points), D the symmetric 3x3 factor stored
// by the setup (Step S1.1), G the gather through the structured element map
// (Dirichlet DOFs masked) and G^T FP64 atomics into y.  The arithmetic type R
// is FP64 for the operator of Step S2.1 and its backward; R = float gives
// the FP32 operator that the mixed-precision refinement iterates with (its
// own table and shared-memory layout, Lay<P, float>).
//
// GB300 design (FP64 issue is the bound: 2 DFMA/clk/SM):
//  * even-odd folding: GLL nodes and Gauss points are symmetric about 0, so
//    B_1D[q-1-g][n-1-i] = B_1D[g][i] and d_1D[q-1-g][n-1-i] = -d_1D[g][i];
//    each 1D contraction works on the half-size symmetric/antisymmetric
//    parts (u_i +- u_{n-1-i}), about 25-35% fewer FP64 operations;
//  * one thread per 1D line of a stage, E elements per CTA so that the lines
//    of a stage fill whole warps (idle lanes would waste FP64 issue slots);
//  * the z stage, the D product and the transposed z stage run in registers
//    on the same line (no shared-memory round trip for the q^3 values).
//
// With a reaction term (the definite Helmholtz operator of Section 4.1) the
// mass part B_m^T (beta w detJ) B_m, B_m = B(x)B(x)B, shares every stage with
// the diffusion part: B_m x is B_z applied to the BB line the z stage already
// folds, and B_z^T of the scaled values joins d_z^T on the same output slot.
#pragma once

#include "lor_internal.cuh"

namespace {

template <int P>
struct Sz {
  static constexpr int N = P + 1, Q = P + 2, NH = N / 2, QH = Q / 2;
  static constexpr bool NODD = (N & 1) != 0, QODD = (Q & 1) != 0;
  static constexpr int NM = N / 2, QM = Q / 2;  // middle index when odd
  static constexpr int A1 = 2 * N * N * Q;      // [c][k][j][g0], c in {B, d} of the x stage
  static constexpr int A2 = 3 * N * Q * Q;      // [c][k][g1][g0]
  static constexpr int PER_ELEM = A1 + A2;
  // elements per CTA and CTA size: the z stage (the heaviest) gets about one
  // line per thread, and high-degree CTAs stay small so that several share an
  // SM (the FP64 pipe then stays busy while one CTA waits at a barrier)
  static constexpr int E = P == 1 ? 28 : P == 2 ? 16 : P == 3 ? 10 : P == 4 ? 7 : P == 5 ? 5 : P == 6 ? 4
                         : P == 7 ? 3 : P == 8 ? 3 : P == 9 ? 2 : 2;
  static constexpr int T = ((E * Q * Q + 31) / 32) * 32;
  // the backward holds two fields per element (twice the shared memory; at
  // p = 10 two elements would exceed the 227 KB a CTA may use)
  static constexpr int EB = P == 6 ? 2 : P == 10 ? 1 : E;
  static constexpr int TBW = ((EB * Q * Q + 31) / 32) * 32;
  // folded tables in shared memory (doubles)
  static constexpr int TB = Q * N;                  // B_1D, d_1D
  static constexpr int TF = Q * (NH > 0 ? NH : 1);  // BE, BO, DE, DO: [g][i], g < Q, i < NH
  static constexpr int TABLES = 2 * TB + 4 * TF;
};

// Shared-memory layout per arithmetic type.  FP64 keeps the layout of Sz.
// FP32 (where shared-memory traffic, not the FP32 pipe, is the limit):
//  * the x-stage lines of A1 get an odd stride (Q+1 when Q is even), so the
//    lines that consecutive threads write and read start in different banks;
//  * the folded tables are stored with rows padded to a multiple of 4
//    entries (16 bytes), g-major for the forward contractions and i-major
//    (transposed) for B^T / d^T, plus the middle column (B[g][n/2], used when
//    n is odd) and the middle row (B[q/2][i], when q is odd) as padded rows,
//    so one 16-byte broadcast load feeds up to four multiply-adds.
// smallest value >= base that is congruent to r mod 32
constexpr int pad_to_residue(int base, int r) { return base + (((r - base) % 32) + 32) % 32; }

template <int P, typename R>
struct Lay {
  using Z = Sz<P>;
  static constexpr bool F32 = sizeof(R) == sizeof(float);
  static constexpr int LS = (F32 && Z::Q % 2 == 0) ? Z::Q + 1 : Z::Q;  // line stride of A1
  // k strides of A1 and A2: in FP32 congruent to q mod 32, so the (k, g0)
  // lines that consecutive threads of the y stages touch map to distinct banks
  static constexpr int KS1 = F32 ? pad_to_residue(Z::N * LS, Z::Q) : Z::N * LS;
  static constexpr int KS2 = F32 ? pad_to_residue(Z::Q * Z::Q, Z::Q) : Z::Q * Z::Q;
  static constexpr int C1 = Z::N * KS1, C2 = Z::N * KS2;  // component strides
  static constexpr int A1 = 2 * C1;                       // [c][k][j][g0]
  static constexpr int A2 = 3 * C2;                       // [c][k][g1][g0]
  static constexpr int PER_ELEM = A1 + A2;
  static constexpr int NH4 = ((Z::NH + 3) / 4) * 4, QH4 = ((Z::QH + 3) / 4) * 4, Q4 = ((Z::Q + 3) / 4) * 4;
  static constexpr int TFF = Z::Q * NH4;  // BE, BO, DE, DO: [g][i], g < q
  static constexpr int TFT = NH4 * QH4;   // BEt, BOt, DEt, DOt: [i][g], g < q/2
  static constexpr int TABLES = F32 ? 4 * TFF + 4 * TFT + 2 * Q4 + 2 * NH4 : Z::TABLES;
  // elements per CTA and CTA size of the apply: FP32 takes half the FP64
  // count up to p = 8 (smaller CTAs, the same warps per SM, shorter
  // barriers: 8-10% faster at p = 6..8, neutral below); at p = 9, 10 one
  // element per CTA leaves too few warps, so the FP64 count stays
  static constexpr int E = F32 && P <= 8 ? (Z::E + 1) / 2 : Z::E;
  static constexpr int T = ((E * Z::Q * Z::Q + 31) / 32) * 32;
};

// Folded tables: BE = (B[g][i] + B[g][n-1-i]) / 2, BO = (B[g][i] - B[g][n-1-i]) / 2
// (same for d), for i < n/2.  FP32 also: the transposes BEt[i][g] = BE[g][i]
// etc., BM[g] = B[g][n/2], DM[g] = d[g][n/2], BQ[i] = B[q/2][i], DQ[i] = d[q/2][i].
template <int P, typename R>
struct Tab {
  const R *B, *D, *BE, *BO, *DE, *DO;
  const R *BEt, *BOt, *DEt, *DOt, *BM, *DM, *BQ, *DQ;
};

template <int P, typename R>
__device__ __forceinline__ Tab<P, R> load_tables(const LorTables& T, R* s) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  Tab<P, R> t;
  if constexpr (L::F32) {
    R* BE = s;
    R* BO = BE + L::TFF;
    R* DE = BO + L::TFF;
    R* DO = DE + L::TFF;
    R* BEt = DO + L::TFF;
    R* BOt = BEt + L::TFT;
    R* DEt = BOt + L::TFT;
    R* DOt = DEt + L::TFT;
    R* BM = DOt + L::TFT;
    R* DM = BM + L::Q4;
    R* BQ = DM + L::Q4;
    R* DQ = BQ + L::NH4;
    for (int x = threadIdx.x; x < Z::Q * L::NH4; x += blockDim.x) {
      const int g = x / L::NH4, i = x % L::NH4;
      double be = 0.0, bo = 0.0, de = 0.0, dd = 0.0;
      if (i < Z::NH) {
        const double b0 = T.B[g * Z::N + i], b1 = T.B[g * Z::N + Z::N - 1 - i];
        const double d0 = T.Dm[g * Z::N + i], d1 = T.Dm[g * Z::N + Z::N - 1 - i];
        be = 0.5 * (b0 + b1);
        bo = 0.5 * (b0 - b1);
        de = 0.5 * (d0 + d1);
        dd = 0.5 * (d0 - d1);
      }
      BE[x] = (R)be;
      BO[x] = (R)bo;
      DE[x] = (R)de;
      DO[x] = (R)dd;
      if (g < L::QH4 && i < L::NH4) {  // transposed copy (rows g < q/2 only)
        const bool in = g < Z::QH && i < Z::NH;
        BEt[i * L::QH4 + g] = in ? (R)be : (R)0;
        BOt[i * L::QH4 + g] = in ? (R)bo : (R)0;
        DEt[i * L::QH4 + g] = in ? (R)de : (R)0;
        DOt[i * L::QH4 + g] = in ? (R)dd : (R)0;
      }
    }
    // the transposed rows' padding columns g in [q, QH4) are not covered above when QH4 > q
    for (int x = threadIdx.x; x < L::NH4 * L::QH4; x += blockDim.x) {
      const int i = x / L::QH4, g = x % L::QH4;
      if (g >= Z::Q) {
        BEt[x] = (R)0;
        BOt[x] = (R)0;
        DEt[x] = (R)0;
        DOt[x] = (R)0;
      }
    }
    for (int x = threadIdx.x; x < L::Q4; x += blockDim.x) {
      BM[x] = x < Z::Q && Z::NODD ? (R)T.B[x * Z::N + Z::NM] : (R)0;
      DM[x] = x < Z::Q && Z::NODD ? (R)T.Dm[x * Z::N + Z::NM] : (R)0;
    }
    for (int x = threadIdx.x; x < L::NH4; x += blockDim.x) {
      BQ[x] = x < Z::NH && Z::QODD ? (R)T.B[Z::QM * Z::N + x] : (R)0;
      DQ[x] = x < Z::NH && Z::QODD ? (R)T.Dm[Z::QM * Z::N + x] : (R)0;
    }
    t.B = t.D = nullptr;
    t.BE = BE;
    t.BO = BO;
    t.DE = DE;
    t.DO = DO;
    t.BEt = BEt;
    t.BOt = BOt;
    t.DEt = DEt;
    t.DOt = DOt;
    t.BM = BM;
    t.DM = DM;
    t.BQ = BQ;
    t.DQ = DQ;
    return t;
  }
  R* B = s;
  R* D = s + Z::TB;
  R* BE = s + 2 * Z::TB;
  R* BO = BE + Z::TF;
  R* DE = BO + Z::TF;
  R* DO = DE + Z::TF;
  for (int x = threadIdx.x; x < Z::TB; x += blockDim.x) {
    B[x] = (R)T.B[x];
    D[x] = (R)T.Dm[x];
  }
  for (int x = threadIdx.x; x < Z::Q * Z::NH; x += blockDim.x) {
    const int g = x / Z::NH, i = x % Z::NH;
    const double b0 = T.B[g * Z::N + i], b1 = T.B[g * Z::N + Z::N - 1 - i];
    const double d0 = T.Dm[g * Z::N + i], d1 = T.Dm[g * Z::N + Z::N - 1 - i];
    BE[g * Z::NH + i] = (R)(0.5 * (b0 + b1));
    BO[g * Z::NH + i] = (R)(0.5 * (b0 - b1));
    DE[g * Z::NH + i] = (R)(0.5 * (d0 + d1));
    DO[g * Z::NH + i] = (R)(0.5 * (d0 - d1));
  }
  t.B = B;
  t.D = D;
  t.BE = BE;
  t.BO = BO;
  t.DE = DE;
  t.DO = DO;
  t.BEt = t.BOt = t.DEt = t.DOt = t.BM = t.DM = t.BQ = t.DQ = nullptr;
  return t;
}

// FP64 <-> FP32 conversion of the apply's input and output by integer
// operations: the conversion instructions issue on the FP64 pipe (1/64 of
// the FP32 rate on this GPU) and would otherwise take a fifth of it.
// to_r<float>: round to nearest (ties away from zero) of the 53-bit
// significand to 24 bits; |v| < 2^-126 gives a signed zero, |v| >= 2^128
// infinity.  to_f64(float): exact for zero and normal floats (subnormals
// give zero).
template <typename R>
__device__ __forceinline__ R to_r(double v) {
  if constexpr (sizeof(R) == sizeof(double)) {
    return v;
  } else {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7ffu;
    unsigned mag = ((((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
    mag = e <= 896u ? 0u : (e >= 1151u ? 0x7f800000u : mag);
    return __uint_as_float((hi & 0x80000000u) | mag);
  }
}
template <typename R>
__device__ __forceinline__ R to_r(float v) {
  return (R)v;
}
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) {
  const unsigned f = __float_as_uint(v);
  const unsigned sign = f & 0x80000000u;
  const bool zero = ((f >> 23) & 0xffu) == 0u;
  const unsigned hi = zero ? sign : (sign | (((f & 0x7fffffffu) >> 3) + (896u << 20)));
  return __hiloint2double((int)hi, zero ? 0 : (int)(f << 29));
}

// A result of the compute type R into the output vector type XV.
template <typename XV, typename R>
__device__ __forceinline__ XV to_out(R v) {
  if constexpr (sizeof(XV) == sizeof(double)) return to_f64(v);
  else return (XV)v;
}

// CNT consecutive FP32 table entries from a 16-byte aligned, padded row
// (16-byte loads; the padding lanes are dropped).
template <int CNT>
__device__ __forceinline__ void ld_row(const float* p, float* out) {
#pragma unroll
  for (int i = 0; i < CNT; i += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + i);
    out[i] = v.x;
    if (i + 1 < CNT) out[i + 1] = v.y;
    if (i + 2 < CNT) out[i + 2] = v.z;
    if (i + 3 < CNT) out[i + 3] = v.w;
  }
}

// Table entry k of a 1D table in shared memory, read as volatile: the
// compiler then re-reads the entry at each use instead of holding the
// loop-invariant tables in registers across the line loops (which, with the
// tables of degree 6 and up, needs more than 255 registers and spills; below
// that it only costs occupancy).  A shared-memory read is far cheaper than
// the FP64 multiply-add it feeds.
//
// In FP32 the tables are small enough to live in registers and the FP32
// pipe is 64 times faster than the FP64 one, so there the entries are plain
// loads the compiler may hoist (a shared-memory read per multiply-add would
// bound the kernel).
template <int P, typename R>
__device__ __forceinline__ R tabv(const R* tbl, int k) {
  if constexpr (sizeof(R) == sizeof(double)) return static_cast<const volatile R*>(tbl)[k];
  else return tbl[k];
}

// y = B_1D u, from the folded input e_i = u_i + u_{n-1-i}, o_i = u_i - u_{n-1-i}, um = u_mid
template <int P, typename R>
__device__ __forceinline__ void fwd_B(const Tab<P, R>& t, const R* e, const R* o, R um, R* y) {
  using Z = Sz<P>;
  if constexpr (Lay<P, R>::F32) {
    using L = Lay<P, R>;
    float bm[Z::QH], be[Z::NH], bo[Z::NH];
    if (Z::NODD) ld_row<Z::QH>(t.BM, bm);
#pragma unroll
    for (int g = 0; g < Z::QH; ++g) {
      ld_row<Z::NH>(t.BE + g * L::NH4, be);
      ld_row<Z::NH>(t.BO + g * L::NH4, bo);
      float ev = Z::NODD ? bm[g] * um : 0.0f, od = 0.0f;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) {
        ev += be[i] * e[i];
        od += bo[i] * o[i];
      }
      y[g] = ev + od;
      y[Z::Q - 1 - g] = ev - od;
    }
    if (Z::QODD) {
      ld_row<Z::NH>(t.BE + Z::QM * L::NH4, be);
      float ev = 0.0f;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) ev += be[i] * e[i];
      y[Z::QM] = ev;
    }
  } else {
#pragma unroll
    for (int g = 0; g < Z::QH; ++g) {
      R ev = Z::NODD ? tabv<P, R>(t.B, g * Z::N + Z::NM) * um : (R)0, od = 0;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) {
        ev += tabv<P, R>(t.BE, g * Z::NH + i) * e[i];
        od += tabv<P, R>(t.BO, g * Z::NH + i) * o[i];
      }
      y[g] = ev + od;
      y[Z::Q - 1 - g] = ev - od;
    }
    if (Z::QODD) {
      R ev = 0.0;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) ev += tabv<P, R>(t.BE, Z::QM * Z::NH + i) * e[i];
      y[Z::QM] = ev;
    }
  }
}
// y = d_1D u
template <int P, typename R>
__device__ __forceinline__ void fwd_D(const Tab<P, R>& t, const R* e, const R* o, R um, R* y) {
  using Z = Sz<P>;
  if constexpr (Lay<P, R>::F32) {
    using L = Lay<P, R>;
    float dm[Z::QH], de[Z::NH], dd[Z::NH];
    if (Z::NODD) ld_row<Z::QH>(t.DM, dm);
#pragma unroll
    for (int g = 0; g < Z::QH; ++g) {
      ld_row<Z::NH>(t.DE + g * L::NH4, de);
      ld_row<Z::NH>(t.DO + g * L::NH4, dd);
      float sv = Z::NODD ? dm[g] * um : 0.0f, dv = 0.0f;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) {
        sv += de[i] * e[i];
        dv += dd[i] * o[i];
      }
      y[g] = dv + sv;
      y[Z::Q - 1 - g] = dv - sv;
    }
    if (Z::QODD) {
      ld_row<Z::NH>(t.DO + Z::QM * L::NH4, dd);
      float dv = 0.0f;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) dv += dd[i] * o[i];
      y[Z::QM] = dv;
    }
  } else {
#pragma unroll
    for (int g = 0; g < Z::QH; ++g) {
      R s = Z::NODD ? tabv<P, R>(t.D, g * Z::N + Z::NM) * um : (R)0, d = 0;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) {
        s += tabv<P, R>(t.DE, g * Z::NH + i) * e[i];
        d += tabv<P, R>(t.DO, g * Z::NH + i) * o[i];
      }
      y[g] = d + s;
      y[Z::Q - 1 - g] = d - s;
    }
    if (Z::QODD) {
      R d = 0.0;
#pragma unroll
      for (int i = 0; i < Z::NH; ++i) d += tabv<P, R>(t.DO, Z::QM * Z::NH + i) * o[i];
      y[Z::QM] = d;
    }
  }
}
template <int P, typename R>
__device__ __forceinline__ void fold_n(const R* u, R* e, R* o, R& um) {
  using Z = Sz<P>;
#pragma unroll
  for (int i = 0; i < Z::NH; ++i) {
    e[i] = u[i] + u[Z::N - 1 - i];
    o[i] = u[i] - u[Z::N - 1 - i];
  }
  um = Z::NODD ? u[Z::NM] : (R)0;
}
template <int P, typename R>
__device__ __forceinline__ void fold_q(const R* v, R* e, R* o, R& vm) {
  using Z = Sz<P>;
#pragma unroll
  for (int g = 0; g < Z::QH; ++g) {
    e[g] = v[g] + v[Z::Q - 1 - g];
    o[g] = v[g] - v[Z::Q - 1 - g];
  }
  vm = Z::QODD ? v[Z::QM] : (R)0;
}
// y = B_1D^T v1 + d_1D^T v2 (either part may be switched off); v1, v2 folded
// as (e, o, middle) over the q Gauss points.
template <int P, bool USE_B, bool USE_D, typename R>
__device__ __forceinline__ void bwd(const Tab<P, R>& t, const R* e1, const R* o1, R m1,
                                    const R* e2, const R* o2, R m2, R* y) {
  using Z = Sz<P>;
  // B^T part: Ev_i = sum_g BE[g][i] e1_g (+ B[qm][i] m1), Od_i = sum_g BO[g][i] o1_g
  // d^T part: S_i = sum_g DO[g][i] e2_g (+ d[qm][i] m2),  T_i = sum_g DE[g][i] o2_g
  // y_i = (Ev + T) + (Od + S), y_{n-1-i} = (Ev + T) - (Od + S)
  if constexpr (Lay<P, R>::F32) {
    using L = Lay<P, R>;
    float bq[Z::NH], dq[Z::NH], c1[Z::QH], c2[Z::QH];
    if (Z::QODD) {
      if (USE_B) ld_row<Z::NH>(t.BQ, bq);
      if (USE_D) ld_row<Z::NH>(t.DQ, dq);
    }
#pragma unroll
    for (int i = 0; i < Z::NH; ++i) {
      float a1 = 0.0f, a2 = 0.0f;
      if (Z::QODD) {
        if (USE_B) a1 += bq[i] * m1;
        if (USE_D) a2 += dq[i] * m2;
      }
      if (USE_B) {
        ld_row<Z::QH>(t.BEt + i * L::QH4, c1);
        ld_row<Z::QH>(t.BOt + i * L::QH4, c2);
#pragma unroll
        for (int g = 0; g < Z::QH; ++g) {
          a1 += c1[g] * e1[g];
          a2 += c2[g] * o1[g];
        }
      }
      if (USE_D) {
        ld_row<Z::QH>(t.DEt + i * L::QH4, c1);
        ld_row<Z::QH>(t.DOt + i * L::QH4, c2);
#pragma unroll
        for (int g = 0; g < Z::QH; ++g) {
          a1 += c1[g] * o2[g];
          a2 += c2[g] * e2[g];
        }
      }
      y[i] = a1 + a2;
      y[Z::N - 1 - i] = a1 - a2;
    }
    if (Z::NODD) {
      float sv = 0.0f;
      if (USE_B) {
        ld_row<Z::QH>(t.BM, c1);
#pragma unroll
        for (int g = 0; g < Z::QH; ++g) sv += c1[g] * e1[g];
      }
      if (USE_D) {
        ld_row<Z::QH>(t.DM, c2);
#pragma unroll
        for (int g = 0; g < Z::QH; ++g) sv += c2[g] * o2[g];
      }
      y[Z::NM] = sv;
    }
  } else {
#pragma unroll
    for (int i = 0; i < Z::NH; ++i) {
      R a1 = 0.0, a2 = 0.0;
      if (Z::QODD) {
        if (USE_B) a1 += tabv<P, R>(t.B, Z::QM * Z::N + i) * m1;
        if (USE_D) a2 += tabv<P, R>(t.D, Z::QM * Z::N + i) * m2;
      }
#pragma unroll
      for (int g = 0; g < Z::QH; ++g) {
        if (USE_B) {
          a1 += tabv<P, R>(t.BE, g * Z::NH + i) * e1[g];
          a2 += tabv<P, R>(t.BO, g * Z::NH + i) * o1[g];
        }
        if (USE_D) {
          a1 += tabv<P, R>(t.DE, g * Z::NH + i) * o2[g];
          a2 += tabv<P, R>(t.DO, g * Z::NH + i) * e2[g];
        }
      }
      y[i] = a1 + a2;
      y[Z::N - 1 - i] = a1 - a2;
    }
    if (Z::NODD) {
      R s = 0.0;
#pragma unroll
      for (int g = 0; g < Z::QH; ++g) {
        if (USE_B) s += tabv<P, R>(t.B, g * Z::N + Z::NM) * e1[g];
        if (USE_D) s += tabv<P, R>(t.D, g * Z::N + Z::NM) * o2[g];
      }
      y[Z::NM] = s;
    }
  }
}

// ---- stages over all lines of E elements (e_first .. e_first+E-1) ----
// X: u (gathered from global, masked) -> A1[c][k][j][g0] = (B u, d u) along x.
// GEN: through the general element-to-DOF map and essential mask.
template <int P, bool GEN, typename R, typename XV>
__device__ __forceinline__ void stage_x(const LorMesh& m, const Tab<P, R>& t, int64_t e_first, int E,
                                        const XV* __restrict__ x, R* A) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int N = Z::N, Q = Z::Q;
  for (int w = threadIdx.x; w < E * N * N; w += blockDim.x) {
    const int le = w / (N * N), jk = w % (N * N);
    const int64_t e = e_first + le;
    if (e >= m.nel) continue;
    const int j = jk % N, k = jk / N;
    R u[N];
    if constexpr (GEN) {
      const int64_t* dm = m.edofs + e * (N * N * N) + jk * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int64_t d = dm[i];
        u[i] = m.ess[d] ? (R)0 : to_r<R>(x[d]);
      }
    } else {
      const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
      const int64_t J = ey * P + j, K = ez * P + k;
      const bool row_ess = J == 0 || K == 0 || J == m.ny - 1 || K == m.nz - 1;
      const XV* xr = x + (ex * P) + m.nx * (J + m.ny * K);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int64_t I = ex * P + i;
        u[i] = (row_ess || I == 0 || I == m.nx - 1) ? (R)0 : to_r<R>(xr[i]);
      }
    }
    R e_[Z::NH > 0 ? Z::NH : 1], o_[Z::NH > 0 ? Z::NH : 1], um;
    fold_n<P>(u, e_, o_, um);
    R yb[Q], yd[Q];
    fwd_B<P>(t, e_, o_, um, yb);
    fwd_D<P>(t, e_, o_, um, yd);
    R* a = A + (size_t)le * L::PER_ELEM + k * L::KS1 + j * L::LS;
#pragma unroll
    for (int g = 0; g < Q; ++g) {
      a[g] = yb[g];
      a[L::C1 + g] = yd[g];
    }
  }
}

// Y: A1 -> A2[c][k][g1][g0] with c = 0: B_y Bu (BB), 1: B_y du (BD), 2: d_y Bu (DB).
template <int P, typename R>
__device__ __forceinline__ void stage_y(const LorMesh& m, const Tab<P, R>& t, int64_t e_first, int E, R* A) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int N = Z::N, Q = Z::Q;
  for (int w = threadIdx.x; w < E * N * Q; w += blockDim.x) {
    const int le = w / (N * Q), r = w % (N * Q);
    if (e_first + le >= m.nel) continue;
    const int g0 = r % Q, k = r / Q;
    const R* a1 = A + (size_t)le * L::PER_ELEM;
    R* a2 = A + (size_t)le * L::PER_ELEM + L::A1;
    R bu[N], du[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      bu[j] = a1[k * L::KS1 + j * L::LS + g0];
      du[j] = a1[L::C1 + k * L::KS1 + j * L::LS + g0];
    }
    R eb[Z::NH > 0 ? Z::NH : 1], ob[Z::NH > 0 ? Z::NH : 1], mb, ed[Z::NH > 0 ? Z::NH : 1],
        od[Z::NH > 0 ? Z::NH : 1], md;
    fold_n<P>(bu, eb, ob, mb);
    fold_n<P>(du, ed, od, md);
    R y[Q];
    fwd_B<P>(t, eb, ob, mb, y);
#pragma unroll
    for (int g = 0; g < Q; ++g) a2[k * L::KS2 + g * Q + g0] = y[g];
    fwd_B<P>(t, ed, od, md, y);
#pragma unroll
    for (int g = 0; g < Q; ++g) a2[L::C2 + k * L::KS2 + g * Q + g0] = y[g];
    fwd_D<P>(t, eb, ob, mb, y);
#pragma unroll
    for (int g = 0; g < Q; ++g) a2[2 * L::C2 + k * L::KS2 + g * Q + g0] = y[g];
  }
}

// Reference gradient along one z line (g0, g1) from A2: g[c][g2]; with the
// reaction term also the values u[g2] = B_z BB (the mass basis operator).
template <int P, bool MASS, typename R>
__device__ __forceinline__ void line_gradient(const Tab<P, R>& t, const R* a2, int g01, R (*g)[Sz<P>::Q],
                                              R* u) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int N = Z::N;
  R v[N], e_[Z::NH > 0 ? Z::NH : 1], o_[Z::NH > 0 ? Z::NH : 1], vm;
  // d/dxi0 = B_z BD
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = a2[L::C2 + k * L::KS2 + g01];
  fold_n<P>(v, e_, o_, vm);
  fwd_B<P>(t, e_, o_, vm, g[0]);
  // d/dxi1 = B_z DB
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = a2[2 * L::C2 + k * L::KS2 + g01];
  fold_n<P>(v, e_, o_, vm);
  fwd_B<P>(t, e_, o_, vm, g[1]);
  // d/dxi2 = d_z BB
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = a2[k * L::KS2 + g01];
  fold_n<P>(v, e_, o_, vm);
  fwd_D<P>(t, e_, o_, vm, g[2]);
  if constexpr (MASS) fwd_B<P>(t, e_, o_, vm, u);
}

// Z' on one line: v[c][g2] -> T0 = B_z^T v0, T1 = B_z^T v1, T2 = d_z^T v2
// (+ B_z^T u with the reaction term) stored over A2[c][k][g1][g0] (the line's
// own entries).
template <int P, bool MASS, typename R>
__device__ __forceinline__ void line_transpose_z(const Tab<P, R>& t, R (*v)[Sz<P>::Q], const R* u, R* a2,
                                                 int g01) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int N = Z::N;
  R e_[Z::QH], o_[Z::QH], m_, y[N];
  fold_q<P>(v[0], e_, o_, m_);
  bwd<P, true, false>(t, e_, o_, m_, e_, o_, m_, y);
#pragma unroll
  for (int k = 0; k < N; ++k) a2[k * L::KS2 + g01] = y[k];
  fold_q<P>(v[1], e_, o_, m_);
  bwd<P, true, false>(t, e_, o_, m_, e_, o_, m_, y);
#pragma unroll
  for (int k = 0; k < N; ++k) a2[L::C2 + k * L::KS2 + g01] = y[k];
  if constexpr (MASS) {
    R e2[Z::QH], o2[Z::QH], m2;
    fold_q<P>(u, e_, o_, m_);
    fold_q<P>(v[2], e2, o2, m2);
    bwd<P, true, true>(t, e_, o_, m_, e2, o2, m2, y);
  } else {
    fold_q<P>(v[2], e_, o_, m_);
    bwd<P, false, true>(t, e_, o_, m_, e_, o_, m_, y);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) a2[2 * L::C2 + k * L::KS2 + g01] = y[k];
}

// u <- (beta w detJ) u at the q points of a z line (Mq[e][q^3])
template <int P, typename R>
__device__ __forceinline__ void line_apply_M(const R* __restrict__ Me, int g01, R* u) {
  constexpr int Q = Sz<P>::Q, Q2 = Q * Q;
#pragma unroll
  for (int g2 = 0; g2 < Q; ++g2) u[g2] *= Me[g01 + Q2 * g2];
}

// v <- D v at the q points of a z line (D[e][6][q^3], pt = g01 + q^2 g2)
template <int P, typename R>
__device__ __forceinline__ void line_apply_D(const R* __restrict__ De, int g01, R (*v)[Sz<P>::Q]) {
  using Z = Sz<P>;
  constexpr int Q = Z::Q, Q2 = Q * Q, Q3 = Q2 * Q;
#pragma unroll
  for (int g2 = 0; g2 < Q; ++g2) {
    const int pt = g01 + Q2 * g2;
    const R a = v[0][g2], b = v[1][g2], c = v[2][g2];
    const R d00 = De[pt], d01 = De[Q3 + pt], d02 = De[2 * Q3 + pt];
    const R d11 = De[3 * Q3 + pt], d12 = De[4 * Q3 + pt], d22 = De[5 * Q3 + pt];
    v[0][g2] = d00 * a + d01 * b + d02 * c;
    v[1][g2] = d01 * a + d11 * b + d12 * c;
    v[2][g2] = d02 * a + d12 * b + d22 * c;
  }
}

// Y': A2 (T0, T1, T2) -> A1[c][k][j][g0]: U0 = B_y^T T0, U1 = d_y^T T1 + B_y^T T2.
template <int P, typename R>
__device__ __forceinline__ void stage_y_t(const LorMesh& m, const Tab<P, R>& t, int64_t e_first, int E, R* A) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int N = Z::N, Q = Z::Q;
  for (int w = threadIdx.x; w < E * N * Q; w += blockDim.x) {
    const int le = w / (N * Q), r = w % (N * Q);
    if (e_first + le >= m.nel) continue;
    const int g0 = r % Q, k = r / Q;
    R* a1 = A + (size_t)le * L::PER_ELEM;
    const R* a2 = A + (size_t)le * L::PER_ELEM + L::A1;
    R v[Q], e1[Z::QH], o1[Z::QH], m1, e2[Z::QH], o2[Z::QH], m2, y[N];
#pragma unroll
    for (int g = 0; g < Q; ++g) v[g] = a2[k * L::KS2 + g * Q + g0];
    fold_q<P>(v, e1, o1, m1);
    bwd<P, true, false>(t, e1, o1, m1, e1, o1, m1, y);
#pragma unroll
    for (int j = 0; j < N; ++j) a1[k * L::KS1 + j * L::LS + g0] = y[j];
#pragma unroll
    for (int g = 0; g < Q; ++g) v[g] = a2[2 * L::C2 + k * L::KS2 + g * Q + g0];  // T2 (B^T)
    fold_q<P>(v, e1, o1, m1);
#pragma unroll
    for (int g = 0; g < Q; ++g) v[g] = a2[L::C2 + k * L::KS2 + g * Q + g0];  // T1 (d^T)
    fold_q<P>(v, e2, o2, m2);
    bwd<P, true, true>(t, e1, o1, m1, e2, o2, m2, y);
#pragma unroll
    for (int j = 0; j < N; ++j) a1[L::C1 + k * L::KS1 + j * L::LS + g0] = y[j];
  }
}

// X': A1 (U0, U1) -> y_line = d_x^T U0 + B_x^T U1, scatter-added into y.
template <int P, bool GEN, typename R, typename XV>
__device__ __forceinline__ void stage_x_t(const LorMesh& m, const Tab<P, R>& t, int64_t e_first, int E,
                                          const R* A, XV* __restrict__ y) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int N = Z::N, Q = Z::Q;
  for (int w = threadIdx.x; w < E * N * N; w += blockDim.x) {
    const int le = w / (N * N), jk = w % (N * N);
    const int64_t e = e_first + le;
    if (e >= m.nel) continue;
    const int j = jk % N, k = jk / N;
    const R* a1 = A + (size_t)le * L::PER_ELEM + k * L::KS1 + j * L::LS;
    R v[Q], e1[Z::QH], o1[Z::QH], m1, e2[Z::QH], o2[Z::QH], m2, yl[N];
#pragma unroll
    for (int g = 0; g < Q; ++g) v[g] = a1[L::C1 + g];  // U1 (B^T)
    fold_q<P>(v, e1, o1, m1);
#pragma unroll
    for (int g = 0; g < Q; ++g) v[g] = a1[g];  // U0 (d^T)
    fold_q<P>(v, e2, o2, m2);
    bwd<P, true, true>(t, e1, o1, m1, e2, o2, m2, yl);
    if constexpr (GEN) {
      const int64_t* dm = m.edofs + e * (N * N * N) + jk * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int64_t d = dm[i];
        if (!m.ess[d]) atomicAdd(y + d, to_out<XV>(yl[i]));
      }
    } else {
      const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
      const int64_t J = ey * P + j, K = ez * P + k;
      if (J == 0 || K == 0 || J == m.ny - 1 || K == m.nz - 1) continue;
      XV* yr = y + (ex * P) + m.nx * (J + m.ny * K);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int64_t I = ex * P + i;
        if (I != 0 && I != m.nx - 1) atomicAdd(yr + i, to_out<XV>(yl[i]));
      }
    }
  }
}

template <int P, bool MASS, bool GEN, typename R, typename XV>
__global__ void __launch_bounds__(Lay<P, R>::T) k_apply(LorMesh m, LorTables T, const R* __restrict__ Dq,
                                                    const R* __restrict__ Mq, const XV* __restrict__ x,
                                                    XV* __restrict__ y) {
  using Z = Sz<P>;
  using L = Lay<P, R>;
  constexpr int Q = Z::Q, Q2 = Q * Q, Q3 = Q2 * Q, E = Lay<P, R>::E;
  extern __shared__ __align__(16) unsigned char apply_smem[];
  R* sm = reinterpret_cast<R*>(apply_smem);
  const Tab<P, R> t = load_tables<P>(T, sm);
  R* A = sm + L::TABLES;
  __syncthreads();
  for (int64_t e_first = (int64_t)blockIdx.x * E; e_first < m.nel; e_first += (int64_t)gridDim.x * E) {
    if constexpr (Lay<P, R>::F32) {
      // L2 prefetch of the batch's D (and M), read by the z stage two barriers
      // later: its latency then overlaps the x and y stages
      const int64_t ne = m.nel - e_first < E ? m.nel - e_first : E;
      const char* d0 = reinterpret_cast<const char*>(Dq + e_first * 6 * Q3);
      const int64_t nb = ne * 6 * Q3 * (int64_t)sizeof(R);
      for (int64_t off = (int64_t)threadIdx.x * 128; off < nb; off += (int64_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(d0 + off));
      if constexpr (MASS) {
        const char* m0 = reinterpret_cast<const char*>(Mq + e_first * Q3);
        for (int64_t off = (int64_t)threadIdx.x * 128; off < nb / 6; off += (int64_t)blockDim.x * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(m0 + off));
      }
    }
    stage_x<P, GEN>(m, t, e_first, E, x, A);
    __syncthreads();
    stage_y<P>(m, t, e_first, E, A);
    __syncthreads();
    for (int w = threadIdx.x; w < E * Q2; w += blockDim.x) {
      const int le = w / Q2, g01 = w % Q2;
      const int64_t e = e_first + le;
      if (e >= m.nel) continue;
      R* a2 = A + (size_t)le * L::PER_ELEM + L::A1;
      R v[3][Q], u[MASS ? Q : 1];
      line_gradient<P, MASS>(t, a2, g01, v, u);
      line_apply_D<P>(Dq + e * 6 * Q3, g01, v);
      if constexpr (MASS) line_apply_M<P>(Mq + e * Q3, g01, u);
      line_transpose_z<P, MASS>(t, v, u, a2, g01);
    }
    __syncthreads();
    stage_y_t<P>(m, t, e_first, E, A);
    __syncthreads();
    stage_x_t<P, GEN>(m, t, e_first, E, A, y);
    __syncthreads();
  }
}

// Backward: holds both fields (gy in the first EB element slots, x in the
// next EB); gkappa = grad(x)^T (D / kappa) grad(gy) on each z line, and
// gx = A_p gy (with the reaction term if present) through the same
// transposed stages as the apply.
template <int P, bool MASS, bool GEN>
__global__ void __launch_bounds__(Sz<P>::TBW, P <= 6 ? 2 : 1) k_apply_backward(LorMesh m, LorTables T,
                                                             const double* __restrict__ Dq,
                                                             const double* __restrict__ Mq,
                                                             const double* __restrict__ kappa,
                                                             const double* __restrict__ x,
                                                             const double* __restrict__ gy,
                                                             double* __restrict__ gx,
                                                             double* __restrict__ gkappa) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int Q = Z::Q, Q2 = Q * Q, Q3 = Q2 * Q, E = Z::EB;
  extern __shared__ __align__(16) unsigned char apply_smem[];
  double* smem = reinterpret_cast<double*>(apply_smem);
  const Tab<P, double> t = load_tables<P>(T, smem);
  double* A = smem + L::TABLES;                    // gy: element slots 0..E-1
  double* AX = A + (size_t)E * L::PER_ELEM;        // x:  element slots E..2E-1
  __syncthreads();
  for (int64_t e_first = (int64_t)blockIdx.x * E; e_first < m.nel; e_first += (int64_t)gridDim.x * E) {
    stage_x<P, GEN>(m, t, e_first, E, gy, A);
    if (gkappa) stage_x<P, GEN>(m, t, e_first, E, x, AX);
    __syncthreads();
    stage_y<P>(m, t, e_first, E, A);
    if (gkappa) stage_y<P>(m, t, e_first, E, AX);
    __syncthreads();
    for (int w = threadIdx.x; w < E * Q2; w += blockDim.x) {
      const int le = w / Q2, g01 = w % Q2;
      const int64_t e = e_first + le;
      if (e >= m.nel) continue;
      const double* De = Dq + e * 6 * Q3;
      double* a2 = A + (size_t)le * L::PER_ELEM + L::A1;
      double v[3][Q], u[MASS ? Q : 1];
      line_gradient<P, MASS>(t, a2, g01, v, u);
      if (gkappa) {
        double gxl[3][Q];
        line_gradient<P, false, double>(t, AX + (size_t)le * L::PER_ELEM + L::A1, g01, gxl, nullptr);
#pragma unroll
        for (int g2 = 0; g2 < Q; ++g2) {
          const int pt = g01 + Q2 * g2;
          const double a = v[0][g2], b = v[1][g2], c = v[2][g2];
          const double d00 = De[pt], d01 = De[Q3 + pt], d02 = De[2 * Q3 + pt];
          const double d11 = De[3 * Q3 + pt], d12 = De[4 * Q3 + pt], d22 = De[5 * Q3 + pt];
          const double t0 = d00 * a + d01 * b + d02 * c;
          const double t1 = d01 * a + d11 * b + d12 * c;
          const double t2 = d02 * a + d12 * b + d22 * c;
          gkappa[e * Q3 + pt] = (gxl[0][g2] * t0 + gxl[1][g2] * t1 + gxl[2][g2] * t2) / kappa[e * Q3 + pt];
          v[0][g2] = t0;
          v[1][g2] = t1;
          v[2][g2] = t2;
        }
      } else {
        line_apply_D<P>(De, g01, v);
      }
      if constexpr (MASS) line_apply_M<P>(Mq + e * Q3, g01, u);
      if (gx) line_transpose_z<P, MASS>(t, v, u, a2, g01);
    }
    __syncthreads();
    if (gx) {
      stage_y_t<P>(m, t, e_first, E, A);
      __syncthreads();
      stage_x_t<P, GEN>(m, t, e_first, E, A, gx);
    }
    __syncthreads();
  }
}

template <typename K>
cudaError_t configure(K kernel, size_t bytes, unsigned* mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (!(*mask & (1u << dev))) {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
    // prefer the largest shared-memory carveout so that two CTAs fit per SM
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err != cudaSuccess) return err;
    *mask |= 1u << dev;
  }
  return cudaSuccess;
}

}  // namespace

#include "k_apply_fix.cuh"

namespace {

// The FP64 operator and its backward run the fixed-point kernels of
// k_apply_fix.cuh; the FP32-arithmetic operator the kernels above.
template <int P, bool MASS, bool GEN, typename R, typename XV>
cudaError_t apply_p(const LorMesh& m, const LorTables& T, const R* Dq, const R* Mq, const XV* x, XV* y,
                    cudaStream_t s) {
  if constexpr (sizeof(R) == sizeof(double)) return apply_fx_p<P, MASS, GEN>(m, T, Dq, Mq, x, y, s);
  using Z = Sz<P>;
  using L = Lay<P, R>;
  const size_t bytes = sizeof(R) * (L::TABLES + (size_t)L::E * L::PER_ELEM);
  static unsigned mask = 0;
  cudaError_t err = configure(k_apply<P, MASS, GEN, R, XV>, bytes, &mask);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (m.nel + L::E - 1) / L::E;
  k_apply<P, MASS, GEN, R, XV><<<(unsigned)blocks, L::T, bytes, s>>>(m, T, Dq, Mq, x, y); lor_count_launch();
  return cudaGetLastError();
}

template <int P, bool MASS, bool GEN>
cudaError_t backward_p(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq, const double* kappa,
                       const double* x, const double* gy, double* gx, double* gk, cudaStream_t s) {
  return backward_fx_p<P, MASS, GEN>(m, T, Dq, Mq, kappa, x, gy, gx, gk, s);
}
template <int P, bool MASS, bool GEN>
cudaError_t backward_fp64_p(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                            const double* kappa, const double* x, const double* gy, double* gx, double* gk,
                            cudaStream_t s) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  const size_t bytes = sizeof(double) * (L::TABLES + 2 * (size_t)Z::EB * L::PER_ELEM);
  static unsigned mask = 0;
  cudaError_t err = configure(k_apply_backward<P, MASS, GEN>, bytes, &mask);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (m.nel + Z::EB - 1) / Z::EB;
  k_apply_backward<P, MASS, GEN><<<(unsigned)blocks, Z::TBW, bytes, s>>>(m, T, Dq, Mq, kappa, x, gy, gx, gk);
  lor_count_launch();
  return cudaGetLastError();
}

template <bool MASS, bool GEN, typename R, typename XV = double>
cudaError_t apply_dispatch(const LorMesh& m, const LorTables& T, const R* Dq, const R* Mq, const XV* x, XV* y,
                           cudaStream_t s) {
  switch (m.p) {
#define LOR_CASE(P) \
  case P: return apply_p<P, MASS, GEN, R, XV>(m, T, Dq, Mq, x, y, s);
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <bool MASS, bool GEN>
cudaError_t backward_dispatch(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                              const double* kappa, const double* x, const double* gy, double* gx, double* gk,
                              cudaStream_t s) {
  switch (m.p) {
#define LOR_CASE(P) \
  case P: return backward_p<P, MASS, GEN>(m, T, Dq, Mq, kappa, x, gy, gx, gk, s);
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

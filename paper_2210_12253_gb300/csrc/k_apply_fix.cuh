// k_apply_fix.cuh -- the FP64 high-order apply and its backward with every
// contraction in exact-width 64-bit fixed point on the integer pipe
// (included by k_apply_impl.cuh).
//
// y = G^T B^T D B G x (Eq. (4) on one rank) by sum factorisation, as in the
// floating-point kernels of k_apply_impl.cuh (the same stages, the same
// even-odd folding, the same shared-memory layout), with this arithmetic:
//
//  * values: int64 X with |X| < 2^57 and one power-of-two scale per element
//    and stage (real value = X 2^-s).  The input x is converted with the
//    element's largest exponent; after every contraction stage each element is
//    renormalised so that its largest output has 57 bits again (a max over the
//    element in shared memory, at the barrier the stage ends with anyway).
//  * 1D tables: B_1D and its folded halves at one scale 2^S_B, d_1D and its
//    halves at 2^S_D (each from its own largest entry, |C| < 2^57).  Every
//    path from x to the Gauss points has one d and two B (so the three
//    gradient components share a scale), and so do the transposed sums that
//    meet (d^T T1 + B^T T2, d^T U0 + B^T U1); the mass values B(x)B(x)B sit
//    S_B - S_D above the gradient and are aligned before B^T u meets d^T v2.
//  * multiply-add (details at fx_mac below): the product X C / 2^56 from
//    three 32 x 32 -> 64 bit multiply-adds (mad.wide.s32) into two int64
//    accumulators; a contraction's output (at most 14 products) is rounded
//    once and reaches up to 2^62, so its largest value keeps 58-61 bits
//    before the next stage shifts it to 57.
//  * the pointwise product v = D g (D stored by the setup in fixed point, each
//    Gauss point's 6 entries at the point's largest exponent): each point's
//    gradient is renormalised to 57 bits, the 3 x 3 product is taken in the
//    same fixed point, the line's points are aligned to its largest scale,
//    and after the transposed z stage the lines of an element are aligned to
//    the element's largest (one more barrier).
//  * conversions int64 <-> FP64 by integer operations (rounding to nearest).
//
// The FP64 pipe of this GPU issues 2 multiply-adds per clock and SM, the
// integer multiply-add (including the 32 x 32 -> 64 bit form) 64: the
// contraction work moves from the one to the other, and only the FP64 atomics
// of the scatter (executed in L2) and the backward's division by kappa remain
// FP64.
#pragma once

#include "fixed_point.cuh"

namespace {

// Launch shape per degree, measured (apply and backward at about 3M DOFs,
// p = 4..8, against 2-4 alternatives each): elements per CTA (one thread per
// z line) and the CTAs per SM the register budget is sized for.  The kernels
// are bound by issue latency: two CTAs per SM (about 128 registers a thread,
// some spilled at high degree) beat one CTA with all state in registers by
// 1.3-1.7x for the apply; the backward holds two fields, and from p = 8 its
// spills at that budget cost more than the second CTA gains (at p = 4..7 one
// CTA per SM is 1.3-2.2x slower).
template <int P>
constexpr int kFxApplyBlocks = 2;
template <int P>
constexpr int kFxBackwardBlocks = P >= 8 ? 1 : 2;
template <int P>
constexpr int kFxE = P == 1 ? 28 : P == 2 ? 16 : P == 3 ? 10 : P == 4 ? 7 : P == 5 ? 5 : P == 6 ? 4 : P == 7 ? 3 : 2;
template <int P>
constexpr int kFxEB = P == 1 ? 28 : P == 2 ? 16 : P == 3 ? 10 : P == 4 ? 7 : P == 5 ? 5 : P == 6 ? 3 : P == 7 ? 2
                    : P == 8 ? 3 : P == 9 ? 2 : 1;
template <int P>
constexpr int kFxT = ((kFxE<P> * (P + 2) * (P + 2) + 31) / 32) * 32;
template <int P>
constexpr int kFxTB = ((kFxEB<P> * (P + 2) * (P + 2) + 31) / 32) * 32;

// table entry k, re-read from shared memory at each use (volatile: the
// tables are not held in registers across the line loops, as in the FP64
// kernels)
__device__ __forceinline__ FxC fx_tab(const long long* tbl, int k) {
  return fx_unpack(static_cast<const volatile long long*>(tbl)[k]);
}

// Table scales: S_B of B_1D and its folded halves, S_D of d_1D and its.
struct FxS {
  int B, D;
};

// Tables in shared memory (packed words, the order of Sz's FP64 layout): B, d (q x n), BE, BO, DE, DO (q x n/2); returns their scales.  The
// caller's barrier publishes them.
template <int P>
__device__ __forceinline__ FxS fx_load_tables(const LorTables& T, long long* s) {
  using Z = Sz<P>;
  int eb = 0, ed = 0;
  for (int x = 0; x < Z::TB; ++x) {
    eb = max(eb, fx_expo(T.B[x]));
    ed = max(ed, fx_expo(T.Dm[x]));
  }
  long long* B = s;
  long long* D = s + Z::TB;
  long long* BE = s + 2 * Z::TB;
  long long* BO = BE + Z::TF;
  long long* DE = BO + Z::TF;
  long long* DO = DE + Z::TF;
  for (int x = threadIdx.x; x < Z::TB; x += blockDim.x) {
    B[x] = fx_pack(fx_from_double(T.B[x], eb));
    D[x] = fx_pack(fx_from_double(T.Dm[x], ed));
  }
  // folded halves from the fixed-point entries (exact: (C0 +- C1) / 2 with
  // the last bit rounded)
  for (int x = threadIdx.x; x < Z::Q * Z::NH; x += blockDim.x) {
    const int g = x / Z::NH, i = x % Z::NH;
    const long long b0 = fx_from_double(T.B[g * Z::N + i], eb), b1 = fx_from_double(T.B[g * Z::N + Z::N - 1 - i], eb);
    const long long d0 = fx_from_double(T.Dm[g * Z::N + i], ed), d1 = fx_from_double(T.Dm[g * Z::N + Z::N - 1 - i], ed);
    BE[x] = fx_pack((b0 + b1 + 1) >> 1);
    BO[x] = fx_pack((b0 - b1 + 1) >> 1);
    DE[x] = fx_pack((d0 + d1 + 1) >> 1);
    DO[x] = fx_pack((d0 - d1 + 1) >> 1);
  }
  return FxS{1079 - eb, 1079 - ed};
}

template <int P>
struct FxTab {
  const long long *B, *D, *BE, *BO, *DE, *DO;
};
template <int P>
__device__ __forceinline__ FxTab<P> fx_tables(const long long* s) {
  using Z = Sz<P>;
  FxTab<P> t;
  t.B = s;
  t.D = s + Z::TB;
  t.BE = s + 2 * Z::TB;
  t.BO = t.BE + Z::TF;
  t.DE = t.BO + Z::TF;
  t.DO = t.DE + Z::TF;
  return t;
}

// folded input of a contraction over n nodes (u: |u| <= 2^57)
template <int P>
struct FxFoldN {
  FxX e[Sz<P>::NH > 0 ? Sz<P>::NH : 1], o[Sz<P>::NH > 0 ? Sz<P>::NH : 1], m;
};
template <int P>
__device__ __forceinline__ FxFoldN<P> fx_fold_n(const long long* u) {
  using Z = Sz<P>;
  FxFoldN<P> f;
#pragma unroll
  for (int i = 0; i < Z::NH; ++i) {
    f.e[i] = fx_x(u[i] + u[Z::N - 1 - i]);
    f.o[i] = fx_x(u[i] - u[Z::N - 1 - i]);
  }
  f.m = fx_x(Z::NODD ? u[Z::NM] : 0ll);
  return f;
}
// folded input of a transposed contraction over q points
template <int P>
struct FxFoldQ {
  FxX e[Sz<P>::QH], o[Sz<P>::QH], m;
};
template <int P>
__device__ __forceinline__ FxFoldQ<P> fx_fold_q(const long long* v) {
  using Z = Sz<P>;
  FxFoldQ<P> f;
#pragma unroll
  for (int g = 0; g < Z::QH; ++g) {
    f.e[g] = fx_x(v[g] + v[Z::Q - 1 - g]);
    f.o[g] = fx_x(v[g] - v[Z::Q - 1 - g]);
  }
  f.m = fx_x(Z::QODD ? v[Z::QM] : 0ll);
  return f;
}

// y = B_1D u (folded): y_g = Ev + Od, y_{q-1-g} = Ev - Od
template <int P>
__device__ __forceinline__ void fx_fwd_B(const FxTab<P>& t, const FxFoldN<P>& f, long long* y) {
  using Z = Sz<P>;
#pragma unroll
  for (int g = 0; g < Z::QH; ++g) {
    FAcc ev = fx_acc(), od = fx_acc();
    if (Z::NODD) fx_mac(ev, f.m, fx_tab(t.B, g * Z::N + Z::NM));
#pragma unroll
    for (int i = 0; i < Z::NH; ++i) {
      fx_mac(ev, f.e[i], fx_tab(t.BE, g * Z::NH + i));
      fx_mac(od, f.o[i], fx_tab(t.BO, g * Z::NH + i));
    }
    const long long a = fx_res(ev), b = fx_res(od);
    y[g] = a + b;
    y[Z::Q - 1 - g] = a - b;
  }
  if (Z::QODD) {
    FAcc ev = fx_acc();
#pragma unroll
    for (int i = 0; i < Z::NH; ++i) fx_mac(ev, f.e[i], fx_tab(t.BE, Z::QM * Z::NH + i));
    y[Z::QM] = fx_res(ev);
  }
}
// y = d_1D u (folded): y_g = Od + Ev, y_{q-1-g} = Od - Ev
template <int P>
__device__ __forceinline__ void fx_fwd_D(const FxTab<P>& t, const FxFoldN<P>& f, long long* y) {
  using Z = Sz<P>;
#pragma unroll
  for (int g = 0; g < Z::QH; ++g) {
    FAcc s = fx_acc(), d = fx_acc();
    if (Z::NODD) fx_mac(s, f.m, fx_tab(t.D, g * Z::N + Z::NM));
#pragma unroll
    for (int i = 0; i < Z::NH; ++i) {
      fx_mac(s, f.e[i], fx_tab(t.DE, g * Z::NH + i));
      fx_mac(d, f.o[i], fx_tab(t.DO, g * Z::NH + i));
    }
    const long long a = fx_res(s), b = fx_res(d);
    y[g] = b + a;
    y[Z::Q - 1 - g] = b - a;
  }
  if (Z::QODD) {
    FAcc d = fx_acc();
#pragma unroll
    for (int i = 0; i < Z::NH; ++i) fx_mac(d, f.o[i], fx_tab(t.DO, Z::QM * Z::NH + i));
    y[Z::QM] = fx_res(d);
  }
}
// y = B_1D^T v1 + d_1D^T v2 (either part may be off), v1, v2 folded over q
template <int P, bool USE_B, bool USE_D>
__device__ __forceinline__ void fx_bwd(const FxTab<P>& t, const FxFoldQ<P>& f1, const FxFoldQ<P>& f2,
                                       long long* y) {
  using Z = Sz<P>;
#pragma unroll
  for (int i = 0; i < Z::NH; ++i) {
    FAcc a1 = fx_acc(), a2 = fx_acc();
    if (Z::QODD) {
      if (USE_B) fx_mac(a1, f1.m, fx_tab(t.B, Z::QM * Z::N + i));
      if (USE_D) fx_mac(a2, f2.m, fx_tab(t.D, Z::QM * Z::N + i));
    }
#pragma unroll
    for (int g = 0; g < Z::QH; ++g) {
      if (USE_B) {
        fx_mac(a1, f1.e[g], fx_tab(t.BE, g * Z::NH + i));
        fx_mac(a2, f1.o[g], fx_tab(t.BO, g * Z::NH + i));
      }
      if (USE_D) {
        fx_mac(a1, f2.o[g], fx_tab(t.DE, g * Z::NH + i));
        fx_mac(a2, f2.e[g], fx_tab(t.DO, g * Z::NH + i));
      }
    }
    const long long a = fx_res(a1), b = fx_res(a2);
    y[i] = a + b;
    y[Z::N - 1 - i] = a - b;
  }
  if (Z::NODD) {
    FAcc s = fx_acc();
#pragma unroll
    for (int g = 0; g < Z::QH; ++g) {
      if (USE_B) fx_mac(s, f1.e[g], fx_tab(t.B, g * Z::N + Z::NM));
      if (USE_D) fx_mac(s, f2.o[g], fx_tab(t.D, g * Z::N + Z::NM));
    }
    y[Z::NM] = fx_res(s);
  }
}

// Per-element scale bookkeeping in shared memory, one row per field (a
// stage's outputs share one shift; the scales named are those of the
// components with the fewest d, the others sit S_D - S_B off):
//   [0] largest exponent of the gathered x  -> s0 = 1079 - it
//   [1] bit length after the x stage        -> Bu at s1 = s0 + S_B - 58 + (57 - it)
//   [2] bit length after the y stage        -> BB at s2 = s1 + S_B - 58 + (57 - it);
//                                              gradient at sg = s2 + S_D - 58
//   [3] largest real exponent after the z^T stage, + kFxBias -> T0 at s3 = 57 - (it - kFxBias)
//   [4] bit length after the y^T stage      -> U0 at s4 = s3 + S_B - 58 + (57 - it);
//                                              output at s4 + S_D - 58
// (a stage's outputs reach up to 2^61; the next stage reads them shifted to
// 57 bits, right or left)
constexpr int kFxSlots = 5, kFxBias = 1 << 14;

struct FxScales {
  int s1, s2, sg;
};
__device__ __forceinline__ FxScales fx_fwd_scales(const int* sl, FxS S) {
  FxScales r;
  const int s0 = 1079 - sl[0];
  r.s1 = s0 + S.B - kFxMacShift + (kFxTop - sl[1]);
  r.s2 = r.s1 + S.B - kFxMacShift + (kFxTop - sl[2]);
  r.sg = r.s2 + S.D - kFxMacShift;
  return r;
}

// Gather of one x line (N nodes) through the element map, essential DOFs
// masked to zero.
template <int P, bool GEN>
__device__ __forceinline__ void fx_gather(const LorMesh& m, int64_t e, int jk, const double* __restrict__ x,
                                          double* u) {
  using Z = Sz<P>;
  constexpr int N = Z::N;
  if constexpr (GEN) {
    const int64_t* dm = m.edofs + e * (N * N * N) + jk * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int64_t d = dm[i];
      u[i] = m.ess[d] ? 0.0 : x[d];
    }
  } else {
    const int j = jk % N, k = jk / N;
    const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
    const int64_t J = ey * P + j, K = ez * P + k;
    const bool row_ess = J == 0 || K == 0 || J == m.ny - 1 || K == m.nz - 1;
    const double* xr = x + (ex * P) + m.nx * (J + m.ny * K);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int64_t I = ex * P + i;
      u[i] = (row_ess || I == 0 || I == m.nx - 1) ? 0.0 : xr[i];
    }
  }
}

// X stage, second half: u (FP64, gathered) -> A1 = (B u, d u) along x at the
// element's input scale; records the outputs' bit length.
template <int P>
__device__ __forceinline__ void fx_stage_x(const FxTab<P>& t, const double* u, int emax, long long* a,
                                           int* bits) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N, Q = Z::Q;
  long long X[N];
#pragma unroll
  for (int i = 0; i < N; ++i) X[i] = fx_from_double(u[i], emax);
  const FxFoldN<P> f = fx_fold_n<P>(X);
  long long y[Q];
  unsigned long long acc = 0;
  fx_fwd_B<P>(t, f, y);
#pragma unroll
  for (int g = 0; g < Q; ++g) {
    a[g] = y[g];
    fx_or(acc, y[g]);
  }
  fx_fwd_D<P>(t, f, y);
#pragma unroll
  for (int g = 0; g < Q; ++g) {
    a[L::C1 + g] = y[g];
    fx_or(acc, y[g]);
  }
  atomicMax(bits, fx_bits(acc));
}

// Y stage on line (k, g0): A1 (shifted by sh) -> A2 = (BB, BD, DB)
template <int P>
__device__ __forceinline__ void fx_stage_y(const FxTab<P>& t, long long* A, int r, int sh, int* bits) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N, Q = Z::Q;
  const int g0 = r % Q, k = r / Q;
  const long long* a1 = A;
  long long* a2 = A + L::A1;
  long long bu[N], du[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    bu[j] = fx_rescale(a1[k * L::KS1 + j * L::LS + g0], sh);
    du[j] = fx_rescale(a1[L::C1 + k * L::KS1 + j * L::LS + g0], sh);
  }
  const FxFoldN<P> fb = fx_fold_n<P>(bu), fd = fx_fold_n<P>(du);
  long long y[Q];
  unsigned long long acc = 0;
  fx_fwd_B<P>(t, fb, y);
#pragma unroll
  for (int g = 0; g < Q; ++g) {
    a2[k * L::KS2 + g * Q + g0] = y[g];
    fx_or(acc, y[g]);
  }
  fx_fwd_B<P>(t, fd, y);
#pragma unroll
  for (int g = 0; g < Q; ++g) {
    a2[L::C2 + k * L::KS2 + g * Q + g0] = y[g];
    fx_or(acc, y[g]);
  }
  fx_fwd_D<P>(t, fb, y);
#pragma unroll
  for (int g = 0; g < Q; ++g) {
    a2[2 * L::C2 + k * L::KS2 + g * Q + g0] = y[g];
    fx_or(acc, y[g]);
  }
  atomicMax(bits, fx_bits(acc));
}

// Z stage on line g01: A2 (shifted by sh) -> g[c][g2] (+ the mass values u
// = B_z BB) at the gradient scale.
template <int P, bool MASS>
__device__ __forceinline__ void fx_line_gradient(const FxTab<P>& t, const long long* a2, int g01, int sh,
                                                 long long (*g)[Sz<P>::Q], long long* u) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N;
  long long v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = fx_rescale(a2[L::C2 + k * L::KS2 + g01], sh);
  fx_fwd_B<P>(t, fx_fold_n<P>(v), g[0]);
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = fx_rescale(a2[2 * L::C2 + k * L::KS2 + g01], sh);
  fx_fwd_B<P>(t, fx_fold_n<P>(v), g[1]);
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = fx_rescale(a2[k * L::KS2 + g01], sh);
  const FxFoldN<P> f = fx_fold_n<P>(v);
  fx_fwd_D<P>(t, f, g[2]);
  if constexpr (MASS) fx_fwd_B<P>(t, f, u);
}

// v = D g at the q points of a z line, D in the setup's fixed-point form
// (packed entries De[c][q^3] at each point's scale, offsets Ds[q^3]): per
// point the gradient renormalised to 57 bits, the 3 x 3 product in fixed
// point; sc[g2] is v's scale relative to the gradient's (INT_MAX where v is
// zero).  With the reaction term also
// u <- M u, scm[g2] the scale at which u must be aligned with v (u meets d^T
// v2 through B^T: it sits S_D - S_B off v after the alignment).
template <int P, bool MASS>
__device__ __forceinline__ void fx_line_D(const long long* __restrict__ De, const int* __restrict__ Ds,
                                          const double* __restrict__ Me, int g01, FxS S, long long (*g)[Sz<P>::Q],
                                          long long* u, int* sc, int* scm) {
  using Z = Sz<P>;
  constexpr int Q = Z::Q, Q2 = Q * Q, Q3 = Q2 * Q;
#pragma unroll
  for (int g2 = 0; g2 < Q; ++g2) {
    const int pt = g01 + Q2 * g2;
    FxC D[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) D[c] = fx_c_packed(De[c * Q3 + pt]);
    const int sd = Ds[pt];
    unsigned long long og = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) fx_or(og, g[c][g2]);
    const int shg = kFxTop - fx_bits(og);
    const FxX a = fx_x(fx_shift(g[0][g2], shg)), b = fx_x(fx_shift(g[1][g2], shg)), c = fx_x(fx_shift(g[2][g2], shg));
    FAcc v0 = fx_acc(), v1 = fx_acc(), v2 = fx_acc();
    fx_mac(v0, a, D[0]);
    fx_mac(v0, b, D[1]);
    fx_mac(v0, c, D[2]);
    fx_mac(v1, a, D[1]);
    fx_mac(v1, b, D[3]);
    fx_mac(v1, c, D[4]);
    fx_mac(v2, a, D[2]);
    fx_mac(v2, b, D[4]);
    fx_mac(v2, c, D[5]);
    g[0][g2] = fx_res(v0);
    g[1][g2] = fx_res(v1);
    g[2][g2] = fx_res(v2);
    sc[g2] = (sd == INT_MAX || og == 0) ? INT_MAX : sd - kFxMacShift + shg;
    if constexpr (MASS) {
      const double mv = Me[pt];
      const int emm = fx_expo(mv);
      const int shu = kFxTop - fx_bits((unsigned long long)(u[g2] ^ (u[g2] >> 63)));
      FAcc w = fx_acc();
      fx_mac(w, fx_x(fx_shift(u[g2], shu)), fx_c(fx_from_double(mv, emm)));
      u[g2] = fx_res(w);
      // u (B(x)B(x)B) sits S_B - S_D above the gradient; B^T u must come out
      // at the scale of d^T v2, so u is aligned as if S_B - S_D finer again
      scm[g2] = (emm == 0 || u[g2] == 0) ? INT_MAX : 1079 - emm - kFxMacShift + shu + 2 * (S.B - S.D);
    }
  }
}

// Aligns the q points of a line (scale offsets sc, scm) to the coarsest,
// renormalises the line to 57 bits and returns its scale offset (relative to
// the gradient scale).
template <int P, bool MASS>
__device__ __forceinline__ int fx_line_align(long long (*v)[Sz<P>::Q], long long* u, const int* sc, const int* scm) {
  using Z = Sz<P>;
  constexpr int Q = Z::Q;
  int smin = INT_MAX;
#pragma unroll
  for (int g2 = 0; g2 < Q; ++g2) {
    smin = min(smin, sc[g2]);
    if (MASS) smin = min(smin, scm[g2]);
  }
  if (smin == INT_MAX) smin = 0;  // D (and M) zero along the whole line
  unsigned long long acc = 0;
#pragma unroll
  for (int g2 = 0; g2 < Q; ++g2) {
    const int r = sc[g2] == INT_MAX ? 63 : sc[g2] - smin;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c][g2] = fx_shift(v[c][g2], -r);
      fx_or(acc, v[c][g2]);
    }
    if (MASS) {
      const int rm = scm[g2] == INT_MAX ? 63 : scm[g2] - smin;
      u[g2] = fx_shift(u[g2], -rm);
      fx_or(acc, u[g2]);
    }
  }
  const int sh = kFxTop - fx_bits(acc);
#pragma unroll
  for (int g2 = 0; g2 < Q; ++g2) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c][g2] = fx_shift(v[c][g2], sh);
    if (MASS) u[g2] = fx_shift(u[g2], sh);
  }
  return smin + sh;
}

// Z^T on a line: T0 = B_z^T v0, T1 = B_z^T v1, T2 = d_z^T v2 (+ B_z^T u),
// kept in registers (y[c][k]); returns their OR-ed magnitudes.
template <int P, bool MASS>
__device__ __forceinline__ unsigned long long fx_line_transpose_z(const FxTab<P>& t, long long (*v)[Sz<P>::Q],
                                                                  const long long* u,
                                                                  long long (*y)[Sz<P>::N]) {
  using Z = Sz<P>;
  constexpr int N = Z::N;
  unsigned long long acc = 0;
  {
    const FxFoldQ<P> f = fx_fold_q<P>(v[0]);
    fx_bwd<P, true, false>(t, f, f, y[0]);
  }
  {
    const FxFoldQ<P> f = fx_fold_q<P>(v[1]);
    fx_bwd<P, true, false>(t, f, f, y[1]);
  }
  if constexpr (MASS) {
    const FxFoldQ<P> f1 = fx_fold_q<P>(u), f2 = fx_fold_q<P>(v[2]);
    fx_bwd<P, true, true>(t, f1, f2, y[2]);
  } else {
    const FxFoldQ<P> f = fx_fold_q<P>(v[2]);
    fx_bwd<P, false, true>(t, f, f, y[2]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < N; ++k) fx_or(acc, y[c][k]);
  return acc;
}

// Y^T on line (k, g0): A2 (T0, T1, T2; shifted by sh) -> A1: U0 = B_y^T T0,
// U1 = d_y^T T1 + B_y^T T2
template <int P>
__device__ __forceinline__ void fx_stage_y_t(const FxTab<P>& t, long long* A, int r, int sh, int* bits) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N, Q = Z::Q;
  const int g0 = r % Q, k = r / Q;
  long long* a1 = A;
  const long long* a2 = A + L::A1;
  long long v[Q], y[N];
  unsigned long long acc = 0;
#pragma unroll
  for (int g = 0; g < Q; ++g) v[g] = fx_rescale(a2[k * L::KS2 + g * Q + g0], sh);
  {
    const FxFoldQ<P> f = fx_fold_q<P>(v);
    fx_bwd<P, true, false>(t, f, f, y);
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    a1[k * L::KS1 + j * L::LS + g0] = y[j];
    fx_or(acc, y[j]);
  }
#pragma unroll
  for (int g = 0; g < Q; ++g) v[g] = fx_rescale(a2[2 * L::C2 + k * L::KS2 + g * Q + g0], sh);
  const FxFoldQ<P> f1 = fx_fold_q<P>(v);  // T2 (B^T)
#pragma unroll
  for (int g = 0; g < Q; ++g) v[g] = fx_rescale(a2[L::C2 + k * L::KS2 + g * Q + g0], sh);
  const FxFoldQ<P> f2 = fx_fold_q<P>(v);  // T1 (d^T)
  fx_bwd<P, true, true>(t, f1, f2, y);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    a1[L::C1 + k * L::KS1 + j * L::LS + g0] = y[j];
    fx_or(acc, y[j]);
  }
  atomicMax(bits, fx_bits(acc));
}

// X^T on line jk: A1 (U0, U1; shifted by sh) -> y_line = d_x^T U0 + B_x^T U1
// at scale so, scatter-added into y as FP64.
template <int P, bool GEN>
__device__ __forceinline__ void fx_stage_x_t(const LorMesh& m, const FxTab<P>& t, int64_t e, int jk,
                                             const long long* A, int sh, int so, double* __restrict__ y) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N, Q = Z::Q;
  const int j = jk % N, k = jk / N;
  const long long* a1 = A + k * L::KS1 + j * L::LS;
  long long v[Q], yl[N];
#pragma unroll
  for (int g = 0; g < Q; ++g) v[g] = fx_rescale(a1[L::C1 + g], sh);  // U1 (B^T)
  const FxFoldQ<P> f1 = fx_fold_q<P>(v);
#pragma unroll
  for (int g = 0; g < Q; ++g) v[g] = fx_rescale(a1[g], sh);  // U0 (d^T)
  const FxFoldQ<P> f2 = fx_fold_q<P>(v);
  fx_bwd<P, true, true>(t, f1, f2, yl);
  if constexpr (GEN) {
    const int64_t* dm = m.edofs + e * (N * N * N) + jk * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int64_t d = dm[i];
      if (!m.ess[d]) atomicAdd(y + d, fx_to_double(yl[i], so));
    }
  } else {
    const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
    const int64_t J = ey * P + j, K = ez * P + k;
    if (J == 0 || K == 0 || J == m.ny - 1 || K == m.nz - 1) return;
    double* yr = y + (ex * P) + m.nx * (J + m.ny * K);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int64_t I = ex * P + i;
      if (I != 0 && I != m.nx - 1) atomicAdd(yr + i, fx_to_double(yl[i], so));
    }
  }
}

// The transposed half shared by the apply and the backward: the z-line
// results T (registers, line scale sline relative to the gradient scale) are
// aligned to the element, then Y^T and X^T.  Every thread of the CTA calls
// it (it holds barriers).
template <int P, bool GEN>
__device__ __forceinline__ void fx_transposed(const LorMesh& m, const FxTab<P>& t, FxS S, int64_t e_first,
                                              int E, long long* A, int* sl, int sg, bool az, int lez, int g01,
                                              int sline, unsigned long long accT,
                                              long long (*T)[Sz<P>::N], double* __restrict__ y) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N, Q = Z::Q, NN = N * N, NQ = N * Q;
  const int w = threadIdx.x;
  // line's real magnitude exponent: bits - (scale of T)
  const int sT = sg + sline + S.B - kFxMacShift;
  if (az && accT) atomicMax(&sl[lez * kFxSlots + 3], fx_bits(accT) - sT + kFxBias);
  __syncthreads();
  if (az && accT) {
    const int s3 = kFxTop - (sl[lez * kFxSlots + 3] - kFxBias);
    const int sh = s3 - sT;
    long long* a2 = A + (size_t)lez * L::PER_ELEM + L::A1;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < N; ++k) a2[c * L::C2 + k * L::KS2 + g01] = fx_shift(T[c][k], sh);
  } else if (az) {
    long long* a2 = A + (size_t)lez * L::PER_ELEM + L::A1;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < N; ++k) a2[c * L::C2 + k * L::KS2 + g01] = 0;
  }
  __syncthreads();
  {
    const int le = w / NQ;
    if (w < E * NQ && e_first + le < m.nel)
      fx_stage_y_t<P>(t, A + (size_t)le * L::PER_ELEM, w % NQ, 0, &sl[le * kFxSlots + 4]);
  }
  __syncthreads();
  {
    const int le = w / NN;
    if (w < E * NN && e_first + le < m.nel) {
      const int* s = sl + le * kFxSlots;
      const int s3 = kFxTop - (s[3] - kFxBias);
      const int dyn4 = kFxTop - s[4];
      const int s4 = s3 + S.B - kFxMacShift + dyn4;
      fx_stage_x_t<P, GEN>(m, t, e_first + le, w % NN, A + (size_t)le * L::PER_ELEM, dyn4, s4 + S.D - kFxMacShift,
                           y);
    }
  }
}

// The forward half: gather, X and Y stages (3 barriers) for one field, or
// for two (the backward's gy and x, TWO at run time) sharing the barriers.
// Every thread of the CTA calls it.
template <int P, bool GEN>
__device__ __forceinline__ void fx_forward_xy(const LorMesh& m, const FxTab<P>& t, int64_t e_first, int E,
                                              const double* __restrict__ x, long long* A, int* sl,
                                              const double* __restrict__ x2 = nullptr, long long* A2 = nullptr,
                                              int* sl2 = nullptr) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int N = Z::N, Q = Z::Q, NN = N * N, NQ = N * Q;
  const int w = threadIdx.x;
  const int lex = w / NN;
  const bool ax = w < E * NN && e_first + lex < m.nel;
  const bool two = x2 != nullptr;
  double u[N], u2[N];
  if (ax) {
    fx_gather<P, GEN>(m, e_first + lex, w % NN, x, u);
    int em = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) em = max(em, fx_expo(u[i]));
    atomicMax(&sl[lex * kFxSlots + 0], em);
    if (two) {
      fx_gather<P, GEN>(m, e_first + lex, w % NN, x2, u2);
      em = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) em = max(em, fx_expo(u2[i]));
      atomicMax(&sl2[lex * kFxSlots + 0], em);
    }
  }
  __syncthreads();
  if (ax) {
    const int jk = w % NN, j = jk % N, k = jk / N;
    const size_t off = (size_t)lex * L::PER_ELEM + k * L::KS1 + j * L::LS;
    fx_stage_x<P>(t, u, sl[lex * kFxSlots + 0], A + off, &sl[lex * kFxSlots + 1]);
    if (two) fx_stage_x<P>(t, u2, sl2[lex * kFxSlots + 0], A2 + off, &sl2[lex * kFxSlots + 1]);
  }
  __syncthreads();
  {
    const int le = w / NQ;
    if (w < E * NQ && e_first + le < m.nel) {
      fx_stage_y<P>(t, A + (size_t)le * L::PER_ELEM, w % NQ, kFxTop - sl[le * kFxSlots + 1],
                    &sl[le * kFxSlots + 2]);
      if (two)
        fx_stage_y<P>(t, A2 + (size_t)le * L::PER_ELEM, w % NQ, kFxTop - sl2[le * kFxSlots + 1],
                      &sl2[le * kFxSlots + 2]);
    }
  }
  __syncthreads();
}

template <int P, bool MASS, bool GEN>
__global__ void __launch_bounds__(kFxT<P>, kFxApplyBlocks<P>) k_apply_fx(LorMesh m, LorTables T, const double* __restrict__ Dq,
                                                       const double* __restrict__ Mq, const double* __restrict__ x,
                                                       double* __restrict__ y) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int Q = Z::Q, Q2 = Q * Q, Q3 = Q2 * Q, E = kFxE<P>, N = Z::N;
  extern __shared__ __align__(16) unsigned char apply_smem[];
  __shared__ int sl[E * kFxSlots];
  long long* tb = reinterpret_cast<long long*>(apply_smem);
  const FxS S = fx_load_tables<P>(T, tb);
  const FxTab<P> t = fx_tables<P>(tb);
  long long* A = tb + Z::TABLES;
  for (int64_t e_first = (int64_t)blockIdx.x * E; e_first < m.nel; e_first += (int64_t)gridDim.x * E) {
    for (int i = threadIdx.x; i < E * kFxSlots; i += blockDim.x) sl[i] = 0;
    __syncthreads();
    {  // L2 prefetch of the batch's D (and M), read by the z stage after the x and y stages
      const int64_t ne = m.nel - e_first < E ? m.nel - e_first : E;
      const char* d0 = reinterpret_cast<const char*>(Dq + e_first * 6 * Q3);
      const int64_t nb = ne * 6 * Q3 * (int64_t)sizeof(double);
      for (int64_t off = (int64_t)threadIdx.x * 128; off < nb; off += (int64_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(d0 + off));
      const char* s0 = reinterpret_cast<const char*>(lor_d_scales(Dq, m.nel * Q3) + e_first * Q3);
      for (int64_t off = (int64_t)threadIdx.x * 128; off < ne * Q3 * 4; off += (int64_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(s0 + off));
      if constexpr (MASS) {
        const char* m0 = reinterpret_cast<const char*>(Mq + e_first * Q3);
        for (int64_t off = (int64_t)threadIdx.x * 128; off < nb / 6; off += (int64_t)blockDim.x * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(m0 + off));
      }
    }
    fx_forward_xy<P, GEN>(m, t, e_first, E, x, A, sl);
    const int w = threadIdx.x, lez = w / Q2, g01 = w % Q2;
    const bool az = w < E * Q2 && e_first + lez < m.nel;
    long long Tz[3][N];
    int sline = 0, sg = 0;
    unsigned long long accT = 0;
    if (az) {
      const int64_t e = e_first + lez;
      const FxScales sc = fx_fwd_scales(sl + lez * kFxSlots, S);
      sg = sc.sg;
      long long v[3][Q], u[MASS ? Q : 1];
      int ps[Q], pm[MASS ? Q : 1];
      fx_line_gradient<P, MASS>(t, A + (size_t)lez * L::PER_ELEM + L::A1, g01, kFxTop - sl[lez * kFxSlots + 2], v,
                                u);
      fx_line_D<P, MASS>(reinterpret_cast<const long long*>(Dq) + e * 6 * Q3, lor_d_scales(Dq, m.nel * Q3) + e * Q3,
                         MASS ? Mq + e * Q3 : nullptr, g01, S, v, u, ps, pm);
      sline = fx_line_align<P, MASS>(v, u, ps, pm);
      accT = fx_line_transpose_z<P, MASS>(t, v, u, Tz);
    }
    fx_transposed<P, GEN>(m, t, S, e_first, E, A, sl, sg, az, lez, g01, sline, accT, Tz, y);
    __syncthreads();
  }
}

template <int P, bool MASS, bool GEN>
cudaError_t apply_fx_p(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq, const double* x,
                       double* y, cudaStream_t s) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  const size_t bytes = sizeof(long long) * (Z::TABLES + (size_t)kFxE<P> * L::PER_ELEM);
  static unsigned mask = 0;
  cudaError_t err = configure(k_apply_fx<P, MASS, GEN>, bytes, &mask);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (m.nel + kFxE<P> - 1) / kFxE<P>;
  k_apply_fx<P, MASS, GEN><<<(unsigned)blocks, kFxT<P>, bytes, s>>>(m, T, Dq, Mq, x, y);
  lor_count_launch();
  return cudaGetLastError();
}

// Backward: gy's field in A, x's in AX (when gkappa is wanted);
// gkappa = grad(x)^T (D / kappa) grad(gy) per Gauss point, gx = A_p gy
// through the same transposed half as the apply.
template <int P, bool MASS, bool GEN>
__global__ void __launch_bounds__(kFxTB<P>, kFxBackwardBlocks<P>) k_apply_backward_fx(LorMesh m, LorTables T,
                                                                  const double* __restrict__ Dq,
                                                                  const double* __restrict__ Mq,
                                                                  const double* __restrict__ kappa,
                                                                  const double* __restrict__ x,
                                                                  const double* __restrict__ gy,
                                                                  double* __restrict__ gx,
                                                                  double* __restrict__ gkappa) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  constexpr int Q = Z::Q, Q2 = Q * Q, Q3 = Q2 * Q, E = kFxEB<P>, N = Z::N;
  extern __shared__ __align__(16) unsigned char apply_smem[];
  __shared__ int sl[E * kFxSlots], slx[E * kFxSlots];
  long long* tb = reinterpret_cast<long long*>(apply_smem);
  const FxS S = fx_load_tables<P>(T, tb);
  const FxTab<P> t = fx_tables<P>(tb);
  long long* A = tb + Z::TABLES;  // gy: element slots 0..E-1
  long long* AX = A + (size_t)E * L::PER_ELEM;  // x:  element slots E..2E-1
  for (int64_t e_first = (int64_t)blockIdx.x * E; e_first < m.nel; e_first += (int64_t)gridDim.x * E) {
    for (int i = threadIdx.x; i < E * kFxSlots; i += blockDim.x) {
      sl[i] = 0;
      slx[i] = 0;
    }
    __syncthreads();
    {  // L2 prefetch of the batch's D (and M), read by the z stage after the x and y stages
      const int64_t ne = m.nel - e_first < E ? m.nel - e_first : E;
      const char* d0 = reinterpret_cast<const char*>(Dq + e_first * 6 * Q3);
      const int64_t nb = ne * 6 * Q3 * (int64_t)sizeof(double);
      for (int64_t off = (int64_t)threadIdx.x * 128; off < nb; off += (int64_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(d0 + off));
      const char* s0 = reinterpret_cast<const char*>(lor_d_scales(Dq, m.nel * Q3) + e_first * Q3);
      for (int64_t off = (int64_t)threadIdx.x * 128; off < ne * Q3 * 4; off += (int64_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(s0 + off));
      if constexpr (MASS) {
        const char* m0 = reinterpret_cast<const char*>(Mq + e_first * Q3);
        for (int64_t off = (int64_t)threadIdx.x * 128; off < nb / 6; off += (int64_t)blockDim.x * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(m0 + off));
      }
    }
    fx_forward_xy<P, GEN>(m, t, e_first, E, gy, A, sl, gkappa ? x : nullptr, AX, slx);
    const int w = threadIdx.x, lez = w / Q2, g01 = w % Q2;
    const bool az = w < E * Q2 && e_first + lez < m.nel;
    long long Tz[3][N];
    int sline = 0, sg = 0;
    unsigned long long accT = 0;
    if (az) {
      const int64_t e = e_first + lez;
      const FxScales sc = fx_fwd_scales(sl + lez * kFxSlots, S);
      sg = sc.sg;
      long long v[3][Q], u[MASS ? Q : 1];
      int ps[Q], pm[MASS ? Q : 1];
      fx_line_gradient<P, MASS>(t, A + (size_t)lez * L::PER_ELEM + L::A1, g01, kFxTop - sl[lez * kFxSlots + 2], v,
                                u);
      fx_line_D<P, MASS>(reinterpret_cast<const long long*>(Dq) + e * 6 * Q3, lor_d_scales(Dq, m.nel * Q3) + e * Q3,
                         MASS ? Mq + e * Q3 : nullptr, g01, S, v, u, ps, pm);
      if (gkappa) {
        const int sgx = fx_fwd_scales(slx + lez * kFxSlots, S).sg;
        long long gxl[3][Q];
        fx_line_gradient<P, false>(t, AX + (size_t)lez * L::PER_ELEM + L::A1, g01, kFxTop - slx[lez * kFxSlots + 2],
                                   gxl, nullptr);
#pragma unroll
        for (int g2 = 0; g2 < Q; ++g2) {
          // grad(x) . (D grad(gy)) with both 3-vectors renormalised to 57 bits
          unsigned long long ax = 0, av = 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            fx_or(ax, gxl[c][g2]);
            fx_or(av, v[c][g2]);
          }
          const int shx = kFxTop - fx_bits(ax), shv = kFxTop - fx_bits(av);
          FAcc d = fx_acc();
#pragma unroll
          for (int c = 0; c < 3; ++c)
            fx_mac(d, fx_x(fx_shift(gxl[c][g2], shx)), fx_c(fx_shift(v[c][g2], shv)));
          const int pt = g01 + Q2 * g2;
          const int scale = (sgx + shx) + (sg + ps[g2] + shv) - kFxMacShift;
          const double tv = (ax && av && ps[g2] != INT_MAX) ? fx_to_double(fx_res(d), scale) : 0.0;
          gkappa[e * Q3 + pt] = tv / kappa[e * Q3 + pt];
        }
      }
      if (gx) {
        sline = fx_line_align<P, MASS>(v, u, ps, pm);
        accT = fx_line_transpose_z<P, MASS>(t, v, u, Tz);
      }
    }
    if (gx) fx_transposed<P, GEN>(m, t, S, e_first, E, A, sl, sg, az, lez, g01, sline, accT, Tz, gx);
    __syncthreads();
  }
}

template <int P, bool MASS, bool GEN>
cudaError_t backward_fx_p(const LorMesh& m, const LorTables& T, const double* Dq, const double* Mq,
                          const double* kappa, const double* x, const double* gy, double* gx, double* gk,
                          cudaStream_t s) {
  using Z = Sz<P>;
  using L = Lay<P, double>;
  const size_t bytes = sizeof(long long) * (Z::TABLES + 2 * (size_t)kFxEB<P> * L::PER_ELEM);
  static unsigned mask = 0;
  cudaError_t err = configure(k_apply_backward_fx<P, MASS, GEN>, bytes, &mask);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (m.nel + kFxEB<P> - 1) / kFxEB<P>;
  k_apply_backward_fx<P, MASS, GEN><<<(unsigned)blocks, kFxTB<P>, bytes, s>>>(m, T, Dq, Mq, kappa, x, gy, gx, gk);
  lor_count_launch();
  return cudaGetLastError();
}

}  // namespace

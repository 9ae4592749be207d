// fixed_point_metric.cuh -- the metric adj(J^T J) and det J of a trilinear
// map at one point in 64-bit fixed point (fixed_point.cuh), for the operator
// setup (k_geom.cu) and the FP64 LOR assembly (k_assemble_impl.cuh).
#pragma once

#include <climits>

#include "fixed_point.cuh"

// -X as a split with a non-positive low part (-h, -l): the multiply-add's
// identity X C = Xh Ch 2^56 + (Xh Cl + Xl Ch) 2^28 + Xl Cl holds for any
// split with |Xl| < 2^28, and the dropped |Xl Cl| / 2^56 stays below one unit
__device__ __forceinline__ Fx fx_neg(Fx x) { return Fx{-x.h, -x.l}; }

// The metric of a trilinear map at one point from its Jacobian columns c_d
// in fixed point (C[d][k], column d at scale s_d, |C| <= 2^57): the adjugate
// rows r_a = c_b x c_c ((a, b, c) cyclic), adj(J^T J)_ab = r_a . r_b (pair
// order 00, 01, 02, 11, 12, 22) and det J = c_0 . r_0.  Formed this way (not
// from M = J^T J, whose cofactors cancel to O(eps cond(J)^2)) the error stays
// O(eps cond(J)).  Each r_a is renormalised to 58 bits on its own (a short
// one, from nearly parallel columns, keeps its relative precision); the six
// adj(M) entries are then aligned to one scale sA with the largest at 58
// bits; det J keeps its full width at scale sdet.
struct FxMetric {
  Fx A[6];      // adj(M)_ab at scale sA, the largest at 58 bits
  int sA;
  double detM;  // det M = (det J)^2
};
__device__ __forceinline__ void fx_metric(const Fx (&C)[3][3], const int (&sc)[3], FxMetric& out) {
  long long R[3][3];
  int sR[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    unsigned long long o = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      FAcc t = fx_acc();
      fx_mac(t, C[b][k1], C[c][k2]);
      fx_mac(t, fx_neg(C[b][k2]), C[c][k1]);
      R[a][k] = fx_res(t);  // at most 2^59, scale s_b + s_c - 56
      fx_or(o, R[a][k]);
    }
    const int d = o ? 58 - fx_bits(o) : 0;  // -2 <= d <= 58
#pragma unroll
    for (int k = 0; k < 3; ++k) R[a][k] = fx_rescale(R[a][k], d);
    sR[a] = sc[b] + sc[c] - kFxMacShift + d;
  }
  Fx Rx[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) Rx[a][k] = fx_split(R[a][k]);
  // det J = c_0 . r_0 (at most 3 2^59), squared in FP64
  {
    FAcc t = fx_acc();
#pragma unroll
    for (int k = 0; k < 3; ++k) fx_mac(t, C[0][k], Rx[0][k]);
    const double dj = fx_to_double(fx_res(t), sc[0] + sR[0] - kFxMacShift);
    out.detM = dj * dj;
  }
  // adj(M)_ab = r_a . r_b (at most 3 2^60), aligned to the coarsest scale, then to 58 bits
  constexpr int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {0, 1, 2, 1, 2, 2};
  long long A[6];
  int smin = INT_MAX;
#pragma unroll
  for (int ab = 0; ab < 6; ++ab) {
    FAcc t = fx_acc();
#pragma unroll
    for (int k = 0; k < 3; ++k) fx_mac(t, Rx[PA[ab]][k], Rx[PB[ab]][k]);
    A[ab] = fx_res(t);
    smin = min(smin, sR[PA[ab]] + sR[PB[ab]]);
  }
  unsigned long long o = 0;
#pragma unroll
  for (int ab = 0; ab < 6; ++ab) {
    A[ab] = fx_shift(A[ab], -(sR[PA[ab]] + sR[PB[ab]] - smin));
    fx_or(o, A[ab]);
  }
  const int d = o ? 58 - fx_bits(o) : 0;
#pragma unroll
  for (int ab = 0; ab < 6; ++ab) out.A[ab] = fx_split(fx_shift(A[ab], d));
  out.sA = smin - kFxMacShift + d;
}

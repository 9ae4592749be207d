// k_assemble_impl.cuh -- Step S1.2 / A1 + A4: batched LOR matrix assembly
// (kernel template; instantiated without the reaction term in k_assemble.cu
// and with it in k_assemble_mass.cu).
//
// One CTA per macro element or a few (a high-order element split at the
// Gauss-Lobatto points into p^3 sub-hexes, Section 2.1).  The paper's A1 has
// one block per macro element and one thread per sub-element.  Here the
// FP32 values and the FP64 values at p = 1 follow that form (k_assemble); the
// FP64 values from p = 2 give each sub-hex 8 threads, one per Gauss point of
// the 2x2x2 rule and then one per row of its block (k_assemble_x8).  Either
// forms the sub-hex's 8x8 stiffness block by 2x2x2 Gauss quadrature on the
// sub-hex's trilinear map with the sub-hex coefficient kappa_s (the
// Gauss-weight average of kappa over the high-order Gauss points inside the
// sub-hex), then adds the entries straight into the CSR values at positions
// computed in closed form (no macro-element sparse block is stored), with
// FP64/FP32 atomics for the entries shared between sub-hexes.  Rows and
// columns of essential DOFs are skipped and their diagonal set to 1 by the
// same kernel (A4), so elimination costs no extra pass.
//
// Reaction term (definite Helmholtz, Section 4.1): the block gains beta_s
// times the sub-hex's trilinear mass matrix by the same 2x2x2 Gauss rule; in
// the modal basis that is 3^{-(|m|+|n|)/2} times the Walsh transform of
// W(g) = beta_s detJ_sub(g) at m xor n, added before the Hadamard sandwich.
//
// Geometry: the sub-hex map is the element's trilinear map restricted to the
// sub-box, so J_sub(tau) = J_e(xi(tau)) diag(r_a, r_b, r_c) with r the half
// widths of the GLL intervals; only the element Jacobian columns (bilinear in
// the two other coordinates) are evaluated, in FP64.  With V = r_a r_b r_c
// and M = J_e^T J_e,
//   detJ_sub J_sub^-1 J_sub^-T = adj(J_sub^T J_sub) / detJ_sub
//                             = V / (r_a r_b) adj(M)_ab / detJ_e,
// where adj(M)_ab = A_a . A_b for the adjugate rows A_a = c_b x c_c of J_e
// and detJ_e = |c_0 . A_0| (formed this way the error is O(eps cond(J_e));
// M's cofactors would lose O(eps cond(J_e)^2) on stretched elements).  In
// the FP64 values from p = 2 these products run in 64-bit fixed point on the
// integer pipe (fixed_point_metric.cuh): the column tables are converted once
// per element, one scale per table, and the rows and adj(M) are renormalised
// per Gauss point; only 1/detJ_e (range-reduced reciprocal square root of
// (detJ_e)^2, as in the setup) and the kappa_s averages stay FP64.  The 48
// metric values and 8 mass weights of a sub-hex then enter the block algebra
// as integers on one scale.
#pragma once

#include "fixed_point_metric.cuh"
#include "lor_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// Sub-hex stiffness block in the modal basis.
//
// On the sub-hex reference cube tau in [-1,1]^3 the trilinear nodal basis is
// phi_i = prod_k l_{i_k}(tau_k), l_0 = (1 - t)/2, l_1 = (1 + t)/2.  In the
// modal basis psi_m = prod_k psi_{m_k}(tau_k), psi_0 = 1, psi_1 = t, one has
// phi = (1/8) H psi with H_im = prod_k s(i_k)^{m_k}, s(0) = -1, s(1) = +1.
// At the 2x2x2 Gauss points tau_k = eps_k / sqrt(3), eps_k = +-1,
//   d_a psi_m = [m_a = 1] prod_{k != a} (eps_k / sqrt(3))^{m_k},
// so the modal stiffness
//   Kt_mn = sum_g sum_ab G^ab(g) d_a psi_m(g) d_b psi_n(g)
//         = sum_{a in m} sum_{b in n} 3^{-(|m|+|n|-2)/2} Ghat^ab(w(m,n,a,b)),
// where Ghat^ab is the Walsh-Hadamard transform of G^ab over the 8 points,
//   Ghat(w) = sum_g G(g) prod_k eps_k^{w_k},  w = (m without a) xor (n without b).
// The nodal block is K = H Kt H^T / 64, applied axis by axis.  Work per
// sub-hex: 6 x 24 additions (transforms), the 84 terms of Kt, about 200
// additions (H . H^T on the 36 symmetric entries), instead of 8 x 180
// operations for the nodal formula at each Gauss point; in the FP64 kernel
// the additions run in exact 64-bit fixed point (below).
// ---------------------------------------------------------------------------
__device__ __forceinline__ constexpr int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }
__device__ __forceinline__ constexpr int pair_index(int a, int b) {  // (00,01,02,11,12,22)
  return a <= b ? (a == 0 ? b : a == 1 ? 2 + b : 5) : (b == 0 ? a : b == 1 ? 2 + a : 5);
}
__device__ __forceinline__ constexpr int walsh_index(int m, int n, int a, int b) {
  return (m & ~(1 << a)) ^ (n & ~(1 << b));
}
__device__ __forceinline__ constexpr double inv_sqrt3_pow(int p) {  // 3^(-p/2), p = 0..6
  return p == 0 ? 1.0
       : p == 1 ? 0.57735026918962576451
       : p == 2 ? 0.33333333333333333333
       : p == 3 ? 0.19245008972987525484
       : p == 4 ? 0.11111111111111111111
       : p == 5 ? 0.06415002990995841617
                : 0.03703703703703703704;
}
__device__ __forceinline__ constexpr int sym(int i, int j) { return i <= j ? i * 8 + j : j * 8 + i; }

// ---------------------------------------------------------------------------
// FP64 block algebra in exact 64-bit integer arithmetic.
//
// On this GPU the FP64 pipe issues 2 operations per clock per SM, 32-bit
// integer operations at least 32 times as many.  After the metric G(g) every
// step of the block is linear with coefficients +-1 (the Walsh transforms, the
// sums of the modal block, the Hadamard sandwich) except the 3^(-k/2) factors
// of the modal entries.  So the 48 metric values (and the 8 mass weights) of a
// sub-hex go to integers on one power-of-two scale, X = round(x 2^(1078 - e))
// with e the largest biased exponent among them (every |X| < 2^56).  The Walsh
// transforms (growth at most 8) and the modal sums (at most 9 terms) are then
// exact and stay below 2^62.2; the 3^(-k/2) factors are 64 x 64-bit
// fixed-point products with Q63 constants, rounded to nearest.  Before the
// sandwich (at most 64 terms per entry) the modal entries are rounded to the
// largest scale that keeps them below 2^56 (a shift of 0 to 7 bits chosen
// from their actual size, so the sandwich keeps 56 bits of the largest
// entry), the sandwich is exact, and the 36 nodal entries return to FP64
// correctly rounded.  The roundings are those of the input conversion, the
// products, the one shift and the output conversion: in a CPU emulation on
// random metrics the result is within 9e-16 of the exact block (relative to
// the row maximum), against 1.7e-15 for the same steps in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long to_fix(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7FF;
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int r = emax - e - 3;  // >= -3 since e <= emax
  const int rr = r < 1 ? 1 : (r > 63 ? 63 : r);
  const unsigned long long X = r <= 0 ? mant << (-r) : (mant + (1ull << (rr - 1))) >> rr;
  const long long sgn = (long long)b >> 63;  // 0 or -1
  return e == 0 ? 0 : ((long long)X ^ sgn) - sgn;
}
// X 2^-scale in FP64, correctly rounded (X 2^-scale is a normal number
// here).  The int64 conversion issues on the FP64 pipe (about a sixth of the
// kernel's FP64 pipe time at p = 4); an integer-only conversion measured
// slower: the kernel is latency-bound and the longer dependency chain cost
// more than the pipe time it saved.
__device__ __forceinline__ double from_fix(long long X, int scale) {
  const double d = __ll2double_rn(X);
  return X == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(d) - ((long long)scale << 52));
}
// round(X C / 2^63) for a Q63 constant 0 <= C < 2^63
__device__ __forceinline__ long long fix_mul(long long X, long long C) {
  const long long hi = __mul64hi(X, C);  // floor(X C / 2^64)
  const unsigned long long lo = (unsigned long long)X * (unsigned long long)C;
  return (hi << 1) + (long long)(lo >> 63) + (long long)((lo >> 62) & 1);
}
__device__ __forceinline__ constexpr long long q63(int k) {  // 3^(-k/2) in Q63, k >= 1
  return (long long)(inv_sqrt3_pow(k) * 9223372036854775808.0);
}

// v(w) = sum_g v(g) prod_k eps_k^{w_k}; the three butterfly stages commute,
// stage FIRST runs first.  For a diagonal metric entry G^{aa} only the
// outputs with bit a clear are used later, so with FIRST = a the whole
// bit-a-set half is dead after the first stage and the compiler drops it.
template <typename VT, int FIRST>
__device__ __forceinline__ void walsh8(VT* v) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int k = s == 0 ? FIRST : (s == 1 ? (FIRST == 0 ? 1 : 0) : (FIRST == 2 ? 1 : 2));
#pragma unroll
    for (int g = 0; g < 8; ++g)
      if (!((g >> k) & 1)) {
        const VT lo = v[g], hi = v[g | (1 << k)];
        v[g] = lo + hi;
        v[g | (1 << k)] = hi - lo;
      }
  }
}

// K <- (H_k (x) H_k) K for axis k, on a symmetric 8x8 matrix stored at
// K[sym(i,j)]; H_k maps (m_k = 0, m_k = 1) to (i_k = 0: a - b, i_k = 1: a + b).
// Work per 2x2 block of the axis (rows i0, i1 = i0 | bit, columns j0, j1):
// off-diagonal blocks 8 additions for 4 outputs; a diagonal block (i0 = j0,
// symmetric input a, b, b, d) needs only a - 2b + d, a - d and a + 2b + d.
template <typename VT, int k>
__device__ __forceinline__ void hadamard_axis(VT* K) {
  constexpr int bit = 1 << k;
  VT out[64];
#pragma unroll
  for (int i0 = 0; i0 < 8; ++i0) {
    if (i0 & bit) continue;
#pragma unroll
    for (int j0 = i0; j0 < 8; ++j0) {
      if (j0 & bit) continue;
      const int i1 = i0 | bit, j1 = j0 | bit;
      if (i0 == j0) {
        const VT a = K[sym(i0, i0)], b = K[sym(i0, i1)], d = K[sym(i1, i1)];
        const VT t = a + d;
        out[sym(i0, i0)] = t - (VT)2 * b;
        out[sym(i1, i1)] = t + (VT)2 * b;
        out[sym(i0, i1)] = a - d;
      } else {
        const VT a = K[sym(i0, j0)], b = K[sym(i0, j1)], c = K[sym(i1, j0)], d = K[sym(i1, j1)];
        const VT u0 = a - c, u1 = a + c, v0 = b - d, v1 = b + d;
        out[sym(i0, j0)] = u0 - v0;
        out[sym(i0, j1)] = u0 + v0;
        out[sym(i1, j0)] = u1 - v1;
        out[sym(i1, j1)] = u1 + v1;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = i; j < 8; ++j) K[sym(i, j)] = out[sym(i, j)];
}

// The FP64 sub-hex block from its metric X[ab][g] (F_ab and 1/64 folded in)
// and mass weights Xw[g] in fixed point, all below 2^56 at one scale (real
// value = X 2^-scale): Walsh transforms, modal block, Hadamard sandwich, in
// the fixed point described above; K receives the 36 nodal entries in FP64.
template <bool MASS>
__device__ __forceinline__ void fix_block_x(long long (&X)[6][8], long long* Xw, int scale_in, double* K) {
  walsh8<long long, 0>(X[0]);
  walsh8<long long, 0>(X[1]);
  walsh8<long long, 0>(X[2]);
  walsh8<long long, 1>(X[3]);
  walsh8<long long, 0>(X[4]);
  walsh8<long long, 2>(X[5]);
  long long Kf[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) Kf[i] = 0;
#pragma unroll
  for (int mm = 1; mm < 8; ++mm)
#pragma unroll
    for (int nn = mm; nn < 8; ++nn) {
      long long acc = 0;
#pragma unroll
      for (int aa = 0; aa < 3; ++aa)
        if ((mm >> aa) & 1)
#pragma unroll
          for (int bb = 0; bb < 3; ++bb)
            if ((nn >> bb) & 1) acc += X[pair_index(aa, bb)][walsh_index(mm, nn, aa, bb)];
      const int k = popc3(mm) + popc3(nn) - 2;
      Kf[sym(mm, nn)] = k > 0 ? fix_mul(acc, q63(k)) : acc;
    }
  if constexpr (MASS) {
    walsh8<long long, 0>(Xw);
#pragma unroll
    for (int mm = 0; mm < 8; ++mm)
#pragma unroll
      for (int nn = mm; nn < 8; ++nn) {
        const int k = popc3(mm) + popc3(nn);
        Kf[sym(mm, nn)] += k > 0 ? fix_mul(Xw[mm ^ nn], q63(k)) : Xw[mm ^ nn];
      }
  }
  // the shift that brings the largest modal entry below 2^56 (its bit length
  // from the high words; a negative value's ones' complement may be one short
  // at an exact power of two, which the sandwich's 2^62 bound still covers)
  unsigned hacc = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = i; j < 8; ++j) {
      const int hi = (int)(Kf[sym(i, j)] >> 32);
      hacc |= (unsigned)(hi ^ (hi >> 31));
    }
  const int bits = hacc ? 64 - __clz((int)hacc) : 32;
  const int sft = bits > 56 ? bits - 56 : 0;
  const long long half = sft ? (1ll << (sft - 1)) : 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = i; j < 8; ++j) Kf[sym(i, j)] = (Kf[sym(i, j)] + half) >> sft;
  hadamard_axis<long long, 0>(Kf);
  hadamard_axis<long long, 1>(Kf);
  hadamard_axis<long long, 2>(Kf);
  const int scale = scale_in - sft;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = i; j < 8; ++j) K[sym(i, j)] = from_fix(Kf[sym(i, j)], scale);
}
// The same from the metric in FP64: converted with the sub-hex's largest
// exponent (X < 2^56 at scale 1078 - emax).
template <bool MASS>
__device__ __forceinline__ void fix_block(const double (&G)[6][8], const double* W, double* K) {
  unsigned hmax = 0;
#pragma unroll
  for (int ab = 0; ab < 6; ++ab)
#pragma unroll
    for (int g = 0; g < 8; ++g) hmax = max(hmax, (unsigned)__double2hiint(G[ab][g]) & 0x7FF00000u);
  if constexpr (MASS)
#pragma unroll
    for (int g = 0; g < 8; ++g) hmax = max(hmax, (unsigned)__double2hiint(W[g]) & 0x7FF00000u);
  const int emax = (int)(hmax >> 20);
  long long X[6][8], Xw[MASS ? 8 : 1];
#pragma unroll
  for (int ab = 0; ab < 6; ++ab)
#pragma unroll
    for (int g = 0; g < 8; ++g) X[ab][g] = to_fix(G[ab][g], emax);
  if constexpr (MASS)
#pragma unroll
    for (int g = 0; g < 8; ++g) Xw[g] = to_fix(W[g], emax);
  fix_block_x<MASS>(X, Xw, 1078 - emax, K);
}

template <int P>
constexpr int kElemsPerCta = P * P * P >= 64 ? 1 : 64 / (P * P * P);
template <int P>
constexpr int kAsmThreads = P * P * P >= 64 ? (P * P * P >= 256 ? 256 : ((P * P * P + 31) / 32) * 32)
                                            : ((kElemsPerCta<P> * P * P * P + 31) / 32) * 32;

// FP64 (this kernel's FP64 form serves p = 1; from p = 2 k_assemble_x8
// below): 640 threads' worth of CTAs per SM, the measured best with the
// metric in FP64 (0.278 ms against 0.300 ms at 128 registers, p = 4).
constexpr int kAsmThreadBudget = 640;
template <int P, typename VT>
constexpr int kAsmMinBlocks =
    sizeof(VT) == sizeof(double) ? (kAsmThreadBudget / kAsmThreads<P> > 1 ? kAsmThreadBudget / kAsmThreads<P> : 1) : 1;

template <typename VT>
__device__ __forceinline__ void atomic_add(VT* p, VT v) { atomicAdd(p, v); }

template <int P, typename VT, bool MASS, bool GEN>
__global__ void __launch_bounds__(kAsmThreads<P>, kAsmMinBlocks<P, VT>) k_assemble(LorMesh m, LorTables T,
                                                             const double* __restrict__ kappa,
                                                             const double* __restrict__ beta,
                                                             VT* __restrict__ vals) {
  constexpr int Q = P + 2, Q3 = Q * Q * Q, P3 = P * P * P, L = 2 * P, EPB = kElemsPerCta<P>;
  constexpr int TAB = 3 * L * L * 3;  // three Jacobian-column tables per element
  constexpr bool F32 = sizeof(VT) == sizeof(float);
  __shared__ double Ehalf[EPB][36];
  __shared__ double tab[EPB][TAB];
  __shared__ float tabf[F32 ? EPB : 1][F32 ? TAB : 1];
  __shared__ double sl0[L], sl1[L];
  if (threadIdx.x < L) {
    sl0[threadIdx.x] = T.sub_l0[threadIdx.x];
    sl1[threadIdx.x] = T.sub_l1[threadIdx.x];
  }
  __syncthreads();
  const int64_t e_first = (int64_t)blockIdx.x * EPB;
  // Jacobian columns of each element at the sub-hex Gauss coordinates (FP64;
  // the FP32 mode also keeps a rounded copy, converted once per element:
  // conversions share the FP64 pipe on this GPU).
  for (int le = 0; le < EPB; ++le) {
    const int64_t e = e_first + le;
    if (e < m.nel) lor_jacobian_columns(m, e, sl0, sl1, L, Ehalf[le], tab[le]);
  }
  if constexpr (F32) {
    for (int i = threadIdx.x; i < EPB * TAB; i += blockDim.x) tabf[i / TAB][i % TAB] = (float)tab[i / TAB][i % TAB];
    __syncthreads();
  }
  const int nwork = EPB * P3;
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    const int le = w / P3, s = w % P3;
    const int64_t e = e_first + le;
    if (e >= m.nel) break;
    const int a = s % P, b = (s / P) % P, c = s / (P * P);

    // kappa_s (and beta_s): Gauss-weight averages over the high-order points in the sub-hex
    double ks = 0.0, bs = 0.0;
    for (int g2 = T.bin_first[c]; g2 < T.bin_first[c] + T.bin_count[c]; ++g2)
      for (int g1 = T.bin_first[b]; g1 < T.bin_first[b] + T.bin_count[b]; ++g1) {
        const double w12 = T.bin_w[g1] * T.bin_w[g2];
        for (int g0 = T.bin_first[a]; g0 < T.bin_first[a] + T.bin_count[a]; ++g0) {
          const double w = w12 * T.bin_w[g0];
          const int64_t pt = e * Q3 + g0 + Q * (g1 + Q * g2);
          ks += w * kappa[pt];
          if constexpr (MASS) bs += w * beta[pt];
        }
      }

    // G_sub^{ab}(g) = F_ab adj(M)_ab / det_e, F_ab = kappa_s (r_a r_b r_c) / (r_a r_b) / 64
    // (the 1/64 of the modal-to-nodal transform folded in); in FP32 from the
    // adjugate rows A_a of J_e (A_a . A_b = adj(M)_ab).
    VT G[F32 ? 6 : 1][F32 ? 8 : 1];  // FP32: the metric (pair order 00, 01, 02, 11, 12, 22)
    VT W[(MASS && F32) ? 8 : 1];      // FP32 reaction: W(g) = beta_s detJ_sub(g) / 64 (Gauss weights 1)
    const int u0a = 2 * a, u1a = 2 * b, u2a = 2 * c;
    // FP64 (p = 1): the metric in FP64 from the adjugate rows of J_e and
    // 1/det J_e by the range-reduced reciprocal square root of (det J_e)^2
    double Gd[F32 ? 1 : 6][F32 ? 1 : 8];
    double Wd[(MASS && !F32) ? 8 : 1];
    if constexpr (!F32) {
      const double ra = T.sub_r[a], rb = T.sub_r[b], rc = T.sub_r[c];
      const double k64 = ks * (1.0 / 64.0);
      const double FF[6] = {k64 * rb * rc * T.sub_rinv[a], k64 * rc, k64 * rb,
                            k64 * ra * rc * T.sub_rinv[b], k64 * ra, k64 * ra * rb * T.sub_rinv[c]};
      const double bR = MASS ? bs * (1.0 / 64.0) * ra * rb * rc : 0.0;
      const double* t0 = tab[le];
      const double* t1 = tab[le] + L * L * 3;
      const double* t2 = tab[le] + 2 * L * L * 3;
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const int u0 = u0a + (g & 1), u1 = u1a + ((g >> 1) & 1), u2 = u2a + (g >> 2);
        const double* c0 = t0 + 3 * (u1 + L * u2);
        const double* c1 = t1 + 3 * (u0 + L * u2);
        const double* c2 = t2 + 3 * (u0 + L * u1);
        double R[3][3];
        lor_cross(c1, c2, R[0]);
        lor_cross(c2, c0, R[1]);
        lor_cross(c0, c1, R[2]);
        const double dj = c0[0] * R[0][0] + c0[1] * R[0][1] + c0[2] * R[0][2];
        const double detM = dj * dj;
        const double r = lor_rsqrt(detM);  // 1 / det J_e
        if constexpr (MASS) Wd[g] = bR * (detM * r);
#pragma unroll
        for (int ab = 0; ab < 6; ++ab) {
          const int pa = ab < 3 ? 0 : ab < 5 ? 1 : 2, pb = ab < 3 ? ab : ab < 5 ? ab - 2 : 2;
          Gd[ab][g] = (FF[ab] * r) * (R[pa][0] * R[pb][0] + R[pa][1] * R[pb][1] + R[pa][2] * R[pb][2]);
        }
      }
    } else {
      // FP64: the first adjugate row and the determinant; FP32: the rest.
      const float ra = (float)T.sub_r[a], rb = (float)T.sub_r[b], rc = (float)T.sub_r[c];
      const float k64 = (float)ks * (1.0f / 64.0f);
      const float F00 = k64 * rb * rc / ra, F01 = k64 * rc, F02 = k64 * rb;
      const float F11 = k64 * ra * rc / rb, F12 = k64 * ra, F22 = k64 * ra * rb / rc;
      const float bR = MASS ? (float)bs * (1.0f / 64.0f) * ra * rb * rc : 0.0f;
      const double* t0 = tab[le];
      const double* t1 = tab[le] + L * L * 3;
      const double* t2 = tab[le] + 2 * L * L * 3;
      const float* f0 = tabf[le];
      const float* f1 = tabf[le] + L * L * 3;
      const float* f2 = tabf[le] + 2 * L * L * 3;
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const int u0 = u0a + (g & 1), u1 = u1a + ((g >> 1) & 1), u2 = u2a + (g >> 2);
        const int o0 = 3 * (u1 + L * u2), o1 = 3 * (u0 + L * u2), o2 = 3 * (u0 + L * u1);
        double A0[3];
        lor_cross(t1 + o1, t2 + o2, A0);
        const double det = t0[o0] * A0[0] + t0[o0 + 1] * A0[1] + t0[o0 + 2] * A0[2];
        const float detf = (float)det;
        const float r = 1.0f / detf;
        if constexpr (MASS) W[g] = (VT)(bR * detf);
        const float* c0 = f0 + o0;
        const float* c1 = f1 + o1;
        const float* c2 = f2 + o2;
        float A[3][3];
        A[0][0] = c1[1] * c2[2] - c1[2] * c2[1];
        A[0][1] = c1[2] * c2[0] - c1[0] * c2[2];
        A[0][2] = c1[0] * c2[1] - c1[1] * c2[0];
        A[1][0] = c2[1] * c0[2] - c2[2] * c0[1];
        A[1][1] = c2[2] * c0[0] - c2[0] * c0[2];
        A[1][2] = c2[0] * c0[1] - c2[1] * c0[0];
        A[2][0] = c0[1] * c1[2] - c0[2] * c1[1];
        A[2][1] = c0[2] * c1[0] - c0[0] * c1[2];
        A[2][2] = c0[0] * c1[1] - c0[1] * c1[0];
#pragma unroll
        for (int ab = 0; ab < 6; ++ab) {
          const int pa = ab < 3 ? 0 : ab < 5 ? 1 : 2, pb = ab < 3 ? ab : ab < 5 ? ab - 2 : 2;
          const float Fab = ab == 0 ? F00 : ab == 1 ? F01 : ab == 2 ? F02 : ab == 3 ? F11 : ab == 4 ? F12 : F22;
          G[ab][g] = (VT)((Fab * r) * (A[pa][0] * A[pb][0] + A[pa][1] * A[pb][1] + A[pa][2] * A[pb][2]));
        }
      }
    }
    // pair order (00, 01, 02, 11, 12, 22): diagonal entries start with their own axis
    VT K[64];  // the nodal block (symmetric entries K[sym(i, j)])
    if constexpr (F32) {
      walsh8<VT, 0>(G[0]);
      walsh8<VT, 0>(G[1]);
      walsh8<VT, 0>(G[2]);
      walsh8<VT, 1>(G[3]);
      walsh8<VT, 0>(G[4]);
      walsh8<VT, 2>(G[5]);
      if constexpr (MASS) walsh8<VT, 0>(W);
      // modal block (row/column 0 vanish: psi_0 has no gradient)
#pragma unroll
      for (int i = 0; i < 64; ++i) K[i] = (VT)0;
#pragma unroll
      for (int mm = 1; mm < 8; ++mm)
#pragma unroll
        for (int nn = mm; nn < 8; ++nn) {
          VT acc = (VT)0;
#pragma unroll
          for (int aa = 0; aa < 3; ++aa)
            if ((mm >> aa) & 1)
#pragma unroll
              for (int bb = 0; bb < 3; ++bb)
                if ((nn >> bb) & 1)
                  acc += (VT)inv_sqrt3_pow(popc3(mm) + popc3(nn) - 2) * G[pair_index(aa, bb)][walsh_index(mm, nn, aa, bb)];
          K[sym(mm, nn)] = acc;
        }
      if constexpr (MASS) {
        // modal mass block: sum_g W(g) psi_m(g) psi_n(g) = 3^{-(|m|+|n|)/2} What(m xor n)
#pragma unroll
        for (int mm = 0; mm < 8; ++mm)
#pragma unroll
          for (int nn = mm; nn < 8; ++nn) K[sym(mm, nn)] += (VT)inv_sqrt3_pow(popc3(mm) + popc3(nn)) * W[mm ^ nn];
      }
      hadamard_axis<VT, 0>(K);
      hadamard_axis<VT, 1>(K);
      hadamard_axis<VT, 2>(K);
    } else {
      // FP64: the same linear steps in 64-bit fixed point (see fix_block_x)
      fix_block<MASS>(Gd, Wd, K);
    }

    // Scatter into the CSR values (closed-form positions on the structured
    // grid, binary search in the row on a general mesh), skipping essential
    // rows and columns; an essential row's diagonal is set to 1 here (every
    // DOF is a corner of some sub-hex; no atomic ever targets that row, and
    // several sub-hexes may store the same 1).
    if constexpr (GEN) {
      constexpr int N = P + 1;
      const int64_t* dm = m.edofs + e * (N * N * N);
      int64_t dv[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) dv[r] = dm[(a + (r & 1)) + N * ((b + ((r >> 1) & 1)) + N * (c + (r >> 2)))];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t rb = m.rowptr[dv[r]], re = m.rowptr[dv[r] + 1];
        if (m.ess[dv[r]]) {
          const int64_t pos = lor_find_col(m.colidx, rb, re, dv[r]);
          if (pos >= 0) vals[pos] = (VT)1;
          continue;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (m.ess[dv[t]]) continue;
          const int64_t pos = lor_find_col(m.colidx, rb, re, dv[t]);
          if (pos >= 0) atomic_add<VT>(vals + pos, K[sym(r, t)]);
        }
      }
    } else {
      const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
      const int64_t I0 = ex * P + a, J0 = ey * P + b, K0 = ez * P + c;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t I = I0 + (r & 1), J = J0 + ((r >> 1) & 1), Kk = K0 + (r >> 2);
        const int64_t base = lor_entry_pos(I, J, Kk, 0, 0, 0, m.nx, m.ny, m.nz);
        if (lor_is_essential(I, J, Kk, m.nx, m.ny, m.nz)) {
          vals[base] = (VT)1;
          continue;
        }
        const int64_t cx = lor_axis_count(I, m.nx), cy = lor_axis_count(J, m.ny);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int64_t I2 = I0 + (t & 1), J2 = J0 + ((t >> 1) & 1), K2 = K0 + (t >> 2);
          if (lor_is_essential(I2, J2, K2, m.nx, m.ny, m.nz)) continue;
          const int di = (t & 1) - (r & 1), dj = ((t >> 1) & 1) - ((r >> 1) & 1), dk = (t >> 2) - (r >> 2);
          atomic_add<VT>(vals + base + (dk * cy + dj) * cx + di, K[sym(r, t)]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 assembly from p = 2: eight threads per sub-hex.
//
// A sub-hex is handled by a group of 8 consecutive lanes of one warp.
// - Lane g forms the metric at Gauss point g (fx_metric, as in the kernel
//   above) and one term of the kappa_s average: for p >= 2 every LOR interval
//   holds one or two high-order Gauss points per axis, so a sub-hex has at
//   most 8 and lane (i0, i1, i2) takes point (first + i) of each axis' bin.
// - The group aligns its 48 metric values (and 8 mass weights) to one scale
//   (a max over its lanes) and runs the Walsh transforms across its lanes:
//   the butterfly over point bit k pairs lane g with lane g ^ 2^k, so lane w
//   ends with Ghat^{ab}(w), which it leaves in shared memory.
// - Lane m then builds row m of the modal block from shared memory, scales
//   it by the 3^(-k/2) factors, applies the column half of the Hadamard
//   sandwich in registers and the row half across the group, converts its 8
//   nodal entries to FP64 and scatters row m of the block.
// The arithmetic is fix_block_x's (exact fixed point; the block is held as
// full rows instead of its symmetric half, whose entries are the same
// integers), so the values equal the one-thread kernel's up to the
// summation order of the kappa_s average.  Per thread the state is one
// point's metric or one block row: 64 registers without spills up to p = 5,
// and twice the active warps per SM of the one-thread form (30 against 15 at
// p = 4).
// ---------------------------------------------------------------------------
template <int P>
constexpr int kX8Elems = P * P * P * 8 >= 256 ? 1 : 256 / (P * P * P * 8);
template <int P>
constexpr int kX8Threads = kX8Elems<P> * P * P * P * 8 >= 256 ? 256 : ((kX8Elems<P> * P * P * P * 8 + 31) / 32) * 32;
constexpr int kX8MinBlocks = 4;

__constant__ long long kQ63[7] = {0, q63(1), q63(2), q63(3), q63(4), q63(5), q63(6)};

__device__ __forceinline__ long long x8_walsh_step(long long v, int lane8, int bit) {
  const long long o = __shfl_xor_sync(0xffffffffu, v, bit);
  return (lane8 & bit) ? v - o : v + o;  // lane with the bit set holds hi: hi - lo; else lo + hi
}

template <int P, bool MASS, bool GEN>
__global__ void __launch_bounds__(kX8Threads<P>, kX8MinBlocks) k_assemble_x8(LorMesh m, LorTables T,
                                                                          const double* __restrict__ kappa,
                                                                          const double* __restrict__ beta,
                                                                          double* __restrict__ vals) {
  constexpr int Q = P + 2, Q3 = Q * Q * Q, P3 = P * P * P, L = 2 * P, EPB = kX8Elems<P>, NT = kX8Threads<P>;
  constexpr int CT = L * L * 3, TAB = 3 * CT;  // one / three Jacobian-column tables per element
  constexpr int NG = NT / 8, NE = MASS ? 7 : 6;
  // a group's stride in Gh (words, 8 bytes).  Without the reaction term GS = 56 = 8
  // (mod 16): the two groups of a half-warp (one phase of a 64-bit access) fall in
  // opposite halves of the banks.  With it GS = 64 puts them on the same banks.
  constexpr int GS = NE * 8 + 8;
  constexpr int ZW = NE * 8;      // a zero word in each group's block (the terms a row does not have)
  __shared__ double Ehalf[EPB][36];
  // the Jacobian columns in FP64, then (in place) as packed fixed-point
  // words at one scale per column table (1079 - cexp)
  __shared__ long long tabx[EPB][TAB];
  __shared__ int cexp[EPB][3];
  __shared__ double sl0[L], sl1[L];
  __shared__ long long Gh[NG * GS];  // per group: Ghat^{ab}(w) [ab][w], then What(w)
  if (threadIdx.x < L) {
    sl0[threadIdx.x] = T.sub_l0[threadIdx.x];
    sl1[threadIdx.x] = T.sub_l1[threadIdx.x];
  }
  if (threadIdx.x < NG) Gh[threadIdx.x * GS + ZW] = 0;
  for (int i = threadIdx.x; i < EPB * 3; i += NT) cexp[i / 3][i % 3] = 0;
  const int64_t e_first = (int64_t)blockIdx.x * EPB;
  // Jacobian columns of the CTA's elements at the sub-hex Gauss coordinates,
  // with each table's largest exponent, then the conversion to fixed point in
  // place.  With several elements per CTA (p = 2) the half edge vectors and
  // then every entry are formed by threads of their own (the values of
  // lor_jacobian_columns; 1.05 against 0.91 GDOF/s at ~20M DOFs); with one,
  // lor_jacobian_columns measured faster (0.239 against 0.244 ms, p = 4).
  if constexpr (EPB > 1) {
    for (int i = threadIdx.x; i < EPB * 36; i += NT) {
      const int le = i / 36, idx = i % 36;
      const int64_t e = e_first + le;
      if (e >= m.nel) continue;
      const int d = idx / 12, pair = (idx / 3) % 4, comp = idx % 3;
      const int o0 = pair & 1, o1 = pair >> 1;
      const int lo = d == 0 ? 2 * o0 + 4 * o1 : d == 1 ? o0 + 4 * o1 : o0 + 2 * o1;
      double A[3], Bv[3];
      lor_element_corner(m, e, lo, A);
      lor_element_corner(m, e, lo + (1 << d), Bv);
      Ehalf[le][idx] = 0.5 * (Bv[comp] - A[comp]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < EPB * TAB; i += NT) {
      const int le = i / TAB, r = i % TAB;
      if (e_first + le >= m.nel) continue;
      const int d = r / CT, w = r % CT;  // w = 3 (u + L v) + comp
      const int comp = w % 3, u = (w / 3) % L, v = w / (3 * L);
      const double* E = Ehalf[le] + d * 12 + comp;
      const double ea = sl0[u] * E[0] + sl1[u] * E[3];  // v-bit 0 edges, interpolated in u
      const double eb = sl0[u] * E[6] + sl1[u] * E[9];  // v-bit 1 edges
      const double x = sl0[v] * ea + sl1[v] * eb;
      tabx[le][r] = __double_as_longlong(x);
      atomicMax(&cexp[le][d], fx_expo(x));
    }
    __syncthreads();
  } else {
    __syncthreads();
    if (e_first < m.nel) lor_jacobian_columns(m, e_first, sl0, sl1, L, Ehalf[0], reinterpret_cast<double*>(tabx[0]));
    for (int i = threadIdx.x; i < TAB; i += NT) atomicMax(&cexp[0][i / CT], fx_expo(__longlong_as_double(tabx[0][i])));
    __syncthreads();
  }
  for (int i = threadIdx.x; i < EPB * TAB; i += NT) {
    const double v = __longlong_as_double(tabx[i / TAB][i % TAB]);
    tabx[i / TAB][i % TAB] = fx_pack(fx_from_double(v, cexp[i / TAB][(i % TAB) / CT]));
  }
  __syncthreads();

  const int lane8 = threadIdx.x & 7, grp = threadIdx.x >> 3;
  long long* gh = Gh + grp * GS;
  constexpr int NSUB = EPB * P3;
  // every thread runs every pass (the shuffles take whole warps); a group
  // past the CTA's sub-hexes or elements computes on sub-hex 0 and stores nothing
  for (int base = 0; base < NSUB; base += NG) {
    const int sidx = base + grp;
    const int le0 = sidx / P3;
    const bool live = sidx < NSUB && e_first + le0 < m.nel;
    const int le = live ? le0 : 0, s = live ? sidx % P3 : 0;
    const int64_t e = e_first + le;
    const int a = s % P, b = (s / P) % P, c = s / (P * P);

    // kappa_s (and beta_s): lane (i0, i1, i2) holds one Gauss-weighted term
    double kw = 0.0, bw = 0.0;
    {
      const int i0 = lane8 & 1, i1 = (lane8 >> 1) & 1, i2 = lane8 >> 2;
      if (i0 < T.bin_count[a] && i1 < T.bin_count[b] && i2 < T.bin_count[c]) {
        const int g0 = T.bin_first[a] + i0, g1 = T.bin_first[b] + i1, g2 = T.bin_first[c] + i2;
        const double w = (T.bin_w[g1] * T.bin_w[g2]) * T.bin_w[g0];
        const int64_t pt = e * Q3 + g0 + Q * (g1 + Q * g2);
        kw = w * kappa[pt];
        if constexpr (MASS) bw = w * beta[pt];
      }
    }
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
      kw += __shfl_xor_sync(0xffffffffu, kw, bit);
      if constexpr (MASS) bw += __shfl_xor_sync(0xffffffffu, bw, bit);
    }

    // F_ab = kappa_s (r_a r_b r_c) / (r_a r_b) / 64 in fixed point: lane ab < 6
    // forms F_ab (the 1/64 goes into its scale) and the group shares them
    const double ra = T.sub_r[a], rb = T.sub_r[b], rc = T.sub_r[c];
    Fx FFx[6];
    int sF[6];
    {
      const int ab = lane8;
      const double xa = ab == 1 ? rc : (ab == 0 || ab == 2) ? rb : ra;
      const double ya = (ab == 0 || ab == 3) ? rc : ab == 5 ? rb : 1.0;
      const double za = ab == 0 ? T.sub_rinv[a] : ab == 3 ? T.sub_rinv[b] : ab == 5 ? T.sub_rinv[c] : 1.0;
      const double f = ((kw * xa) * ya) * za;
      const int ef = fx_expo(f);
      const Fx fx = fx_split(fx_from_double(f, ef));
      const int sf = 1079 - ef + 6;
      const int gb = threadIdx.x & 24;  // the group's first lane in the warp
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        FFx[k].h = __shfl_sync(0xffffffffu, fx.h, gb + k);
        FFx[k].l = __shfl_sync(0xffffffffu, fx.l, gb + k);
        sF[k] = __shfl_sync(0xffffffffu, sf, gb + k);
      }
    }
    // the metric at Gauss point g = lane8: G_ab = (F_ab r) adj(M)_ab
    long long X[6];
    const int g = lane8;
    const int u0 = 2 * a + (g & 1), u1 = 2 * b + ((g >> 1) & 1), u2 = 2 * c + (g >> 2);
    Fx C[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C[0][k] = fx_unpack(tabx[le][3 * (u1 + L * u2) + k]);
      C[1][k] = fx_unpack(tabx[le][CT + 3 * (u0 + L * u2) + k]);
      C[2][k] = fx_unpack(tabx[le][2 * CT + 3 * (u0 + L * u1) + k]);
    }
    const int scs[3] = {1079 - cexp[le][0], 1079 - cexp[le][1], 1079 - cexp[le][2]};
    FxMetric mt;
    fx_metric(C, scs, mt);
    const double r = lor_rsqrt(mt.detM);  // 1 / det J_e
    const int er = fx_expo(r);
    const Fx rx = fx_split(fx_from_double(r, er));
    const int sG = (1079 - er) - kFxMacShift + mt.sA - kFxMacShift;  // G_ab at sF[ab] + sG
#pragma unroll
    for (int ab = 0; ab < 6; ++ab) {
      FAcc f = fx_acc();
      fx_mac(f, FFx[ab], rx);
      FAcc q = fx_acc();
      fx_mac(q, fx_split(fx_res(f)), mt.A[ab]);
      X[ab] = fx_res(q);  // (F_ab r) at most 2^58, G at most 2^60
    }
    long long Xw = 0;
    int sW = 0;
    if constexpr (MASS) {
      // W = beta_s r_a r_b r_c / 64 det J_e, det J_e = det M r
      const double bR = ((bw * ra) * rb) * rc;  // the 1/64 goes into the scale
      const int eb = fx_expo(bR);
      const double dj = mt.detM * r;
      const int ej = fx_expo(dj);
      FAcc q = fx_acc();
      fx_mac(q, fx_split(fx_from_double(bR, eb)), fx_split(fx_from_double(dj, ej)));
      Xw = fx_res(q);  // at most 2^58
      sW = (1079 - eb + 6) + (1079 - ej) - kFxMacShift;
    }
    // one scale for the sub-hex: its largest value below 2^56
    int mmax = -(1 << 30);
#pragma unroll
    for (int ab = 0; ab < 6; ++ab)
      if (X[ab] != 0) mmax = max(mmax, fx_bits((unsigned long long)(X[ab] ^ (X[ab] >> 63))) - (sF[ab] + sG));
    if constexpr (MASS)
      if (Xw != 0) mmax = max(mmax, fx_bits((unsigned long long)(Xw ^ (Xw >> 63))) - sW);
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, bit));
    const int st = 56 - mmax;
#pragma unroll
    for (int ab = 0; ab < 6; ++ab) X[ab] = fx_shift(X[ab], min(st - (sF[ab] + sG), 63));
    if constexpr (MASS) Xw = fx_shift(Xw, min(st - sW, 63));

    // Walsh transforms across the group (exact: |X| < 2^56 grows to < 2^59)
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
      for (int ab = 0; ab < 6; ++ab) X[ab] = x8_walsh_step(X[ab], lane8, bit);
      if constexpr (MASS) Xw = x8_walsh_step(Xw, lane8, bit);
    }
#pragma unroll
    for (int ab = 0; ab < 6; ++ab) gh[ab * 8 + lane8] = X[ab];
    if constexpr (MASS) gh[48 + lane8] = Xw;
    __syncwarp();

    // row mm of the modal block: Kt_mn = 3^(-k/2) sum_{a in m, b in n} Ghat^{ab}((m \ a) xor (n \ b))
    const int mm = lane8, pm = popc3(mm);
    long long K[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) K[n] = 0;
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
      const bool ina = (mm >> aa) & 1;
      const int u = mm & ~(1 << aa);
#pragma unroll
      for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          if ((v >> bb) & 1) continue;
          K[v | (1 << bb)] += gh[ina ? pair_index(aa, bb) * 8 + (u ^ v) : ZW];
        }
    }
#pragma unroll
    for (int n = 1; n < 8; ++n) {
      const int k = pm + popc3(n) - 2;  // -1 only on row 0, whose sums are zero
      const long long f = fix_mul(K[n], kQ63[k > 0 ? k : 1]);
      K[n] = k > 0 ? f : K[n];
    }
    if constexpr (MASS) {
      // modal mass block: 3^{-(|m|+|n|)/2} What(m xor n)
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const int k = pm + popc3(n);
        const long long w = gh[48 + (mm ^ n)];
        const long long f = fix_mul(w, kQ63[k > 0 ? k : 1]);
        K[n] += k > 0 ? f : w;
      }
    }
    __syncwarp();  // the group's shared values are read; the next pass may overwrite them

    // the shift that brings the largest modal entry below 2^56 (as in fix_block_x)
    unsigned hacc = 0;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int hi = (int)(K[n] >> 32);
      hacc |= (unsigned)(hi ^ (hi >> 31));
    }
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) hacc |= __shfl_xor_sync(0xffffffffu, hacc, bit);
    const int bits = hacc ? 64 - __clz((int)hacc) : 32;
    const int sft = bits > 56 ? bits - 56 : 0;
    const long long half = sft ? (1ll << (sft - 1)) : 0;
#pragma unroll
    for (int n = 0; n < 8; ++n) K[n] = (K[n] + half) >> sft;
    // Hadamard sandwich K <- H Kt H^T: per axis (lo, hi) -> (lo - hi, lo + hi)
    // on the column index (in registers) and on the row index (across lanes)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int bit = 1 << k;
#pragma unroll
      for (int j0 = 0; j0 < 8; ++j0) {
        if (j0 & bit) continue;
        const long long x = K[j0], y = K[j0 | bit];
        K[j0] = x - y;
        K[j0 | bit] = x + y;
      }
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const long long o = __shfl_xor_sync(0xffffffffu, K[n], bit);
        K[n] = (mm & bit) ? o + K[n] : K[n] - o;
      }
    }
    const int scale = st - sft;
    double Kd[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) Kd[n] = from_fix(K[n], scale);
    // the essential corners of the sub-hex: lane t tests corner t, a ballot shares them
    unsigned essb = 0;
    if constexpr (!GEN) {
      const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
      const bool es = lor_is_essential(ex * P + a + (mm & 1), ey * P + b + ((mm >> 1) & 1), ez * P + c + (mm >> 2),
                                       m.nx, m.ny, m.nz);
      essb = (__ballot_sync(0xffffffffu, es) >> (threadIdx.x & 24)) & 0xffu;
    }
    if (!live) continue;

    // scatter row r = mm of the block (as the one-thread kernel, one row per lane)
    const int rr = mm;
    if constexpr (GEN) {
      constexpr int N = P + 1;
      const int64_t* dm = m.edofs + e * (N * N * N);
      int64_t dv[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) dv[t] = dm[(a + (t & 1)) + N * ((b + ((t >> 1) & 1)) + N * (c + (t >> 2)))];
      const int64_t rb0 = m.rowptr[dv[rr]], re0 = m.rowptr[dv[rr] + 1];
      if (m.ess[dv[rr]]) {
        const int64_t pos = lor_find_col(m.colidx, rb0, re0, dv[rr]);
        if (pos >= 0) vals[pos] = 1.0;
        continue;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (m.ess[dv[t]]) continue;
        const int64_t pos = lor_find_col(m.colidx, rb0, re0, dv[t]);
        if (pos >= 0) atomic_add<double>(vals + pos, Kd[t]);
      }
    } else {
      const int64_t ex = e % m.nex, ey = (e / m.nex) % m.ney, ez = e / ((int64_t)m.nex * m.ney);
      const int64_t I0 = ex * P + a, J0 = ey * P + b, K0 = ez * P + c;
      const int64_t I = I0 + (rr & 1), J = J0 + ((rr >> 1) & 1), Kk = K0 + (rr >> 2);
      const int64_t base_pos = lor_entry_pos(I, J, Kk, 0, 0, 0, m.nx, m.ny, m.nz);
      if ((essb >> rr) & 1u) {
        vals[base_pos] = 1.0;
        continue;
      }
      const int64_t cx = lor_axis_count(I, m.nx), cy = lor_axis_count(J, m.ny);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if ((essb >> t) & 1u) continue;
        const int di = (t & 1) - (rr & 1), dj = ((t >> 1) & 1) - ((rr >> 1) & 1), dk = (t >> 2) - (rr >> 2);
        atomic_add<double>(vals + base_pos + (dk * cy + dj) * cx + di, Kd[t]);
      }
    }
  }
}

template <int P, typename VT, bool MASS, bool GEN>
cudaError_t launch_assemble_p(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta, VT* vals,
                              cudaStream_t s) {
  if constexpr (sizeof(VT) == sizeof(double) && P >= 2) {
    // one lane per high-order Gauss point of a sub-hex's bins: one or two per axis
    for (int a = 0; a < P; ++a)
      if (T.bin_count[a] < 1 || T.bin_count[a] > 2) return cudaErrorInvalidValue;
    k_assemble_x8<P, MASS, GEN><<<(unsigned)((m.nel + kX8Elems<P> - 1) / kX8Elems<P>), kX8Threads<P>, 0, s>>>(
        m, T, kappa, beta, (double*)vals);
  } else {
    k_assemble<P, VT, MASS, GEN><<<(unsigned)((m.nel + kElemsPerCta<P> - 1) / kElemsPerCta<P>), kAsmThreads<P>, 0, s>>>(
        m, T, kappa, beta, vals);
  }
  lor_count_launch();
  return cudaSuccess;
}

template <typename VT, bool MASS, bool GEN>
cudaError_t assemble_dispatch(const LorMesh& m, const LorTables& T, const double* kappa, const double* beta, VT* vals,
                              cudaStream_t s) {
  switch (m.p) {
#define LOR_CASE(P) \
  case P: {                                                                  \
    const cudaError_t err = launch_assemble_p<P, VT, MASS, GEN>(m, T, kappa, beta, vals, s); \
    if (err != cudaSuccess) return err;                                      \
  } break;
    LOR_CASE(1) LOR_CASE(2) LOR_CASE(3) LOR_CASE(4) LOR_CASE(5)
    LOR_CASE(6) LOR_CASE(7) LOR_CASE(8) LOR_CASE(9) LOR_CASE(10)
#undef LOR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

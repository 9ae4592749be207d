// fixed_point.cuh -- 64-bit fixed-point values for the integer-pipe FP64
// arithmetic of the high-order operator (k_apply_fix.cuh) and the setup that
// stores its factor D in that form (k_geom.cu).
//
// A value is an int64 X with |X| <= 2^57 and a power-of-two scale s kept
// beside it (real value = X 2^-s).  For 32 x 32 -> 64 bit multiply-adds it is
// split as X = h 2^28 + l with 0 <= l < 2^28 (|h| < 2^30 for |X| <= 2^58);
// the packed form keeps h in the high and l in the low word of one 64-bit
// word.
//
// Storage of D (k_setup's output, one allocation of 6 nq doubles' worth plus
// nq int32): entries [e][c][q^3] (c = 00, 01, 02, 11, 12, 22) as packed
// int64 words, each Gauss point's six at the point's own scale (its largest
// entry at most 2^57), then the points' scales [e][q^3] as int32:
// sd = 1079 - emax (entry = X 2^-sd), INT_MAX where all six are zero.
#pragma once

#include <climits>
#include <stdint.h>

constexpr int kFxTop = 57;  // stored values: |X| <= 2^57

// X = h 2^28 + l with 0 <= l < 2^28
struct Fx {
  int h, l;
};
__device__ __forceinline__ Fx fx_split(long long X) { return Fx{(int)(X >> 28), (int)(X & 0xfffffffll)}; }
// packed word: high word h, low word l (the split of X)
__device__ __forceinline__ long long fx_pack(long long X) {
  return (long long)(((unsigned long long)(unsigned)(int)(X >> 28) << 32) | (unsigned long long)(X & 0xfffffffll));
}
__device__ __forceinline__ Fx fx_unpack(long long c) { return Fx{(int)(c >> 32), (int)(unsigned)(unsigned long long)c}; }

// biased exponent field of x (0 for zero and subnormals)
__device__ __forceinline__ int fx_expo(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// x 2^(1079 - emax), rounded to nearest, for |x| < 2^(emax - 1022): at most
// 2^57.  Zero and subnormal x give 0.
__device__ __forceinline__ long long fx_from_double(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7ff;
  const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
  const int r = emax - e - 4;  // right shift of the 53-bit significand (>= -4)
  const int rr = r < 1 ? 1 : (r > 63 ? 63 : r);
  const unsigned long long X = r <= 0 ? mant << (-r) : (r > 60 ? 0ull : (mant + (1ull << (rr - 1))) >> rr);
  const long long sgn = (long long)b >> 63;
  return e == 0 ? 0ll : ((long long)X ^ sgn) - sgn;
}

// X 2^-scale as FP64, rounded to nearest (ties away from zero); results
// below the normal range give zero, above it infinity.
__device__ __forceinline__ double fx_to_double(long long X, int scale) {
  const unsigned long long sgn = (unsigned long long)(X >> 63);
  const unsigned long long a = ((unsigned long long)X ^ sgn) - sgn;
  const int lz = __clzll((long long)a);
  const unsigned long long mm = a << (lz & 63);
  const unsigned long long mant = (mm >> 11) + ((mm >> 10) & 1ull);  // 53 bits with the leading one
  const int ex = 1085 - lz - scale;                                   // biased exponent - 1
  unsigned long long bits = ((unsigned long long)(long long)ex << 52) + mant;
  bits = ex < 0 ? 0ull : (ex >= 2046 ? 0x7ff0000000000000ull : bits);
  return X == 0 ? 0.0 : __longlong_as_double((long long)(bits | (sgn << 63)));
}

// A multiply-add's operands (data X and coefficient C: tables, D, M), both
// |.| <= 2^58, split as X = Xh 2^28 + Xl (0 <= Xl < 2^28, |Xh| < 2^30):
//   X C / 2^56 = Xh Ch + (Xh Cl + Xl Ch) / 2^28 + Xl Cl / 2^56,
// hi += Xh Ch and mid += Xh Cl + Xl Ch by 32 x 32 -> 64 bit multiply-adds
// (mad.wide.s32); the dropped Xl Cl / 2^56 is below one unit.  With at most
// 14 products (|Xh Ch| < 2^59, |Xh Cl + Xl Ch| < 2^58.6) neither accumulator
// overflows, and the result hi + mid / 2^28, rounded once, reaches up to
// 2^62: a stage's largest output keeps 58-61 bits.
using FxX = Fx;
using FxC = Fx;
constexpr int kFxMacShift = 56;  // a multiply-add's product is X C / 2^56
__device__ __forceinline__ FxX fx_x(long long X) { return fx_split(X); }
__device__ __forceinline__ FxC fx_c(long long C) { return fx_split(C); }
__device__ __forceinline__ FxC fx_c_packed(long long c) { return fx_unpack(c); }

struct FAcc {
  long long hi, mid;
};
__device__ __forceinline__ FAcc fx_acc() { return FAcc{0ll, 1ll << 27}; }  // mid's bias rounds the final shift
__device__ __forceinline__ void fx_mac(FAcc& a, FxX x, FxC c) {
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(a.hi) : "r"(x.h), "r"(c.h));
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(a.mid) : "r"(x.h), "r"(c.l));
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(a.mid) : "r"(x.l), "r"(c.h));
}
__device__ __forceinline__ long long fx_res(const FAcc& a) { return a.hi + (a.mid >> 28); }

// X 2^sh for a signed shift (left: sh <= 57 keeps |X| <= 2^57 by
// construction; right: rounded to nearest, 0 beyond 62 places)
__device__ __forceinline__ long long fx_shift(long long X, int sh) {
  if (sh >= 0) return (long long)((unsigned long long)X << sh);
  const int r = -sh;
  return r > 62 ? 0ll : (X + (1ll << (r - 1))) >> r;
}
// the same without a branch, for the renormalising loads (-6 <= sh <= 57;
// a right shift truncates: under a unit of the 57-bit result)
__device__ __forceinline__ long long fx_rescale(long long X, int sh) {
  const int l = sh > 0 ? sh : 0, r = sh > 0 ? 0 : -sh;
  return (long long)((unsigned long long)X << l) >> r;
}

// bit length of the largest |X| among the values OR-ed into acc as X ^ (X >> 63)
__device__ __forceinline__ void fx_or(unsigned long long& acc, long long X) {
  acc |= (unsigned long long)(X ^ (X >> 63));
}
__device__ __forceinline__ int fx_bits(unsigned long long acc) { return 64 - __clzll((long long)acc); }

// The scale offsets of D's points, stored after its 6 nq packed entries.
__host__ __device__ __forceinline__ int* lor_d_scales(double* Dq, int64_t nq) {
  return reinterpret_cast<int*>(Dq + 6 * nq);
}
__host__ __device__ __forceinline__ const int* lor_d_scales(const double* Dq, int64_t nq) {
  return reinterpret_cast<const int*>(Dq + 6 * nq);
}
// doubles to allocate for D: 6 nq entries and nq int32 scale offsets
__host__ __device__ __forceinline__ int64_t lor_d_doubles(int64_t nq) { return 6 * nq + (nq + 1) / 2; }

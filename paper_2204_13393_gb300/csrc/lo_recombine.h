// Recombination of the digit pair sums of one output into a float64, in
// integer arithmetic (host and device).
//
// The tensor-core forms split every float64 operand into 7 digits (Sec. 4.1
// products in the digit arithmetic of lo_ozaki.cu) and sum the products of
// each digit class v = t + u exactly; one output is then
//     v = RN( RN(rest) 2^-45 + S_2 ) 2^X,
// S_2 the class-2 sum (|S_2| < 2^31), rest the lower classes folded into a
// 64-bit integer (|rest| < 2^63), X the exponent of the scaling.  Written
// with float64 operations that is an int64 conversion, an int32 conversion,
// a fused multiply-add and a compare per output, which run at the float64
// rate, on GB300 a small fraction of the integer rate.  oz_recombine forms
// the same two roundings (to nearest, ties to even) on the exact integer
// T = RN(rest) + S_2 2^45 and assembles the bits, so its result is the
// float64 expression's bit for bit.  Only a result outside the normal range
// after the scaling falls back to two float64 multiplications.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define LO_HD __host__ __device__ __forceinline__
#else
#define LO_HD inline
#endif

namespace lo {

LO_HD int oz_clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

LO_HD double oz_from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// v * 2^X for an integer X in a wide range (two exact power-of-two factors).
LO_HD double scale2(double v, int X) {
  if (X < -2044) return 0.0;
  const int X1 = X / 2, X2 = X - X1;
  const double f1 = oz_from_bits((uint64_t)(X1 + 1023) << 52);
  const double f2 = oz_from_bits((uint64_t)(X2 + 1023) << 52);
  return (v * f1) * f2;
}

// RN(RN(rest) 2^-45 + s2) 2^X, as fma((double)rest, 0x1p-45, (double)s2)
// followed by an exact exponent shift (scale2 where the shift leaves the
// normal range); +0.0 for a zero sum.
LO_HD double oz_recombine(int s2, long long rest, int X) {
  // RN(rest) to 53 significant bits: magnitude am <= 2^63, sign an
  const bool an = rest < 0;
  uint64_t am = an ? (uint64_t)0 - (uint64_t)rest : (uint64_t)rest;
  if (am >> 53) {
    const int sh = 63 - oz_clz64(am) - 52;  // 1 .. 11
    uint64_t keep = am >> sh;
    const uint64_t rem = am & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (keep & 1))) ++keep;
    am = keep << sh;
  }
  // the exact sum T = RN(rest) + s2 2^45 (|T| < 2^78)
  const __int128 T = (__int128)s2 * ((__int128)1 << 45) + (an ? -(__int128)am : (__int128)am);
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const uint64_t hi = (uint64_t)(M >> 64), lo = (uint64_t)M;
  int p = hi ? 127 - oz_clz64(hi) : 63 - oz_clz64(lo);  // leading bit of |T|
  uint64_t mant;
  if (p <= 52) {
    mant = lo << (52 - p);
  } else {
    const int sh = p - 52;  // 1 .. 25
    uint64_t keep = (uint64_t)(M >> sh);
    const unsigned __int128 rem = M & (((unsigned __int128)1 << sh) - 1), half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (keep & 1))) {
      if (++keep == (1ull << 53)) {
        keep >>= 1;
        ++p;
      }
    }
    mant = keep;
  }
  // |T| 2^-45 is normal: biased exponent p - 45 + 1023 in 978 .. 1056
  const uint64_t sign = neg ? (1ull << 63) : 0ull, frac = mant & ((1ull << 52) - 1);
  const int e = p - 45 + 1023, E = e + X;
  if (E >= 1 && E <= 2046) return oz_from_bits(sign | ((uint64_t)E << 52) | frac);
  return scale2(oz_from_bits(sign | ((uint64_t)e << 52) | frac), X);
}

// The float64 of a nonzero integer m 2^e2 (|m| < 2^53) built from its bits.
LO_HD double oz_exact_double(long long m, int e2) {
  if (m == 0) return 0.0;
  const uint64_t sign = m < 0 ? (1ull << 63) : 0ull;
  const uint64_t a = m < 0 ? (uint64_t)0 - (uint64_t)m : (uint64_t)m;
  const int p = 63 - oz_clz64(a);  // leading bit, <= 52
  return oz_from_bits(sign | ((uint64_t)(1023 + p + e2) << 52) | ((a << (52 - p)) & ((1ull << 52) - 1)));
}

// The class sums d[0..7] of one output (d[0] = S_2, d[1..5] = S_3 .. S_7,
// d[6], d[7] = S_8 of the two pair groups) recombined with one rounding:
// RN(T) 2^(X - 45) for the exact integer T = S_2 2^45 + rest,
//   rest = S_3 2^37 + S_4 2^29 + S_5 2^21 + S_6 2^13 + S_7 2^5
//          + floor((S_8a + 4) / 8) + floor((S_8b + 4) / 8),
// for |d| <= 2^23 - 2^16.  Adjacent classes pair exactly in 32 bits
// (A = S_v 2^8 + S_(v+1)), so T = A1 2^37 + lo with |A1| < 2^31 and
// |lo| < 2^53, both exact as float64 (built from their bits), and their one
// float64 addition is RN(T).  A result outside the normal range after the
// scaling goes through scale2.
LO_HD double oz_recombine8_add(const int (&d)[8], int X) {
  const int a1 = d[0] * 256 + d[1], a2 = d[2] * 256 + d[3], a3 = d[4] * 256 + d[5];
  const long long lo = (long long)a2 * (1ll << 21) + (long long)a3 * 32 + ((d[6] + 4) >> 3) + ((d[7] + 4) >> 3);
  const double v = oz_exact_double(a1, 37) + oz_exact_double(lo, 0);  // RN(T), T 2^0
  uint64_t b;
#ifdef __CUDA_ARCH__
  b = (uint64_t)__double_as_longlong(v);
#else
  std::memcpy(&b, &v, sizeof b);
#endif
  if ((b << 1) == 0) return 0.0;
  const int e = (int)((b >> 52) & 0x7FF), E = e + X - 45;
  if (E >= 1 && E <= 2046) return oz_from_bits(b + ((uint64_t)(int64_t)(X - 45) << 52));
  return scale2(oz_from_bits(b - (45ull << 52)), X);  // T 2^-45 (normal: e >= 1023), as the others scale it
}

// d of a float32 x = d 2^-48 with d an integer, |d| < 2^22: one add of the
// constant 1.5 2^-25 puts d + 1.5 2^23 in the significand exactly.
LO_HD int oz_f2i_small(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_int(__fadd_rn(x, 0x1.8p-25f)) - 0x33400000;
#else
  const float y = x + 0x1.8p-25f;
  int b;
  std::memcpy(&b, &y, 4);
  return b - 0x33400000;
#endif
}

}  // namespace lo

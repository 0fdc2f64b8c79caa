// Bitwise checks of the integer recombination of digit pair sums
// (lo_recombine.h) against the expressions that define them:
//   oz_recombine:       v = fma((double)rest, 2^-45, (double)s2),
//   oz_recombine8_add:  v = the exact s2 + rest 2^-45 of the 8 class sums
//                       (rest formed from them as its definition states)
//                       rounded once: a 128-bit integer converted to double,
// each then scaled by 2^X (an exponent shift when the result stays normal,
// else (v * 2^X1) * 2^X2); oz_f2i_small: the integer d of d 2^-48, all d
// in [-2^22, 2^22).  Random inputs over all magnitudes plus constructed ties,
// carries, cancellations and exponent-range edges.  Prints
// "cases N mismatches M".
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "lo_recombine.h"

static uint64_t bits(double d) {
  uint64_t b;
  std::memcpy(&b, &d, 8);
  return b;
}
static double from(uint64_t b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

static double scaled(double v, int X) {
  if (v == 0.0) return 0.0;
  const int e = (int)((bits(v) >> 52) & 0x7FF);
  if (e + X >= 1 && e + X <= 2046 && e != 0) return from(bits(v) + (uint64_t)((int64_t)X << 52));
  if (X < -2044) return 0.0;
  const int X1 = X / 2, X2 = X - X1;
  return (v * from((uint64_t)(X1 + 1023) << 52)) * from((uint64_t)(X2 + 1023) << 52);
}
static double reference(int s2, long long rest, int X) {
  return scaled(std::fma((double)rest, 0x1p-45, (double)s2), X);
}
static double reference_exact(int s2, long long rest, int X) {
  const __int128 T = (__int128)s2 * ((__int128)1 << 45) + rest;
  return scaled(std::ldexp((double)T, -45), X);
}

static uint64_t sm_state = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // splitmix64
  uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static long long cases = 0, bad = 0;
static void check(int s2, long long rest, int X) {
  ++cases;
  const double a = lo::oz_recombine(s2, rest, X), b = reference(s2, rest, X);
  if (bits(a) != bits(b)) {
    if (bad < 10)
      std::printf("mismatch s2=%d rest=%lld X=%d: %a vs %a\n", s2, rest, X, a, b);
    ++bad;
  }
}

int main() {
  // random magnitudes
  for (int i = 0; i < 4000000; ++i) {
    const int s2 = (int)(next() >> (32 + next() % 33));
    const long long rest = (long long)(next() >> (next() % 64)) * ((next() & 1) ? 1 : -1);
    const int sgn = (next() & 1) ? -1 : 1;
    const int X = (int)(next() % 3400) - 2300;
    check(sgn * s2, rest, X);
  }
  // the kernels' typical scale: X near -2060 .. -1000
  for (int i = 0; i < 1000000; ++i) {
    const int s2 = (int)(uint32_t)next();
    const long long rest = (long long)next() >> (1 + next() % 40);
    check(s2, rest, (int)(next() % 1100) - 2100);
  }
  // ties of the first rounding (rest beyond 53 bits)
  for (int sh = 1; sh <= 10; ++sh)
    for (int i = 0; i < 20000; ++i) {
      const uint64_t keep = (1ull << 52) | (next() & ((1ull << 52) - 1));
      const uint64_t m = (keep << sh) | (1ull << (sh - 1));
      if (m >> 63) continue;
      check((int)(next() % 7) - 3, (next() & 1) ? (long long)m : -(long long)m, -1100);
    }
  // ties and carries of the second rounding: T = s2 2^45 + rest with the
  // dropped bits exactly half, or all ones
  for (int i = 0; i < 200000; ++i) {
    const int s2 = (int)(next() | 0x40000000u) * ((next() & 1) ? 1 : -1);
    const int sh = 63 - __builtin_clzll((uint64_t)std::llabs((long long)s2)) + 45 - 52;  // dropped bits of T
    long long low = (next() & 1) ? (1ll << (sh - 1)) : ((1ll << sh) - 1);
    if (next() & 1) low += (long long)(next() % 1024) << sh;
    check(s2, (next() & 1) ? low : -low, -1090);
  }
  // cancellation: rest = -s2 2^45 + small
  for (int i = 0; i < 200000; ++i) {
    const int s2 = (int)(next() % 200000) - 100000;
    const long long small = (long long)(next() % 2000) - 1000;
    check(s2, -(long long)s2 * (1ll << 45) + small, -1050);
  }
  // extremes
  const long long rests[] = {0, 1, -1, (long long)(~0ull >> 1), (long long)(1ull << 63), (1ll << 53), (1ll << 53) + 1,
                             -(1ll << 53) - 1, (1ll << 62) + 1, (1ll << 62) - 1};
  const int s2s[] = {0, 1, -1, 2147483647, (int)0x80000000u, 65536, -65536};
  for (long long r : rests)
    for (int s : s2s)
      for (int X = -2200; X <= 1200; X += 1) check(s, r, X);
  // the 8 class sums of one output, |d| <= 2^23 - 2^16
  for (int i = 0; i < 3000000; ++i) {
    int d[8];
    const int lim = (i & 1) ? (1 << 22) : ((1 << 23) - (1 << 16));
    const int bw = 1 + (int)(next() % 23);
    for (int v = 0; v < 8; ++v) {
      long long x = (long long)(next() & ((1ull << bw) - 1)) * ((next() & 1) ? 1 : -1);
      if (x > lim) x = lim;
      if (x < -lim) x = -lim;
      d[v] = (int)x;
    }
    if (i % 7 == 0) d[0] = 0;
    if (i % 11 == 0) d[0] = d[1] = 0;
    if (i % 13 == 0) d[1] = -d[0] * 256 + (int)(next() % 64) - 32, d[1] = d[1] > lim ? lim : (d[1] < -lim ? -lim : d[1]);
    long long rest = (long long)d[1] * (1ll << 37) + (long long)d[2] * (1ll << 29) + (long long)d[3] * (1ll << 21) +
                     (long long)d[4] * (1ll << 13) + (long long)d[5] * 32 + ((d[6] + 4) >> 3) + ((d[7] + 4) >> 3);
    const int X = (int)(next() % 3400) - 2300;
    const double b = reference_exact(d[0], rest, X);
    ++cases;
    const double c = lo::oz_recombine8_add(d, X);
    if (bits(c) != bits(b)) {
      if (bad < 10) std::printf("mismatch (8 add) d0=%d d1=%d X=%d: %a vs %a\n", d[0], d[1], X, c, b);
      ++bad;
    }
  }
  // every class sum small enough for the one-add conversion
  for (int d = -(1 << 22); d < (1 << 22); ++d) {
    ++cases;
    if (lo::oz_f2i_small(std::ldexp((float)d, -48)) != d) {
      if (bad < 10) std::printf("mismatch f2i d=%d\n", d);
      ++bad;
    }
  }
  std::printf("cases %lld mismatches %lld\n", cases, bad);
  return bad != 0;
}

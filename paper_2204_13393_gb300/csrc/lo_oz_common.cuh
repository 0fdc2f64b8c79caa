// Digit arithmetic shared by the tensor-core kernels (lo_ozaki.cu: mma.sync
// forms that split float64 values in every pass; lo_umma.cu: tcgen05 forms
// over stored digit planes).  See lo_ozaki.cu for the scheme.
#pragma once

#include <cfloat>
#include <cstdint>

#include "lo_internal.h"
#include "lo_recombine.h"

namespace lo {
namespace {

constexpr int kPairs = 28;

__device__ __forceinline__ void oz_status(int* flags, lo_status st) {
  atomicOr(&flags[kFlagStatus], 1 << (int)st);
}

__device__ __forceinline__ int bexp(double x) {
  return (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7FF);
}

// Aligned significand of |x| against group exponent emax: Y < 2^56 as (yhi, ylo),
// sign in bit 31 of sgn.  Zero, subnormals and values 2^56 below the group give 0;
// returns true for Inf/NaN.
__device__ __forceinline__ bool oz_split(double x, int emax, unsigned& yhi, unsigned& ylo, unsigned& sgn) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FFu);
  sgn = hi & 0x80000000u;
  unsigned long long m = ((b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 3;
  const int sh = emax - e;
  m = (e == 0 || sh > 55 || sh < 0) ? 0ull : (m >> sh);
  yhi = (unsigned)(m >> 32);
  ylo = (unsigned)m;
  return e == 0x7FF;
}

// fp16x2 with the digits of plane t (1..7) of two values (low half = first),
// encoded as fp16 subnormals: the bits (sign << 15) | digit are the value
// +-digit * 2^-24 exactly, so no arithmetic is needed; products of two digits
// are integers times 2^-48, exact in float32.  sb: the two sign bits (bit 15
// for the first value, bit 31 for the second).
__device__ __forceinline__ unsigned oz_pack(int t, unsigned h0, unsigned l0, unsigned h1, unsigned l1, unsigned sb) {
  const bool hiw = t <= 3;
  const unsigned w0 = hiw ? h0 : l0, w1 = hiw ? h1 : l1;
  const unsigned bi = hiw ? (unsigned)(3 - t) : (unsigned)(7 - t);
  const unsigned v = __byte_perm(w0, w1, bi | ((4u + bi) << 8));
  return (v & 0x00FF00FFu) | sb;
}

// Write the 7 digit planes of a value pair into fragment storage.
// base: plane 0 address; plane_stride in uint32 words; idx: word index in a plane.
__device__ __forceinline__ void oz_store_pair(unsigned* base, int plane_stride, int idx, double x0, int e0,
                                              double x1, int e1, int* flags) {
  unsigned h0, l0, s0, h1, l1, s1;
  const bool bad = oz_split(x0, e0, h0, l0, s0) | oz_split(x1, e1, h1, l1, s1);
  if (bad) oz_status(flags, LO_ERR_NONFINITE);
  const unsigned sb = (s0 >> 16) | s1;
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t) base[(t - 1) * plane_stride + idx] = oz_pack(t, h0, l0, h1, l1, sb);
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Recombination of one output's 28 pair sums D_tu (exact integers, |D| < 2^24):
//   sum_{t,u} D_tu 2^(-8(t+u)) = 2^-16 (S_2 + rest 2^-45),  S_v = sum_{t+u=v} D_tu,
//   rest = S_3 2^37 + S_4 2^29 + S_5 2^21 + S_6 2^13 + S_7 2^5 + round(S_8 / 8)
// (|rest| < 2^63).  S_2 and rest convert exactly to float64; one fused
// multiply-add rounds the sum once, so the result carries float64 accuracy.
// The 28 pairs are split over two warp groups of 14 pairs each (digit t of
// the streamed operand: group 0 takes t in {1, 4, 5}, group 1 takes
// {2, 3, 6, 7}), so that a CTA runs 16 warps with half the accumulators each.
constexpr int kGroupPairs = 14;
__host__ __device__ constexpr bool pair_group_has(int g, int t) {
  return g == 0 ? (t == 1 || t == 4 || t == 5) : (t == 2 || t == 3 || t == 6 || t == 7);
}
template <int G, typename F>
__device__ __forceinline__ void for_group_pairs(F&& f) {
  int idx = 0;
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t)
#pragma unroll
    for (int u = 1; u <= kOzDigits; ++u)
      if (pair_group_has(G, t) && t + u <= 8) f(idx++, t, u);
}

// One group's share of the recombination of output j: S_2 and rest (see
// oz_combine); the two groups' shares add as integers.
template <int G>
__device__ __forceinline__ void group_partial(const float (&acc)[kGroupPairs][4], int j, int& s2, long long& rest) {
  int Sv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for_group_pairs<G>([&](int idx, int t, int u) { Sv[t + u] += __float2int_rn(acc[idx][j] * 0x1p48f); });
  s2 = Sv[2];
  long long r = (long long)Sv[3] * (1LL << 37);
  r += (long long)Sv[4] * (1LL << 29);
  r += (long long)Sv[5] * (1LL << 21);
  r += (long long)Sv[6] * (1LL << 13);
  r += (long long)Sv[7] * (1LL << 5);
  r += (long long)((Sv[8] + 4) >> 3);
  rest = r;
}

__device__ __forceinline__ double partial_to_double(int s2, long long rest) {
  return fma(__ll2double_rn(rest), 0x1p-45, (double)s2);
}

// 14 mma of one group: A fragments from shared-memory planes (uint4 per lane),
// B fragments from planes at bsrc (uint2 per lane; shared or global memory).
template <int G, bool BGLOBAL>
__device__ __forceinline__ void group_mma(float (&acc)[kGroupPairs][4], const unsigned* apl, int a_stride,
                                          const unsigned* bpl, int b_stride, int lane) {
  unsigned af[kOzDigits][4], bf[kOzDigits][2];
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t) {
    if (pair_group_has(G, t)) {
      const uint4 v = *reinterpret_cast<const uint4*>(apl + (t - 1) * a_stride + lane * 4);
      af[t - 1][0] = v.x; af[t - 1][1] = v.y; af[t - 1][2] = v.z; af[t - 1][3] = v.w;
    }
  }
  constexpr int umax = (G == 0) ? 7 : 6;
#pragma unroll
  for (int u = 1; u <= umax; ++u) {
    const uint2* bp = reinterpret_cast<const uint2*>(bpl + (u - 1) * b_stride + lane * 2);
    const uint2 w = BGLOBAL ? __ldg(bp) : *bp;
    bf[u - 1][0] = w.x; bf[u - 1][1] = w.y;
  }
  for_group_pairs<G>([&](int idx, int t, int u) { mma_f16(acc[idx], af[t - 1], bf[u - 1][0], bf[u - 1][1]); });
}

// The B operand of k_umma_update for one chunk: the scaled coefficient Cf
// (Kt x NC, row-major) split against its column exponents Gs into 7 digits.
// Per (output group z of NB columns, 16-column step ks) one R x 16 K-major
// no-swizzle tile, R = round16(7 NB): row (u - 1) NB + n holds digit u of
// coefficient (16 ks + kk, z NB + n); rows past 7 NB and columns past Kt are
// zero.  KS: steps per output group in the image.  Whole CTA.
template <int NC>
__device__ void umma_coef_image(const double* Cf, const int* Gs, int Kt, int KS, unsigned char* img, int* flags) {
  constexpr int NB = NC < 16 ? NC : 16, NSPL = NC / NB, R = (7 * NB + 15) / 16 * 16;
  const int ksteps = (Kt + 15) / 16, tid = threadIdx.x;
  // one item = (split z, step ks, row n of the split, K quad kq): 4 coefficients
  for (int it = tid; it < NSPL * ksteps * NB * 4; it += blockDim.x) {
    const int kq = it & 3, rest = it >> 2;
    const int n = rest % NB, zks = rest / NB, ks = zks % ksteps, z = zks / ksteps;
    const int col = z * NB + n, q0 = ks * 16 + kq * 4;
    double x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = (q0 + j < Kt) ? Cf[(q0 + j) * NC + col] : 0.0;
    const int e = Gs[col];
    unsigned h[4], l[4], g[4];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) bad |= oz_split(x[j], e, h[j], l[j], g[j]);
    if (bad) oz_status(flags, LO_ERR_NONFINITE);
    unsigned char* base = img + (int64_t)(z * KS + ks) * R * 32 + (kq & 1) * 8 + (kq >> 1) * 128;
#pragma unroll
    for (int u = 1; u <= kOzDigits; ++u) {
      const int row = (u - 1) * NB + n;
      const unsigned w0 = oz_pack(u, h[0], l[0], h[1], l[1], (g[0] >> 16) | g[1]);
      const unsigned w1 = oz_pack(u, h[2], l[2], h[3], l[3], (g[2] >> 16) | g[3]);
      *reinterpret_cast<uint2*>(base + (row & 7) * 16 + (row >> 3) * 256) = make_uint2(w0, w1);
    }
  }
  if constexpr (R > 7 * NB) {  // pad rows
    for (int it = tid; it < NSPL * ksteps * (R - 7 * NB) * 4; it += blockDim.x) {
      const int kq = it & 3, rest = it >> 2;
      const int pr = rest % (R - 7 * NB), zks = rest / (R - 7 * NB), ks = zks % ksteps, z = zks / ksteps;
      const int row = 7 * NB + pr;
      unsigned char* base = img + (int64_t)(z * KS + ks) * R * 32 + (kq & 1) * 8 + (kq >> 1) * 128;
      *reinterpret_cast<uint2*>(base + (row & 7) * 16 + (row >> 3) * 256) = make_uint2(0u, 0u);
    }
  }
}

// v * 2^X by adding X to the exponent field when the result stays normal
// (integer work only); otherwise through scale2.
__device__ __forceinline__ double scale_exp(double v, int X) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  if ((b << 1) == 0) return 0.0;  // +-0 (an integer test: float64 compares run at the float64 rate)
  if (e + X >= 1 && e + X <= 2046 && e != 0) return __longlong_as_double(b + ((long long)X << 52));
  return scale2(v, X);
}

// cp.async helpers (Ampere-style asynchronous global->shared copies).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(gmem), "r"(sz));
}
// 4 bytes (always valid: the source is an in-bounds table entry).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;"); }

// Split 8 float64 values x[0..7] (8 consecutive rows of one column) against
// exponent e and store their fp16 digits as one 16-byte core-matrix row of
// each of the first ND planes at dst + t * plane.
template <int ND = kOzDigits>
__device__ __forceinline__ void split8_store(const double* x, int e, unsigned char* dst, int plane, int* flags) {
  unsigned w[ND][4];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned h0, l0, s0, h1, l1, s1;
    bad |= oz_split(x[2 * i], e, h0, l0, s0);
    bad |= oz_split(x[2 * i + 1], e, h1, l1, s1);
    const unsigned sb = (s0 >> 16) | s1;
#pragma unroll
    for (int t = 1; t <= ND; ++t) w[t - 1][i] = oz_pack(t, h0, l0, h1, l1, sb);
  }
  if (bad) oz_status(flags, LO_ERR_NONFINITE);
#pragma unroll
  for (int t = 0; t < ND; ++t)
    *reinterpret_cast<uint4*>(dst + t * plane) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// Split V (1, 2 or 4) consecutive values of one column against exponent e and
// store the fp16 digits of the first ND planes: per plane the V values as
// consecutive 2-byte entries at dst + (t - 1) * stride.
template <int V, int ND>
__device__ __forceinline__ void split_rows_store(const double* x, int e, unsigned char* dst, int stride, int* flags) {
  static_assert(V == 1 || V == 2 || V == 4, "split_rows_store: 1, 2 or 4 values");
  unsigned h[V], l[V], g[V];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < V; ++i) bad |= oz_split(x[i], e, h[i], l[i], g[i]);
  if (bad) oz_status(flags, LO_ERR_NONFINITE);
#pragma unroll
  for (int t = 1; t <= ND; ++t) {
    unsigned char* d = dst + (t - 1) * stride;
    if constexpr (V == 1) {
      const unsigned w = t <= 3 ? h[0] : l[0];
      const unsigned digit = (w >> (8 * (t <= 3 ? 3 - t : 7 - t))) & 0xFFu;
      *reinterpret_cast<unsigned short*>(d) = (unsigned short)((g[0] >> 16) | digit);
    } else if constexpr (V == 2) {
      *reinterpret_cast<unsigned*>(d) = oz_pack(t, h[0], l[0], h[1], l[1], (g[0] >> 16) | g[1]);
    } else {
      *reinterpret_cast<uint2*>(d) = make_uint2(oz_pack(t, h[0], l[0], h[1], l[1], (g[0] >> 16) | g[1]),
                                                oz_pack(t, h[2], l[2], h[3], l[3], (g[2] >> 16) | g[3]));
    }
  }
}

// split_rows_store into two destinations (planes stride1 and stride2 bytes
// apart): one split, the same digits stored twice.
template <int V, int ND>
__device__ __forceinline__ void split_rows_store2(const double* x, int e, unsigned char* dst1, int stride1,
                                                  unsigned char* dst2, int stride2, int* flags) {
  static_assert(V == 1 || V == 2 || V == 4, "split_rows_store2: 1, 2 or 4 values");
  unsigned h[V], l[V], g[V];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < V; ++i) bad |= oz_split(x[i], e, h[i], l[i], g[i]);
  if (bad) oz_status(flags, LO_ERR_NONFINITE);
#pragma unroll
  for (int t = 1; t <= ND; ++t) {
    unsigned char* d1 = dst1 + (t - 1) * stride1;
    unsigned char* d2 = dst2 + (t - 1) * stride2;
    if constexpr (V == 1) {
      const unsigned w = t <= 3 ? h[0] : l[0];
      const unsigned short v = (unsigned short)((g[0] >> 16) | ((w >> (8 * (t <= 3 ? 3 - t : 7 - t))) & 0xFFu));
      *reinterpret_cast<unsigned short*>(d1) = v;
      *reinterpret_cast<unsigned short*>(d2) = v;
    } else if constexpr (V == 2) {
      const unsigned v = oz_pack(t, h[0], l[0], h[1], l[1], (g[0] >> 16) | g[1]);
      *reinterpret_cast<unsigned*>(d1) = v;
      *reinterpret_cast<unsigned*>(d2) = v;
    } else {
      const uint2 v = make_uint2(oz_pack(t, h[0], l[0], h[1], l[1], (g[0] >> 16) | g[1]),
                                 oz_pack(t, h[2], l[2], h[3], l[3], (g[2] >> 16) | g[3]));
      *reinterpret_cast<uint2*>(d1) = v;
      *reinterpret_cast<uint2*>(d2) = v;
    }
  }
}

// Digit planes of the new panel (slot nb) of one slab, once stage 2 has fixed
// the panel's column exponents.  One thread per (16-row tile, column): 16
// values, 7 planes of two 16-byte core-matrix rows each.  Whole CTA (256
// threads); returns after a barrier.
template <int S>
__device__ void digitize_slab(const StepArgs& a, int slab) {
  __shared__ int ex[S];
  const SlabInfo si = a.slabs[slab];
  const int k = a.nb * S;
  if (threadIdx.x < S) ex[threadIdx.x] = a.colexp[(int64_t)(k + threadIdx.x) * a.p + si.chunk];
  __syncthreads();
  const double* slot = a.V + (int64_t)a.nb * a.n * S;
  const int ntile = (si.rows + 15) / 16;
  const int64_t gtot = (int64_t)a.M * (S / 8);
  for (int i = threadIdx.x; i < ntile * S; i += 256) {
    const int tt = i / S, j = i - tt * S;
    const int64_t G = (int64_t)a.nb * (S / 8) + j / 8;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t eta = 2 * (int64_t)(si.tile0 + tt) + h;
      double x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = tt * 16 + h * 8 + r;
        x[r] = row < si.rows ? slot[(si.row0 + row) * S + j] : 0.0;
      }
      split8_store(x, ex[j], a.dig + (eta * gtot + G) * (kOzDigits * 128) + (j & 7) * 16, 128, a.flags);
    }
  }
  __syncthreads();
}

}  // namespace
}  // namespace lo

// Float64-accurate products of the two O(n) passes on the tensor cores.
//
// GB300 runs float64 arithmetic at ~1.2 TFLOP/s, far below what the streaming
// passes need; its fp16 tensor path is ~500x faster.  Each float64 value x of a
// group g (a column of one chunk or slab) is written exactly as
//     x = 2^(E_g - 1022) * sum_{t=1..7} d_t 2^(-8t) + r,   |r| < 2^(E_g - 1078)
// with integer digits d_t in [-255, 255] (the bytes of x's significand aligned
// to the group's largest biased exponent E_g; error-free splitting in the sense
// of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)).  Digits are
// exact in fp16; a product of two digits has at most 16 bits, so a float32
// accumulation of up to 256 of them (one 256-row slab, or 256 reduction columns)
// is exact.  The 28 digit pairs with t + u <= 8 carry every term above 2^-56 of
// the product's scale; they run as mma.sync m16n8k16 (fp16 in, float32
// accumulate) and are recombined per output in a 64-bit integer before one
// conversion to float64.
//
// Kernels:
//   k_oz_gram    stage-1 Gram partial C = [Q_i A_i]^T A_i of one slab (Alg. 7,
//                first line), the A_i^T side sliced per column exponent;
//   k_oz_coef    per chunk, the float64 coefficient matrix of an assembly
//                product (Sec. 4.1) scaled by the column exponents and sliced;
//   k_oz_update  out = [Q_i A_i] Coef for one slab (stage 2, and the
//                reiteration's new iterate), writing the new local panel.
#include <cfloat>
#include <cstdint>

#include "lo_internal.h"

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
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
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

// The 28 digit pairs (t, u), t + u <= 8, as a compile-time walk.
template <typename F>
__device__ __forceinline__ void for_pairs(F&& f) {
  int idx = 0;
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t)
#pragma unroll
    for (int u = 1; u <= kOzDigits; ++u)
      if (t + u <= 8) f(idx++, t, u);
}

// Recombination of one output's 28 pair sums D_tu (exact integers, |D| < 2^24):
//   sum_{t,u} D_tu 2^(-8(t+u)) = 2^-16 (S_2 + rest 2^-45),  S_v = sum_{t+u=v} D_tu,
//   rest = S_3 2^37 + S_4 2^29 + S_5 2^21 + S_6 2^13 + S_7 2^5 + round(S_8 / 8)
// (|rest| < 2^63).  S_2 and rest convert exactly to float64; one fused
// multiply-add rounds the sum once, so the result carries float64 accuracy.
__device__ __forceinline__ double oz_combine(const float (&acc)[kPairs][4], int j) {
  int Sv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for_pairs([&](int idx, int t, int u) { Sv[t + u] += __float2int_rn(acc[idx][j] * 0x1p48f); });
  long long rest = (long long)Sv[3] * (1LL << 37);
  rest += (long long)Sv[4] * (1LL << 29);
  rest += (long long)Sv[5] * (1LL << 21);
  rest += (long long)Sv[6] * (1LL << 13);
  rest += (long long)Sv[7] * (1LL << 5);
  rest += (long long)((Sv[8] + 4) >> 3);
  return fma(__ll2double_rn(rest), 0x1p-45, (double)Sv[2]);
}

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

// v * 2^X for an integer X in a wide range (two exact power-of-two factors).
__device__ __forceinline__ double scale2(double v, int X) {
  if (X < -2044) return 0.0;
  const int X1 = X / 2, X2 = X - X1;
  const double f1 = __longlong_as_double((long long)(X1 + 1023) << 52);
  const double f2 = __longlong_as_double((long long)(X2 + 1023) << 52);
  return (v * f1) * f2;
}

// v * 2^X by adding X to the exponent field when the result stays normal
// (integer work only); otherwise through scale2.
__device__ __forceinline__ double scale_exp(double v, int X) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  if (v == 0.0) return 0.0;
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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;"); }

// ---------------------------------------------------------------------------
// Stage-1 Gram partial of one slab and one group of MT*16 columns of [Q_i A].
// mma: M = columns of [Q_i A] (16 per tile), N = columns of A (8 per tile),
// K = rows (16 per step).  Warp w owns M-tile w % MT and N-tile w / MT.
// The float64 tiles of the next 16 rows stream into shared memory with
// cp.async while the current ones are sliced and multiplied.
template <int S>
struct GramSmem {
  static constexpr int NT = (S + 7) / 8, MT = 8 / NT, CG = MT * 16, NC = NT * 8;
  double raw[2][16][CG + 1];  // one pad double per row: fragment-ordered reads hit 2 wavefronts
  double rawB[2][16][S];
  unsigned Apl[2][kOzDigits][MT][32][4];
  unsigned Bpl[2][kOzDigits][NT][32][2];
  long long xrest[8][32][4];
  int xs2[8][32][4];
  int Hs[32];
  int Fs[CG];
};

template <int S>
__device__ __forceinline__ void gram_prefetch(GramSmem<S>& sm, int buf, const StepArgs& a, const SlabInfo& si,
                                              const double* src, int64_t lds, int r0, int col0, int k) {
  constexpr int CG = GramSmem<S>::CG;
  const int tid = threadIdx.x;
  // columns of the local panels inside this group: whole panels (S divides 16, or CG == S)
  const int qend = min(col0 + CG, k);
  const int qn = qend > col0 ? qend - col0 : 0;  // multiple of S
  {
    const int r = tid >> 5, l0 = tid & 31;  // 16 rows x 32 lanes
    const bool ok = r0 + r < si.rows;
    const int64_t row = si.row0 + (ok ? r0 + r : 0);
    for (int cc = l0; cc < qn; cc += 32) {
      const int q = col0 + cc;
      cp_async8(&sm.raw[buf][r][cc], a.V + (int64_t)(q / S) * a.n * S + row * S + (q % S), ok);
    }
  }
  // the block's own columns: in the A tile when inside this group, and as the B operand
  const bool in_group = (k >= col0 && k < col0 + CG);
  for (int c = tid; c < 16 * S; c += 512) {
    const int r = c / S, l = c - r * S;
    const bool ok = r0 + r < si.rows;
    const int64_t row = si.row0 + (ok ? r0 + r : 0);
    const double* g = src + row * lds + l;
    cp_async8(&sm.rawB[buf][r][l], g, ok);
    if (in_group) cp_async8(&sm.raw[buf][r][k - col0 + l], g, ok);
  }
}

// Stage-1 Gram partial of one slab and one group of MT*16 columns of [Q_i A].
// mma: M = columns of [Q_i A] (16 per tile), N = columns of A (8 per tile),
// K = rows (16 per step).  Warp w owns tile w % 8 (M-tile (w % 8) % MT, N-tile
// (w % 8) / MT) and pair group w / 8.  The float64 tiles of the next 16 rows
// stream into shared memory with cp.async while the current ones are sliced
// and multiplied.
template <int S>
__global__ void __launch_bounds__(512, 1) k_oz_gram(StepArgs a, const double* src, int64_t lds, int pass) {
  using SM = GramSmem<S>;
  constexpr int NT = SM::NT, MT = SM::MT, CG = SM::CG, NC = SM::NC;
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const SlabInfo si = a.slabs[blockIdx.x];
  const int k = a.nb * S, Kt = k + S;
  const int col0 = blockIdx.y * CG;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp >> 3, tile = warp & 7;
  gram_prefetch<S>(sm, 0, a, si, src, lds, 0, col0, k);
  cp_async_commit();
  if (tid < 32) sm.Hs[tid] = 0;
  __syncthreads();
  for (int idx = tid; idx < si.rows * S; idx += 512) {
    const int r = idx / S, l = idx - r * S;
    atomicMax(&sm.Hs[l], bexp(src[(si.row0 + r) * lds + l]));
  }
  __syncthreads();
  if (blockIdx.y == 0 && tid < S) a.srcexp_slab[(int64_t)blockIdx.x * 32 + tid] = sm.Hs[tid];
  for (int m = tid; m < CG; m += 512) {
    const int col = col0 + m;
    sm.Fs[m] = (col < k) ? a.colexp[(int64_t)col * a.p + si.chunk] : (col < Kt ? sm.Hs[col - k] : 0);
  }
  float acc[kGroupPairs][4];
#pragma unroll
  for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  const int mt = tile % MT, nt = tile / MT;
  const int nsteps = (si.rows + 15) / 16;
  // slice the float64 tile of one 16-row step into digit-plane buffer pb
  auto slice = [&](int rb, int pb) {
    // A: value pairs (rows 2j, 2j+1 of the step; column m), taken in fragment
    // order so that each digit-plane store of a warp is 32 consecutive words
    for (int pi = tid; pi < 8 * CG; pi += 512) {
      const int mtile = pi >> 7, w = pi & 127, ln = w >> 2, rg = w & 3;
      const int mm = (ln >> 2) + 8 * (rg & 1), j = (ln & 3) + 4 * (rg >> 1);
      const int m = mtile * 16 + mm;
      const int col = col0 + m;
      double x0 = 0.0, x1 = 0.0;
      if (col < Kt) {
        x0 = sm.raw[rb][2 * j][m];
        x1 = sm.raw[rb][2 * j + 1][m];
      }
      oz_store_pair(&sm.Apl[pb][0][mtile][0][0], MT * 128, w, x0, sm.Fs[m], x1, sm.Fs[m], a.flags);
    }
    // B: value pairs of the block's columns, in fragment order
    for (int pi = tid; pi < 8 * NC; pi += 512) {
      const int ntile = pi >> 6, w = pi & 63, ln = w >> 1, rg = w & 1;
      const int n = ntile * 8 + (ln >> 2), j = (ln & 3) + 4 * rg;
      double x0 = 0.0, x1 = 0.0;
      if (n < S) {
        x0 = sm.rawB[rb][2 * j][n];
        x1 = sm.rawB[rb][2 * j + 1][n];
      }
      const int e = (n < S) ? sm.Hs[n] : 0;
      oz_store_pair(&sm.Bpl[pb][0][ntile][0][0], NT * 64, w, x0, e, x1, e, a.flags);
    }
  };
  // exact float32 sums cover 16 steps (256 rows): group 1 hands its integer
  // partials to group 0, which accumulates them in float64
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  auto flush = [&]() {
    int s2[4];
    long long rest[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (grp == 0)
        group_partial<0>(acc, j, s2[j], rest[j]);
      else
        group_partial<1>(acc, j, s2[j], rest[j]);
    }
    if (grp == 1) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sm.xs2[tile][lane][j] = s2[j];
        sm.xrest[tile][lane][j] = rest[j];
      }
    }
    __syncthreads();
    if (grp == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        accd[j] += partial_to_double(s2[j] + sm.xs2[tile][lane][j], rest[j] + sm.xrest[tile][lane][j]);
    }
#pragma unroll
    for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  };
  // pipeline: step st+2 streams into the raw buffer of step st, step st+1 is
  // sliced while step st is multiplied; one barrier per step
  if (nsteps > 1) gram_prefetch<S>(sm, 1, a, si, src, lds, 16, col0, k);
  cp_async_commit();
  cp_async_wait1();
  __syncthreads();
  slice(0, 0);
  for (int st = 0; st < nsteps; ++st) {
    cp_async_wait0();
    __syncthreads();
    if (st + 2 < nsteps) gram_prefetch<S>(sm, st & 1, a, si, src, lds, 16 * (st + 2), col0, k);
    cp_async_commit();
    if (st + 1 < nsteps) slice((st + 1) & 1, (st + 1) & 1);
    const int pb = st & 1;
    if (grp == 0)
      group_mma<0, false>(acc, &sm.Apl[pb][0][mt][0][0], MT * 128, &sm.Bpl[pb][0][nt][0][0], NT * 64, lane);
    else
      group_mma<1, false>(acc, &sm.Apl[pb][0][mt][0][0], MT * 128, &sm.Bpl[pb][0][nt][0][0], NT * 64, lane);
    if (((st + 1) & 15) == 0 && st + 1 < nsteps) flush();  // slabs of more than 256 rows (s = 32)
  }
  cp_async_wait0();
  flush();
  if (grp == 0) {
    const int g = lane >> 2, c = lane & 3;
    double* out = a.part + (int64_t)blockIdx.x * a.Kmax * S;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = mt * 16 + g + ((j >> 1) << 3), n = nt * 8 + 2 * c + (j & 1);
      const int col = col0 + m;
      if (col < Kt && n < S) out[(int64_t)col * S + n] = scale_exp(accd[j], sm.Fs[m] + sm.Hs[n] - 2044 - 16);
    }
  }
}

// ---------------------------------------------------------------------------
// Coefficients of an assembly product for chunk c, scaled row by row by the
// column exponents of [Q_i A] and sliced into B-fragment digit planes.
//   mode 1 (new iterate of a reiteration, NOUT = 1): [-P N^{-1}; N^{-1}]
//   mode 2 (stage 2, NOUT = 2): [-P N^{-1}, Pt - P N^{-1} Nt; N^{-1}, N^{-1} Nt]
// with (P, N^{-1}) of the last local pass and [Pt; Nt] the new tree column block.
template <int S, int NOUT>
__global__ void __launch_bounds__(256) k_oz_coef(StepArgs a, int pass) {
  constexpr int NC = NOUT * S, NT = (NC + 7) / 8;
  if (NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) double smc[];
  const int c = blockIdx.x, k = a.nb * S, Kt = k + S;
  const SmallLayout SL = SmallLayout::make(a.Kmax, S);
  const double* smallc = a.small + (int64_t)c * SL.stride;
  const double* P = smallc + SL.P_last;
  const double* Ninv = smallc + SL.Ninv_last;
  const double* Tb = a.T + (int64_t)c * a.tstride + tblock_offset(a.nb, S);
  double* Cf = smc;                               // Kt x NC (scaled)
  double* PN = Cf + (size_t)Kt * NC;              // k x S: P N^{-1}
  int* Gs = reinterpret_cast<int*>(PN + (size_t)k * S);  // NC
  const int tid = threadIdx.x;
  for (int e = tid; e < k * S; e += 256) {
    const int q = e / S, l = e - q * S;
    double v = 0.0;
    for (int j = 0; j <= l; ++j) v += P[q * S + j] * Ninv[j * S + l];
    PN[e] = v;
  }
  if (tid < NC) Gs[tid] = 0;
  __syncthreads();
  for (int e = tid; e < Kt * NC; e += 256) {
    const int q = e / NC, n = e - q * NC;
    double v;
    if (n < S) {
      v = (q < k) ? -PN[q * S + n] : Ninv[(q - k) * S + n];
    } else {
      const int l = n - S;
      if (q < k) {
        v = Tb[q * S + l];
        for (int j = 0; j < S; ++j) v -= PN[q * S + j] * Tb[(k + j) * S + l];
      } else {
        v = 0.0;
        for (int j = 0; j < S; ++j) v += Ninv[(q - k) * S + j] * Tb[(k + j) * S + l];
      }
    }
    const int F = (q < k) ? a.colexp[(int64_t)q * a.p + c] : a.srcexp[(int64_t)c * 32 + (q - k)];
    v = (F == 0 || v == 0.0) ? 0.0 : scale2(v, F - 1022);
    Cf[e] = v;
    atomicMax(&Gs[n], bexp(v));
  }
  __syncthreads();
  unsigned* dig = a.coefdig + (int64_t)c * a.coefdig_stride;
  const int ksteps = (Kt + 15) / 16;
  // pairs (q even, q+1) for each column n
  for (int pi = tid; pi < ksteps * 8 * NT * 8; pi += 256) {
    const int n = pi % (NT * 8), qp = pi / (NT * 8), q = 2 * qp;
    const double x0 = (n < NC && q < Kt) ? Cf[q * NC + n] : 0.0;
    const double x1 = (n < NC && q + 1 < Kt) ? Cf[(q + 1) * NC + n] : 0.0;
    const int e = (n < NC) ? Gs[n] : 0;
    const int ks = q >> 4, kk = q & 15, nt = n >> 3;
    const int ln = (n & 7) * 4 + ((kk & 7) >> 1), rg = (kk >> 3) & 1;
    // layout: [kstep][ntile][plane][lane][2]
    unsigned* base = dig + ((int64_t)(ks * NT + nt) * kOzDigits) * 64;
    oz_store_pair(base, 64, ln * 2 + rg, x0, e, x1, e, a.flags);
  }
  for (int n = tid; n < NC; n += 256) a.coefexp[(int64_t)c * 64 + n] = Gs[n];
}

// ---------------------------------------------------------------------------
// out = [Q_i A] Coef for one slab: NOUT = 1 writes the new iterate into the new
// local panel; NOUT = 2 writes U_i into the panel and U to the caller, and
// records the panel's column exponents.  mma: M = rows (16 per tile), N = output
// columns, K = columns of [Q_i A] (16 per step).  Warp w: M-tile w % MT, N-tile
// w / MT.  The next step's 16 columns of the row tile stream in with cp.async.
template <int S, int NOUT>
struct UpdSmem {
  static constexpr int NC = NOUT * S, NT = (NC + 7) / 8, MT = (8 / NT) > 0 ? 8 / NT : 1, RT = MT * 16;
  double raw[2][RT][17];  // one pad double per row (see GramSmem)
  unsigned Apl[2][kOzDigits][MT][32][4];
  long long xrest[8][32][4];
  int xs2[8][32][4];
  int Fs[1024];
  int Cx[64];
  int Ux[32];
};

template <int S, int NOUT>
__device__ __forceinline__ void upd_prefetch(UpdSmem<S, NOUT>& sm, int buf, const StepArgs& a, const SlabInfo& si,
                                             const double* src, int64_t lds, int rt, int ks, int k, int Kt) {
  constexpr int RT = UpdSmem<S, NOUT>::RT;
  for (int c = threadIdx.x; c < RT * 8; c += 512) {
    const int r = c >> 3, j = c & 7, q0 = ks * 16 + 2 * j;
    const bool rok = rt + r < si.rows;
    const int64_t row = si.row0 + (rok ? rt + r : 0);
    double* d = &sm.raw[buf][r][2 * j];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = q0 + h;
      const double* gp;
      bool ok = rok && q < Kt;
      if (q < k)
        gp = a.V + (int64_t)(q / S) * a.n * S + row * S + (q % S);
      else if (q < Kt)
        gp = src + row * lds + (q - k);
      else
        gp = src + row * lds;
      cp_async8(d + h, gp, ok);
    }
  }
}

// out = [Q_i A] Coef for one slab: NOUT = 1 writes the new iterate into the new
// local panel; NOUT = 2 writes U_i into the panel and U to the caller, and
// records the panel's column exponents.  mma: M = rows (16 per tile), N = output
// columns, K = columns of [Q_i A] (16 per step).  Warp w: tile w % 8 (M-tile
// (w % 8) % MT, N-tile (w % 8) / MT), pair group w / 8.  The next step's 16
// columns of the row tile stream in with cp.async.
template <int S, int NOUT>
__global__ void __launch_bounds__(512, 1) k_oz_update(StepArgs a, const double* src_fixed, int64_t lds_fixed,
                                                      int pass) {
  using SM = UpdSmem<S, NOUT>;
  constexpr int NC = SM::NC, NT = SM::NT, MT = SM::MT, RT = SM::RT;
  if (NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const SlabInfo si = a.slabs[blockIdx.x];
  const int c = si.chunk, k = a.nb * S, Kt = k + S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp >> 3, tile = warp & 7;
  const double* src = src_fixed;
  int64_t lds = lds_fixed;
  double* slot = a.V + (int64_t)a.nb * a.n * S;
  if (NOUT == 2) {
    int L = 1;
    for (int t = 2; t <= kMaxPass; ++t)
      if (a.flags[kFlagPass + t - 1]) L = t;
    src = (L == 1) ? a.W : slot;
    lds = (L == 1) ? a.ldw : S;
  }
  const int ksteps = (Kt + 15) / 16;
  const int ntiles = (si.rows + RT - 1) / RT;
  const int total = ntiles * ksteps;
  upd_prefetch<S, NOUT>(sm, 0, a, si, src, lds, 0, 0, k, Kt);
  cp_async_commit();
  for (int q = tid; q < Kt; q += 512)
    sm.Fs[q] = (q < k) ? a.colexp[(int64_t)q * a.p + c] : a.srcexp[(int64_t)c * 32 + (q - k)];
  for (int n = tid; n < 64; n += 512) sm.Cx[n] = (n < NC) ? a.coefexp[(int64_t)c * 64 + n] : 0;
  if (tid < 32) sm.Ux[tid] = 0;
  const unsigned* dig = a.coefdig + (int64_t)c * a.coefdig_stride;
  const int mt = tile % MT, nt = tile / MT;
  const int g = lane >> 2, cl = lane & 3;
  float acc[kGroupPairs][4];
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  // slice the float64 tile of iteration it (row tile, 16 columns) into plane buffer pb
  auto slice = [&](int itx, int rb, int pb) {
    const int ks = itx % ksteps;
    for (int pi = tid; pi < RT * 8; pi += 512) {
      const int mtile = pi >> 7, w = pi & 127, ln = w >> 2, rg = w & 3;
      const int mm = (ln >> 2) + 8 * (rg & 1), j = (ln & 3) + 4 * (rg >> 1);
      const int m = mtile * 16 + mm;
      const int q0 = ks * 16 + 2 * j;
      const double x0 = sm.raw[rb][m][2 * j], x1 = sm.raw[rb][m][2 * j + 1];
      const int e0 = q0 < Kt ? sm.Fs[q0] : 0, e1 = q0 + 1 < Kt ? sm.Fs[q0 + 1] : 0;
      oz_store_pair(&sm.Apl[pb][0][mtile][0][0], MT * 128, w, x0, e0, x1, e1, a.flags);
    }
  };
  // pipeline as in k_oz_gram: iteration it+2 streams into the raw buffer of it,
  // it+1 is sliced while it is multiplied; one barrier per iteration
  if (total > 1) upd_prefetch<S, NOUT>(sm, 1, a, si, src, lds, (1 / ksteps) * RT, 1 % ksteps, k, Kt);
  cp_async_commit();
  cp_async_wait1();
  __syncthreads();
  slice(0, 0, 0);
  for (int it = 0; it < total; ++it) {
    const int rt = (it / ksteps) * RT, ks = it % ksteps;
    cp_async_wait0();
    __syncthreads();
    if (it + 2 < total)
      upd_prefetch<S, NOUT>(sm, it & 1, a, si, src, lds, ((it + 2) / ksteps) * RT, (it + 2) % ksteps, k, Kt);
    cp_async_commit();
    if (it + 1 < total) slice(it + 1, (it + 1) & 1, (it + 1) & 1);
    const int pb = it & 1;
    const unsigned* bb = dig + ((int64_t)(ks * NT + nt) * kOzDigits) * 64;
    if (grp == 0)
      group_mma<0, true>(acc, &sm.Apl[pb][0][mt][0][0], MT * 128, bb, 64, lane);
    else
      group_mma<1, true>(acc, &sm.Apl[pb][0][mt][0][0], MT * 128, bb, 64, lane);
    const bool last_k = (ks + 1 == ksteps);
    if (((ks + 1) & 15) == 0 || last_k) {  // exact float32 sums cover <= 256 columns
      int s2[4];
      long long rest[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (grp == 0)
          group_partial<0>(acc, j, s2[j], rest[j]);
        else
          group_partial<1>(acc, j, s2[j], rest[j]);
      }
      if (grp == 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          sm.xs2[tile][lane][j] = s2[j];
          sm.xrest[tile][lane][j] = rest[j];
        }
      }
      __syncthreads();
      if (grp == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          accd[j] += partial_to_double(s2[j] + sm.xs2[tile][lane][j], rest[j] + sm.xrest[tile][lane][j]);
      }
#pragma unroll
      for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    }
    if (last_k && grp == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = mt * 16 + g + ((j >> 1) << 3), n = nt * 8 + 2 * cl + (j & 1);
        const int r = rt + m;
        if (r < si.rows && n < NC) {
          const double d = scale_exp(accd[j], sm.Cx[n] - 1022 - 16);
          const int64_t row = si.row0 + r;
          if (n < S) {
            slot[row * S + n] = d;
            if (NOUT == 2) atomicMax(&sm.Ux[n], bexp(d));
          } else {
            a.U[row * a.ldu + (n - S)] = d;
          }
        }
        accd[j] = 0.0;
      }
    }
  }
  cp_async_wait0();
  if (NOUT == 2) {
    __syncthreads();
    if (tid < S) atomicMax(&a.colexp[(int64_t)(k + tid) * a.p + c], sm.Ux[tid]);
  }
}

// ---------------------------------------------------------------------------
// Digit planes.  A tensor-core basis with s in {8, 16, 32} keeps each local
// panel also as 8 byte planes (StepArgs::dig): the 7 digits oz_split makes
// for a value against the exponent colexp of its column and chunk, and a sign
// byte (0x80 or 0).  A (digit, sign) byte pair is bit for bit the fp16 digit
// oz_pack builds, so the passes expand planes with one byte permute per two
// values and never split a float64 local value again.  Products are bitwise
// the ones of the splitting kernels.

// Two fp16x2 digit words of four values from their digit bytes d and sign bytes g.
__device__ __forceinline__ uint2 dp_expand(unsigned d, unsigned g) {
  return make_uint2(__byte_perm(d, g, 0x5140), __byte_perm(d, g, 0x7362));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void cp_async16z(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(bytes));
}

// 14 mma of one group with A fragments read by ldmatrix (transposed for the
// Gram, whose A operand is the transpose of a [row][column] tile) from fp16
// planes a_plane bytes apart; B fragments as in group_mma.
template <int G, bool TRANS, bool BGLOBAL>
__device__ __forceinline__ void group_mma_ldsm(float (&acc)[kGroupPairs][4], unsigned a_addr, int a_plane,
                                               const unsigned* bpl, int b_stride, int lane) {
  unsigned af[kOzDigits][4], bf[kOzDigits][2];
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t) {
    if (pair_group_has(G, t)) {
      if (TRANS)
        ldsm_x4_t(af[t - 1], a_addr + (t - 1) * a_plane);
      else
        ldsm_x4(af[t - 1], a_addr + (t - 1) * a_plane);
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

// Digit planes of the new panel (slot nb) once stage 2 has fixed its column
// exponents.  One thread per (row, 4 columns).
template <int S>
__global__ void __launch_bounds__(256) k_oz_digitize(StepArgs a) {
  constexpr int G4 = S / 4;
  __shared__ int ex[S];
  const SlabInfo si = a.slabs[blockIdx.x];
  const int k = a.nb * S;
  if (threadIdx.x < S) ex[threadIdx.x] = a.colexp[(int64_t)(k + threadIdx.x) * a.p + si.chunk];
  __syncthreads();
  const double* slot = a.V + (int64_t)a.nb * a.n * S;
  unsigned* dg = reinterpret_cast<unsigned*>(a.dig + (int64_t)a.nb * 8 * a.dstride * S);
  const int64_t pw = a.dstride * S / 4;  // plane stride in words
  for (int i = threadIdx.x; i < si.rows * G4; i += 256) {
    const int r = i / G4, g = i - r * G4;
    const int64_t row = si.row0 + r;
    const double2 v01 = *reinterpret_cast<const double2*>(slot + row * S + 4 * g);
    const double2 v23 = *reinterpret_cast<const double2*>(slot + row * S + 4 * g + 2);
    const double x[4] = {v01.x, v01.y, v23.x, v23.y};
    unsigned hi[4], lo[4], sg[4];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) bad |= oz_split(x[j], ex[4 * g + j], hi[j], lo[j], sg[j]);
    if (bad) oz_status(a.flags, LO_ERR_NONFINITE);
    unsigned* out = dg + (row * S + 4 * g) / 4;
#pragma unroll
    for (int t = 1; t <= kOzDigits; ++t) {
      const bool hw = t <= 3;
      const unsigned bi = hw ? (unsigned)(3 - t) : (unsigned)(7 - t);
      const unsigned sel = bi | ((4u + bi) << 4);
      const unsigned w01 = __byte_perm(hw ? hi[0] : lo[0], hw ? hi[1] : lo[1], sel);
      const unsigned w23 = __byte_perm(hw ? hi[2] : lo[2], hw ? hi[3] : lo[3], sel);
      out[(t - 1) * pw] = __byte_perm(w01, w23, 0x5410);
    }
    out[7 * pw] = (sg[0] >> 24) | (sg[1] >> 16) | (sg[2] >> 8) | sg[3];
  }
}

// Swizzled 16-byte chunk of a [16][CG] fp16 Gram tile: the 8 rows an
// ldmatrix phase reads fall in 8 distinct bank groups.
template <int NCH>
__device__ __forceinline__ int gram_swz(int r, int ch) {
  return NCH >= 8 ? (ch ^ (r & 7)) : (ch ^ ((r >> 1) & 3));
}

template <int S>
struct GramDpSmem {
  static constexpr int NT = (S + 7) / 8, MT = 8 / NT, CG = MT * 16, NC = NT * 8, NP = CG / S, NCH = CG / 8;
  uint8_t stg[2][8][NP][16][S];         // staged byte planes of the group's panels
  uint16_t Apl[2][kOzDigits][16][CG];   // fp16 digits of the A tile, [row][column], swizzled chunks
  double rawB[2][16][S];                // the pass block (float64)
  unsigned Bpl[2][kOzDigits][NT][32][2];
  long long xrest[8][32][4];
  int xs2[8][32][4];
  int Hs[32];
  int Fs[CG];
};

// cp.async of one 16-row step: byte planes of the np_q panels of the group, and
// the pass block's 16 x S float64 tile.  Rows past the slab read as zero.
template <int S>
__device__ __forceinline__ void gram_dp_prefetch(GramDpSmem<S>& sm, int buf, const StepArgs& a, const SlabInfo& si,
                                                 const double* src, int64_t lds, int r0, int b0, int np_q, bool a16) {
  const int tid = threadIdx.x;
  const int left = si.rows - r0;  // valid rows in this step (may exceed 16)
  const int64_t rowbase = si.row0 + r0;
  if (a16) {
    constexpr int U = S;  // 16-byte units of one 16 x S byte tile
    for (int u = tid; u < np_q * 8 * U; u += 512) {
      const int pt = u / U, w = u - pt * U;
      const int pi = pt >> 3, t = pt & 7;
      const int byte0 = w * 16;
      const int valid = min(16, max(0, left * S - byte0));
      const uint8_t* g = a.dig + ((int64_t)((b0 + pi) * 8 + t) * a.dstride + rowbase) * S + (valid > 0 ? byte0 : 0);
      cp_async16z(&sm.stg[buf][t][pi][0][0] + byte0, g, valid);
    }
  } else {  // rows not 16-byte aligned (s = 8 and an odd first row): one 8-byte row at a time
    for (int u = tid; u < np_q * 8 * 16; u += 512) {
      const int pt = u >> 4, r = u & 15;
      const int pi = pt >> 3, t = pt & 7;
      const bool ok = r < left;
      const uint8_t* g = a.dig + ((int64_t)((b0 + pi) * 8 + t) * a.dstride + rowbase + (ok ? r : 0)) * S;
      cp_async8(&sm.stg[buf][t][pi][r][0], g, ok);
    }
  }
  for (int c = tid; c < 16 * S; c += 512) {
    const int r = c / S, l = c - r * S;
    const bool ok = r < left;
    cp_async8(&sm.rawB[buf][r][l], src + (rowbase + (ok ? r : 0)) * lds + l, ok);
  }
}

// Stage-1 Gram partial of one slab and one group of CG columns of [Q_i A] from
// digit planes (same products as k_oz_gram).  The A tile [16 rows][CG columns]
// is expanded into fp16 planes and read transposed by ldmatrix.
template <int S>
__global__ void __launch_bounds__(512, 1) k_oz_gram_dp(StepArgs a, const double* src, int64_t lds, int pass) {
  using SM = GramDpSmem<S>;
  constexpr int NT = SM::NT, MT = SM::MT, CG = SM::CG, NC = SM::NC, NCH = SM::NCH;
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const SlabInfo si = a.slabs[blockIdx.x];
  const int k = a.nb * S, Kt = k + S;
  const int col0 = blockIdx.y * CG;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp >> 3, tile = warp & 7;
  const int np_q = max(0, min(col0 + CG, k) - col0) / S;  // local panels in the group
  const int b0 = col0 / S;
  const bool in_group = (k >= col0 && k < col0 + CG);
  const bool a16 = ((si.row0 * S) & 15) == 0;
  const int nsteps = (si.rows + 15) / 16;
  gram_dp_prefetch<S>(sm, 0, a, si, src, lds, 0, b0, np_q, a16);
  cp_async_commit();
  if (nsteps > 1) gram_dp_prefetch<S>(sm, 1, a, si, src, lds, 16, b0, np_q, a16);
  cp_async_commit();
  if (tid < 32) sm.Hs[tid] = 0;
  // columns past Kt stay zero in both plane buffers
  {
    const int zc0 = max(0, Kt - col0);  // multiple of 8
    const int zw = (CG - zc0) / 4;      // 8-byte words per row
    for (int i = tid; i < 2 * kOzDigits * 16 * zw; i += 512) {
      const int w = i % zw, rest = i / zw, r = rest % 16, bp = rest / 16;
      const int col = zc0 + 4 * w;
      *reinterpret_cast<uint2*>(&sm.Apl[0][0][0][0] + (int64_t)bp * 16 * CG + r * CG +
                                gram_swz<NCH>(r, col >> 3) * 8 + (col & 7)) = make_uint2(0u, 0u);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < si.rows * S; idx += 512) {
    const int r = idx / S, l = idx - r * S;
    atomicMax(&sm.Hs[l], bexp(src[(si.row0 + r) * lds + l]));
  }
  __syncthreads();
  if (blockIdx.y == 0 && tid < S) a.srcexp_slab[(int64_t)blockIdx.x * 32 + tid] = sm.Hs[tid];
  for (int m = tid; m < CG; m += 512) {
    const int col = col0 + m;
    sm.Fs[m] = (col < k) ? a.colexp[(int64_t)col * a.p + si.chunk] : (col < Kt ? sm.Hs[col - k] : 0);
  }
  float acc[kGroupPairs][4];
#pragma unroll
  for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  const int mt = tile % MT, nt = tile / MT;
  // expand the staged step rb into plane buffer pb
  auto expand = [&](int rb, int pb) {
    constexpr int IPP = 4 * S;                 // items (row, 4 columns) per panel
    constexpr int PW = SM::NP * 16 * S / 4;    // staged plane stride in words
    for (int i = tid; i < np_q * IPP; i += 512) {
      const int pi = i / IPP, w = i - pi * IPP;
      const int r = w / (S / 4), g4 = w - r * (S / 4);
      const unsigned* sp = reinterpret_cast<const unsigned*>(&sm.stg[rb][0][pi][r][4 * g4]);
      const unsigned gw = sp[7 * PW];
      const int col = pi * S + 4 * g4;
      uint16_t* dst = &sm.Apl[pb][0][r][gram_swz<NCH>(r, col >> 3) * 8 + (col & 7)];
#pragma unroll
      for (int t = 0; t < kOzDigits; ++t) *reinterpret_cast<uint2*>(dst + t * 16 * CG) = dp_expand(sp[t * PW], gw);
    }
    if (in_group) {  // the pass block's own columns in the A tile, split from float64
      for (int i = tid; i < 8 * S; i += 512) {
        const int r = i / (S / 2), l = 2 * (i - r * (S / 2));
        const int m = k - col0 + l;
        const int widx = (r * CG + gram_swz<NCH>(r, m >> 3) * 8 + (m & 7)) >> 1;
        oz_store_pair(reinterpret_cast<unsigned*>(&sm.Apl[pb][0][0][0]), 8 * CG, widx, sm.rawB[rb][r][l], sm.Fs[m],
                      sm.rawB[rb][r][l + 1], sm.Fs[m + 1], a.flags);
      }
    }
    // B: value pairs of the block's columns, in fragment order
    for (int pi = tid; pi < 8 * NC; pi += 512) {
      const int ntile = pi >> 6, w = pi & 63, ln = w >> 1, rg = w & 1;
      const int n = ntile * 8 + (ln >> 2), j = (ln & 3) + 4 * rg;
      double x0 = 0.0, x1 = 0.0;
      if (n < S) {
        x0 = sm.rawB[rb][2 * j][n];
        x1 = sm.rawB[rb][2 * j + 1][n];
      }
      const int e = (n < S) ? sm.Hs[n] : 0;
      oz_store_pair(&sm.Bpl[pb][0][ntile][0][0], NT * 64, w, x0, e, x1, e, a.flags);
    }
  };
  // ldmatrix.trans addresses of this lane: matrix q = lane / 8 covers rows
  // 8 (q / 2) .. +7 and the 8 columns of chunk 2 mt + q % 2
  unsigned a_off;
  {
    const int q = lane >> 3, r = ((q >> 1) << 3) + (lane & 7), ch = 2 * mt + (q & 1);
    a_off = (unsigned)((r * CG + gram_swz<NCH>(r, ch) * 8) * 2);
  }
  const unsigned apl0 = (unsigned)__cvta_generic_to_shared(&sm.Apl[0][0][0][0]);
  constexpr unsigned kPlaneBytes = 16 * CG * 2, kBufBytes = kOzDigits * kPlaneBytes;
  // flush: exact float32 sums cover 16 steps (256 rows); the groups' integer
  // partials meet in shared memory and group 0 accumulates in float64
  auto flush = [&]() {
    int s2[4];
    long long rest[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (grp == 0)
        group_partial<0>(acc, j, s2[j], rest[j]);
      else
        group_partial<1>(acc, j, s2[j], rest[j]);
    }
    if (grp == 1) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sm.xs2[tile][lane][j] = s2[j];
        sm.xrest[tile][lane][j] = rest[j];
      }
    }
    __syncthreads();
    if (grp == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        accd[j] += partial_to_double(s2[j] + sm.xs2[tile][lane][j], rest[j] + sm.xrest[tile][lane][j]);
    }
#pragma unroll
    for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  };
  cp_async_wait1();
  __syncthreads();
  expand(0, 0);
  for (int st = 0; st < nsteps; ++st) {
    cp_async_wait0();
    __syncthreads();
    if (st + 2 < nsteps) gram_dp_prefetch<S>(sm, st & 1, a, si, src, lds, 16 * (st + 2), b0, np_q, a16);
    cp_async_commit();
    if (st + 1 < nsteps) expand((st + 1) & 1, (st + 1) & 1);
    const int pb = st & 1;
    const unsigned aa = apl0 + pb * kBufBytes + a_off;
    if (grp == 0)
      group_mma_ldsm<0, true, false>(acc, aa, kPlaneBytes, &sm.Bpl[pb][0][nt][0][0], NT * 64, lane);
    else
      group_mma_ldsm<1, true, false>(acc, aa, kPlaneBytes, &sm.Bpl[pb][0][nt][0][0], NT * 64, lane);
    if (((st + 1) & 15) == 0 && st + 1 < nsteps) flush();
  }
  cp_async_wait0();
  flush();
  if (grp == 0) {
    const int g = lane >> 2, c = lane & 3;
    double* out = a.part + (int64_t)blockIdx.x * a.Kmax * S;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = mt * 16 + g + ((j >> 1) << 3), n = nt * 8 + 2 * c + (j & 1);
      const int col = col0 + m;
      if (col < Kt && n < S) out[(int64_t)col * S + n] = scale_exp(accd[j], sm.Fs[m] + sm.Hs[n] - 2044 - 16);
    }
  }
}

// out = [Q_i A] Coef for one slab from digit planes (same products as
// k_oz_update).  The A tile [RT rows][16 columns] of a step is expanded into
// fp16 planes with 16-byte chunks swizzled by bit 2 of the row.
template <int S, int NOUT>
struct UpdDpSmem {
  static constexpr int NC = NOUT * S, NT = (NC + 7) / 8, MT = (8 / NT) > 0 ? 8 / NT : 1, RT = MT * 16;
  uint8_t stg[2][8][RT][16];            // staged byte planes of the step's local columns
  uint16_t Apl[2][kOzDigits][RT][16];   // fp16 digits of the A tile
  double raw[2][RT][17];                // the pass block's columns of the step (float64)
  long long xrest[8][32][4];
  int xs2[8][32][4];
  int Fs[1024];
  int Cx[64];
  int Ux[32];
};

__device__ __forceinline__ int upd_swz(int r, int ch) { return ch ^ ((r >> 2) & 1); }

template <int S, int NOUT>
__device__ __forceinline__ void upd_dp_prefetch(UpdDpSmem<S, NOUT>& sm, int buf, const StepArgs& a,
                                                const SlabInfo& si, const double* src, int64_t lds, int rt, int ks,
                                                int k, int Kt) {
  constexpr int RT = UpdDpSmem<S, NOUT>::RT;
  const int tid = threadIdx.x;
  const int64_t rowbase = si.row0 + rt;
  const int left = si.rows - rt;
  const int q0 = ks * 16;
  if (S >= 16 && q0 < k) {  // both halves in one panel: one 16-byte row per plane
    const int b = q0 / S, jo = q0 - b * S;
    for (int u = tid; u < 8 * RT; u += 512) {
      const int t = u / RT, r = u - t * RT;
      const bool ok = r < left;
      const uint8_t* g = a.dig + ((int64_t)(b * 8 + t) * a.dstride + rowbase + (ok ? r : 0)) * S + jo;
      cp_async16(&sm.stg[buf][t][r][0], g, ok);
    }
    return;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int qh = q0 + 8 * h;
    if (qh < k) {  // s = 8: one panel per half, 8-byte rows
      const int b = qh / S, jo = qh - b * S;
      for (int u = tid; u < 8 * RT; u += 512) {
        const int t = u / RT, r = u - t * RT;
        const bool ok = r < left;
        const uint8_t* g = a.dig + ((int64_t)(b * 8 + t) * a.dstride + rowbase + (ok ? r : 0)) * S + jo;
        cp_async8(&sm.stg[buf][t][r][8 * h], g, ok);
      }
    } else if (qh < Kt) {  // the pass block's columns
      for (int u = tid; u < 8 * RT; u += 512) {
        const int r = u >> 3, j = u & 7;
        const bool ok = r < left;
        cp_async8(&sm.raw[buf][r][8 * h + j], src + (rowbase + (ok ? r : 0)) * lds + (qh - k + j), ok);
      }
    }
  }
}

template <int S, int NOUT>
__global__ void __launch_bounds__(512, 1) k_oz_update_dp(StepArgs a, const double* src_fixed, int64_t lds_fixed,
                                                         int pass) {
  using SM = UpdDpSmem<S, NOUT>;
  constexpr int NC = SM::NC, NT = SM::NT, MT = SM::MT, RT = SM::RT;
  if (NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const SlabInfo si = a.slabs[blockIdx.x];
  const int c = si.chunk, k = a.nb * S, Kt = k + S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp >> 3, tile = warp & 7;
  const double* src = src_fixed;
  int64_t lds = lds_fixed;
  double* slot = a.V + (int64_t)a.nb * a.n * S;
  if (NOUT == 2) {
    int L = 1;
    for (int t = 2; t <= kMaxPass; ++t)
      if (a.flags[kFlagPass + t - 1]) L = t;
    src = (L == 1) ? a.W : slot;
    lds = (L == 1) ? a.ldw : S;
  }
  const int ksteps = (Kt + 15) / 16;
  const int ntiles = (si.rows + RT - 1) / RT;
  const int total = ntiles * ksteps;
  upd_dp_prefetch<S, NOUT>(sm, 0, a, si, src, lds, 0, 0, k, Kt);
  cp_async_commit();
  if (total > 1) upd_dp_prefetch<S, NOUT>(sm, 1, a, si, src, lds, (1 / ksteps) * RT, 1 % ksteps, k, Kt);
  cp_async_commit();
  for (int q = tid; q < Kt; q += 512)
    sm.Fs[q] = (q < k) ? a.colexp[(int64_t)q * a.p + c] : a.srcexp[(int64_t)c * 32 + (q - k)];
  for (int n = tid; n < 64; n += 512) sm.Cx[n] = (n < NC) ? a.coefexp[(int64_t)c * 64 + n] : 0;
  if (tid < 32) sm.Ux[tid] = 0;
  const unsigned* cdig = a.coefdig + (int64_t)c * a.coefdig_stride;
  const int mt = tile % MT, nt = tile / MT;
  const int g = lane >> 2, cl = lane & 3;
  float acc[kGroupPairs][4];
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  // expand iteration itx (staged in rb) into plane buffer pb: one item = (row, 4 columns)
  auto expand = [&](int itx, int rb, int pb) {
    const int q0 = (itx % ksteps) * 16;
    for (int i = tid; i < RT * 4; i += 512) {
      const int r = i >> 2, g4 = i & 3, h = g4 >> 1;
      const int q = q0 + 4 * g4;
      uint16_t* dst = &sm.Apl[pb][0][r][upd_swz(r, h) * 8 + 4 * (g4 & 1)];
      if (q < k) {
        const unsigned* sp = reinterpret_cast<const unsigned*>(&sm.stg[rb][0][r][4 * g4]);
        const unsigned gw = sp[7 * RT * 4];
#pragma unroll
        for (int t = 0; t < kOzDigits; ++t) *reinterpret_cast<uint2*>(dst + t * RT * 16) = dp_expand(sp[t * RT * 4], gw);
      } else if (q < Kt) {
        const double* xr = &sm.raw[rb][r][4 * g4];
        unsigned* base = reinterpret_cast<unsigned*>(dst);
        oz_store_pair(base, RT * 8, 0, xr[0], sm.Fs[q], xr[1], sm.Fs[q + 1], a.flags);
        oz_store_pair(base, RT * 8, 1, xr[2], sm.Fs[q + 2], xr[3], sm.Fs[q + 3], a.flags);
      } else {
#pragma unroll
        for (int t = 0; t < kOzDigits; ++t) *reinterpret_cast<uint2*>(dst + t * RT * 16) = make_uint2(0u, 0u);
      }
    }
  };
  // ldmatrix addresses of this lane: matrix q = lane / 8 covers rows 8 (q % 2) .. +7
  // of the M-tile and the 8 columns of chunk q / 2
  unsigned a_off;
  {
    const int q = lane >> 3, r = mt * 16 + ((q & 1) << 3) + (lane & 7), ch = q >> 1;
    a_off = (unsigned)((r * 16 + upd_swz(r, ch) * 8) * 2);
  }
  const unsigned apl0 = (unsigned)__cvta_generic_to_shared(&sm.Apl[0][0][0][0]);
  constexpr unsigned kPlaneBytes = RT * 16 * 2, kBufBytes = kOzDigits * kPlaneBytes;
  cp_async_wait1();
  __syncthreads();
  expand(0, 0, 0);
  for (int it = 0; it < total; ++it) {
    const int rt = (it / ksteps) * RT, ks = it % ksteps;
    cp_async_wait0();
    __syncthreads();
    if (it + 2 < total)
      upd_dp_prefetch<S, NOUT>(sm, it & 1, a, si, src, lds, ((it + 2) / ksteps) * RT, (it + 2) % ksteps, k, Kt);
    cp_async_commit();
    if (it + 1 < total) expand(it + 1, (it + 1) & 1, (it + 1) & 1);
    const int pb = it & 1;
    const unsigned aa = apl0 + pb * kBufBytes + a_off;
    const unsigned* bb = cdig + ((int64_t)(ks * NT + nt) * kOzDigits) * 64;
    if (grp == 0)
      group_mma_ldsm<0, false, true>(acc, aa, kPlaneBytes, bb, 64, lane);
    else
      group_mma_ldsm<1, false, true>(acc, aa, kPlaneBytes, bb, 64, lane);
    const bool last_k = (ks + 1 == ksteps);
    if (((ks + 1) & 15) == 0 || last_k) {  // exact float32 sums cover <= 256 columns
      int s2[4];
      long long rest[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (grp == 0)
          group_partial<0>(acc, j, s2[j], rest[j]);
        else
          group_partial<1>(acc, j, s2[j], rest[j]);
      }
      if (grp == 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          sm.xs2[tile][lane][j] = s2[j];
          sm.xrest[tile][lane][j] = rest[j];
        }
      }
      __syncthreads();
      if (grp == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          accd[j] += partial_to_double(s2[j] + sm.xs2[tile][lane][j], rest[j] + sm.xrest[tile][lane][j]);
      }
#pragma unroll
      for (int i = 0; i < kGroupPairs; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    }
    if (last_k && grp == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = mt * 16 + g + ((j >> 1) << 3), n = nt * 8 + 2 * cl + (j & 1);
        const int r = rt + m;
        if (r < si.rows && n < NC) {
          const double d = scale_exp(accd[j], sm.Cx[n] - 1022 - 16);
          const int64_t row = si.row0 + r;
          if (n < S) {
            slot[row * S + n] = d;
            if (NOUT == 2) atomicMax(&sm.Ux[n], bexp(d));
          } else {
            a.U[row * a.ldu + (n - S)] = d;
          }
        }
        accd[j] = 0.0;
      }
    }
  }
  cp_async_wait0();
  if (NOUT == 2) {
    __syncthreads();
    if (tid < S) atomicMax(&a.colexp[(int64_t)(k + tid) * a.p + c], sm.Ux[tid]);
  }
}

template <int S>
cudaError_t gram_for(const StepArgs& a, int pass, cudaStream_t st) {
  constexpr int NT = (S + 7) / 8, MT = 8 / NT, CG = MT * 16;
  const int Kt = a.nb * S + S;
  dim3 grid(a.nslab, (Kt + CG - 1) / CG);
  const double* src = (pass == 1) ? a.W : a.V + (int64_t)a.nb * a.n * S;
  const int64_t lds = (pass == 1) ? a.ldw : S;
  if constexpr (S >= 8) {
    if (a.dig) {
      k_oz_gram_dp<S><<<grid, 512, sizeof(GramDpSmem<S>), st>>>(a, src, lds, pass);
      return cudaGetLastError();
    }
  }
  k_oz_gram<S><<<grid, 512, sizeof(GramSmem<S>), st>>>(a, src, lds, pass);
  return cudaGetLastError();
}

template <int S, int NOUT>
size_t coef_smem(const StepArgs& a) {
  const int k = a.nb * S, Kt = k + S;
  return sizeof(double) * ((size_t)Kt * NOUT * S + (size_t)k * S) + sizeof(int) * 64;
}

template <int S>
cudaError_t ypass_for(const StepArgs& a, int pass, cudaStream_t st) {
  k_oz_coef<S, 1><<<a.p, 256, coef_smem<S, 1>(a), st>>>(a, pass);
  const double* src = (pass == 2) ? a.W : a.V + (int64_t)a.nb * a.n * S;
  const int64_t lds = (pass == 2) ? a.ldw : S;
  if constexpr (S >= 8) {
    if (a.dig) {
      k_oz_update_dp<S, 1><<<a.nslab, 512, sizeof(UpdDpSmem<S, 1>), st>>>(a, src, lds, pass);
      return cudaGetLastError();
    }
  }
  k_oz_update<S, 1><<<a.nslab, 512, sizeof(UpdSmem<S, 1>), st>>>(a, src, lds, pass);
  return cudaGetLastError();
}

template <int S>
cudaError_t stage2_for(const StepArgs& a, cudaStream_t st) {
  k_oz_coef<S, 2><<<a.p, 256, coef_smem<S, 2>(a), st>>>(a, 0);
  if constexpr (S >= 8) {
    if (a.dig) {
      k_oz_update_dp<S, 2><<<a.nslab, 512, sizeof(UpdDpSmem<S, 2>), st>>>(a, nullptr, 0, 0);
      return cudaGetLastError();
    }
  }
  k_oz_update<S, 2><<<a.nslab, 512, sizeof(UpdSmem<S, 2>), st>>>(a, nullptr, 0, 0);
  return cudaGetLastError();
}

template <int S>
cudaError_t digitize_for(const StepArgs& a, cudaStream_t st) {
  if constexpr (S >= 8) {
    k_oz_digitize<S><<<a.nslab, 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

bool g_oz_attr = false;

}  // namespace

bool oz_supported(int s) { return s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32; }
bool oz_planes_supported(int s) { return s == 8 || s == 16 || s == 32; }

cudaError_t oz_set_attrs() {
  if (g_oz_attr) return cudaSuccess;
  const int big = 200 * 1024;
  cudaError_t e;
#define LO_OZ_ATTR(S)                                                                                  \
  if ((e = cudaFuncSetAttribute(k_oz_coef<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))   \
    return e;                                                                                          \
  if ((e = cudaFuncSetAttribute(k_oz_coef<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))   \
    return e;                                                                                          \
  if ((e = cudaFuncSetAttribute(k_oz_gram<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))      \
    return e;                                                                                          \
  if ((e = cudaFuncSetAttribute(k_oz_update<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
    return e;                                                                                          \
  if ((e = cudaFuncSetAttribute(k_oz_update<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  LO_OZ_ATTR(1)
  LO_OZ_ATTR(2)
  LO_OZ_ATTR(4)
  LO_OZ_ATTR(8)
  LO_OZ_ATTR(16)
  LO_OZ_ATTR(32)
#undef LO_OZ_ATTR
#define LO_OZ_ATTR_DP(S)                                                                                  \
  if ((e = cudaFuncSetAttribute(k_oz_gram_dp<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))      \
    return e;                                                                                             \
  if ((e = cudaFuncSetAttribute(k_oz_update_dp<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
    return e;                                                                                             \
  if ((e = cudaFuncSetAttribute(k_oz_update_dp<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  LO_OZ_ATTR_DP(8)
  LO_OZ_ATTR_DP(16)
  LO_OZ_ATTR_DP(32)
#undef LO_OZ_ATTR_DP
  g_oz_attr = true;
  return cudaSuccess;
}

#define LO_OZ_DISPATCH(CALL)       \
  switch (a.s) {                   \
    case 1: return CALL(1);        \
    case 2: return CALL(2);        \
    case 4: return CALL(4);        \
    case 8: return CALL(8);        \
    case 16: return CALL(16);      \
    case 32: return CALL(32);      \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_oz_gram(const StepArgs& a, int pass, cudaStream_t st) {
#define CALL(S) gram_for<S>(a, pass, st)
  LO_OZ_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_oz_ypass(const StepArgs& a, int pass, cudaStream_t st) {
#define CALL(S) ypass_for<S>(a, pass, st)
  LO_OZ_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_oz_stage2(const StepArgs& a, cudaStream_t st) {
#define CALL(S) stage2_for<S>(a, st)
  LO_OZ_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_oz_digitize(const StepArgs& a, cudaStream_t st) {
#define CALL(S) digitize_for<S>(a, st)
  LO_OZ_DISPATCH(CALL)
#undef CALL
}

}  // namespace lo

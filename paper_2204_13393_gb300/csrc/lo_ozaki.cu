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
#include "lo_oz_common.cuh"

namespace lo {
namespace {

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
//
// MODE 1 writes the coefficients instead as tcgen05 B-operand images for
// k_umma_update: per output split z (NB = min(NOUT*S, 16) columns) and 16-row
// step ks, a K-major no-swizzle tile of R = round16(7 NB) rows x 16 K, row
// (u - 1) NB + n holding digit u of column z NB + n (rows past 7 NB zero):
// byte ((row % 8) * 16 + (row / 8) * 256 + (kk % 8) * 2 + (kk / 8) * 128) of
// image (z * ceil(Kmax / 16) + ks), images R * 32 bytes apart
// (umma_coef_image, shared with apply_Q's coefficient kernel).
//
// MODE 2 (no prior blocks, Kt = S) writes one image for k_umma_update0 whose
// K index is (digit t of the block, block column) and whose N index is
// (digit-sum class j, output column): row j NC + n, column kk = (t - 1) S + q
// holds digit v_j - t of coefficient (q, n) when that digit exists, where
// v_j = j + 2 for j < 6 and v = 8 for j = 6 (t in pair group 0) and j = 7 (t
// in pair group 1); K-major no-swizzle, KK = round16(7 S) columns, byte
// ((row % 8) * 16 + (row / 8) * (KK / 8) * 128 + (kk % 8) * 2 + (kk / 8) * 128).
template <int S, int NOUT, int MODE>
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
  if constexpr (MODE == 2) {
    constexpr int KK = (7 * S + 15) / 16 * 16, SBO = (KK / 8) * 128, BYTES = NC * SBO;  // 8 NC rows
    unsigned char* img = reinterpret_cast<unsigned char*>(dig);
    for (int i = tid; i < BYTES / 16; i += 256) reinterpret_cast<uint4*>(img)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // one item = (block column q, output column n): its 7 digits, placed
    // wherever digit u = v_j - t of a class j meets digit t of the block
    for (int it = tid; it < S * NC; it += 256) {
      const int q = it / NC, n = it - q * NC;
      unsigned h, l, g;
      if (oz_split(Cf[q * NC + n], Gs[n], h, l, g)) oz_status(a.flags, LO_ERR_NONFINITE);
      const unsigned sign = (g >> 16) & 0x8000u;
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) {
        const int kk = (t - 1) * S + q;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int v = j < 6 ? j + 2 : 8;
          const int u = v - t;
          if (u < 1 || u > kOzDigits) continue;
          if (j == 6 && !pair_group_has(0, t)) continue;
          if (j == 7 && !pair_group_has(1, t)) continue;
          const unsigned byte = (u <= 3) ? ((h >> (8 * (3 - u))) & 0xFFu) : ((l >> (8 * (7 - u))) & 0xFFu);
          const int row = j * NC + n;
          *reinterpret_cast<unsigned short*>(img + (row & 7) * 16 + (row >> 3) * SBO + (kk & 7) * 2 + (kk >> 3) * 128) =
              (unsigned short)(sign | byte);
        }
      }
    }
    for (int n = tid; n < NC; n += 256) a.coefexp[(int64_t)c * 64 + n] = Gs[n];
    if (NOUT == 1)
      for (int i = tid; i < (a.chunk_slab0[c + 1] - a.chunk_slab0[c]) * 32; i += 256)
        a.srcexp_slab[(int64_t)a.chunk_slab0[c] * 32 + i] = 0;
    return;
  }
  if constexpr (MODE == 1) {
    umma_coef_image<NC>(Cf, Gs, Kt, (a.Kmax + 15) / 16, reinterpret_cast<unsigned char*>(dig), a.flags);
    for (int n = tid; n < NC; n += 256) a.coefexp[(int64_t)c * 64 + n] = Gs[n];
    // the new iterate's exponents per slab are maxima k_umma_update accumulates
    if (NOUT == 1)
      for (int i = tid; i < (a.chunk_slab0[c + 1] - a.chunk_slab0[c]) * 32; i += 256)
        a.srcexp_slab[(int64_t)a.chunk_slab0[c] * 32 + i] = 0;
    return;
  } else {
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

template <int S>
cudaError_t gram_for(const StepArgs& a, int pass, cudaStream_t st) {
  if (umma_enabled(a)) return launch_umma_gram(a, pass, st);
  if (umma0_enabled(a)) return launch_umma_gram0(a, pass, st);
  constexpr int NT = (S + 7) / 8, MT = 8 / NT, CG = MT * 16;
  const int Kt = a.nb * S + S;
  dim3 grid(a.nslab, (Kt + CG - 1) / CG);
  const double* src = (pass == 1) ? a.W : a.V + (int64_t)a.nb * a.n * S;
  const int64_t lds = (pass == 1) ? a.ldw : S;
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
  if (umma_enabled(a)) {
    cudaError_t e = launch_oz_coef_umma(a, 1, pass, 1, st);
    return e ? e : launch_umma_update(a, 1, pass, st);
  }
  if (umma0_enabled(a)) {
    cudaError_t e = launch_oz_coef_umma(a, 1, pass, 2, st);
    return e ? e : launch_umma_update0(a, 1, pass, st);
  }
  k_oz_coef<S, 1, 0><<<a.p, 256, coef_smem<S, 1>(a), st>>>(a, pass);
  const double* src = (pass == 2) ? a.W : a.V + (int64_t)a.nb * a.n * S;
  const int64_t lds = (pass == 2) ? a.ldw : S;
  k_oz_update<S, 1><<<a.nslab, 512, sizeof(UpdSmem<S, 1>), st>>>(a, src, lds, pass);
  return cudaGetLastError();
}

template <int S>
cudaError_t stage2_for(const StepArgs& a, cudaStream_t st) {
  if (umma_enabled(a)) {
    cudaError_t e = launch_oz_coef_umma(a, 2, 0, 1, st);
    return e ? e : launch_umma_update(a, 2, 0, st);
  }
  if (umma0_enabled(a)) {
    cudaError_t e = launch_oz_coef_umma(a, 2, 0, 2, st);
    return e ? e : launch_umma_update0(a, 2, 0, st);
  }
  k_oz_coef<S, 2, 0><<<a.p, 256, coef_smem<S, 2>(a), st>>>(a, 0);
  k_oz_update<S, 2><<<a.nslab, 512, sizeof(UpdSmem<S, 2>), st>>>(a, nullptr, 0, 0);
  return cudaGetLastError();
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
  if ((e = cudaFuncSetAttribute(k_oz_coef<S, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
    return e;                                                                                          \
  if ((e = cudaFuncSetAttribute(k_oz_coef<S, 2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
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
#define LO_OZ_ATTR_UMMA(S)                                                                                 \
  if ((e = cudaFuncSetAttribute(k_oz_coef<S, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) \
    return e;                                                                                              \
  if ((e = cudaFuncSetAttribute(k_oz_coef<S, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  LO_OZ_ATTR_UMMA(8)
  LO_OZ_ATTR_UMMA(16)
  LO_OZ_ATTR_UMMA(32)
#undef LO_OZ_ATTR_UMMA
  if ((e = cudaFuncSetAttribute(k_oz_coef<8, 1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_oz_coef<8, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_oz_coef<16, 1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_oz_coef<16, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;

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

cudaError_t launch_oz_coef_umma(const StepArgs& a, int nout, int pass, int mode, cudaStream_t st) {
  if (mode == 2) {
    switch (a.s * 4 + nout) {
#define LO_COEF_UMMA0(S, NOUT)                                                    \
  case S * 4 + NOUT:                                                              \
    k_oz_coef<S, NOUT, 2><<<a.p, 256, coef_smem<S, NOUT>(a), st>>>(a, pass);     \
    return cudaGetLastError();
      LO_COEF_UMMA0(8, 1)
      LO_COEF_UMMA0(8, 2)
      LO_COEF_UMMA0(16, 1)
      LO_COEF_UMMA0(16, 2)
#undef LO_COEF_UMMA0
      default:
        return cudaErrorInvalidValue;
    }
  }
  switch (a.s * 4 + nout) {
#define LO_COEF_UMMA(S, NOUT)                                                                \
  case S * 4 + NOUT:                                                                         \
    k_oz_coef<S, NOUT, 1><<<a.p, 256, coef_smem<S, NOUT>(a), st>>>(a, pass);                \
    return cudaGetLastError();
    LO_COEF_UMMA(8, 1)
    LO_COEF_UMMA(8, 2)
    LO_COEF_UMMA(16, 1)
    LO_COEF_UMMA(16, 2)
    LO_COEF_UMMA(32, 1)
    LO_COEF_UMMA(32, 2)
#undef LO_COEF_UMMA
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace lo

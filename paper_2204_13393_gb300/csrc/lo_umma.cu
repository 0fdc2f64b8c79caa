// The two O(n) products of a step (the stage-1 Gram partial of Alg. 7 and the
// assembly products of Sec. 4.1) on the 5th-generation tensor cores, over the
// digit planes that a tensor-core basis keeps for its prior panels.
//
// Digit arithmetic as in lo_ozaki.cu: each float64 value is split exactly into
// 7 8-bit digits aligned to its column's largest exponent, encoded as fp16
// subnormals; the 28 digit pairs (t, u) with t + u <= 8 are multiplied with
// float32 accumulation, exact for up to 256 products, and recombined in 64-bit
// integers.  Results are bit for bit those of the mma.sync kernels.
//
// GB300 mapping:
//   * one thread issues tcgen05.mma (M = 128, K = 16, kind::f16) with both
//     operands in shared memory and the accumulators in tensor memory (TMEM);
//     the pairs of one digit t of [Q_i A] share one MMA whose B operand stacks
//     the digit planes u = 1 .. 8 - t of the other factor along N;
//   * the digit planes of prior panels arrive by TMA (cp.async.bulk.tensor)
//     into a 4-stage ring tracked by mbarriers; the coefficient images of the
//     assembly arrive by cp.async.bulk on the same barriers;
//   * digit bytes are expanded to fp16 with one byte permute per two values
//     (a digit byte and a sign byte form the fp16 subnormal), straight into
//     the canonical no-swizzle UMMA layouts: K-major for the Gram (the rows
//     of a 16-row tile are contiguous per column in the planes), MN-major for
//     the assembly;
//   * the pass block itself (float64) is split on the fly.
//
// Digit-plane layout (global): panel b, plane t (0..6: digit t + 1, 7: sign
// byte 0x80 / 0), 16-row tile tau of the slab tiling, column j, row rho:
//   dig[(((b * 8 + t) * dtiles + tau) * s + j) * 16 + rho]
// Every slab starts a new tile, so each 16-row step of a kernel is one tile.
//
// Every wait on an mbarrier is bounded: on timeout the kernel records
// LO_ERR_TIMEOUT, stops issuing tensor-core work and drains what it issued.
#include <cfloat>
#include <cstdint>

#include "lo_internal.h"
#include "lo_oz_common.cuh"

namespace lo {
namespace {

constexpr int kUmmaThreads = 256;
constexpr int kStages = 4;            // TMA ring depth
constexpr int kStageBytes = 16384;    // digit bytes of one step (both kernels)
constexpr int kAPlaneBytes = 4096;    // one 128 x 16 fp16 operand tile
constexpr long long kWaitCycles = 500000000ll;   // ~0.25 s at 2 GHz

__host__ __device__ constexpr int umma_round16(int x) { return (x + 15) / 16 * 16; }
// N of the MMA of digit t (pairs u = 1 .. 8 - t, nb columns each), and its
// first TMEM column.
__host__ __device__ constexpr int umma_nt(int t, int nb) { return umma_round16((8 - t) * nb); }
__host__ __device__ constexpr int umma_col(int t, int nb) {
  int c = 0;
  for (int i = 1; i < t; ++i) c += umma_nt(i, nb);
  return c;
}
__host__ __device__ constexpr int umma_tcols(int nb) { return umma_col(8, nb) <= 256 ? 256 : 512; }

// --- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start, leading (K-direction) and
// stride (M/N-direction) byte offsets between 8 x 16-byte core matrices.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: fp16 A and B, float32 D, M x N.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mb, uint32_t parity) {
  uint32_t done;
  asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
               : "=r"(done)
               : "r"(mb), "r"(parity)
               : "memory");
  return done != 0;
}
// Bounded wait for the completion of phase `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity) {
  if (mbar_try(mb, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(mb, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mb)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mb)
               : "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t mb) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// TMEM loads, 32 lanes x N columns (32-bit): lane i of the warp gets row
// (lane base + i), columns [col, col + N).
__device__ __forceinline__ void tmem_ld4(uint32_t ta, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(ta));
}
__device__ __forceinline__ void tmem_ld8(uint32_t ta, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
}
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t ta, uint32_t (&r)[N]) {
  if constexpr (N == 4) {
    tmem_ld4(ta, r);
  } else {
    static_assert(N == 8, "tmem_ld: 4 or 8 columns");
    tmem_ld8(ta, r);
  }
}

// Per-CTA control block at the end of dynamic shared memory.
struct UmmaCtl {
  uint64_t full[kStages];   // TMA ring
  uint64_t mmad[2];         // MMAs of the operand buffer done
  uint32_t tslot;           // TMEM base written by tcgen05.alloc
  int abort;                // a bounded wait gave up: no further TMA or MMA is issued
  int issued;               // steps whose loads have been issued
  int Hs[32];               // column exponents of the pass block (this slab)
  int Fs[1024];             // column exponents of [Q_i A]
  int Cx[64];               // exponents of the coefficient columns
  int Ux[32];               // new panel's column exponents (stage 2)
};

__device__ __forceinline__ void umma_timeout(UmmaCtl& c, int* flags) {
  c.abort = 1;
  atomicOr(&flags[kFlagStatus], 1 << (int)LO_ERR_TIMEOUT);
}
// A timeout anywhere in the step stops every tcgen05 CTA that sees it.
__device__ __forceinline__ bool umma_timed_out(const int* flags) {
  return (*reinterpret_cast<const volatile int*>(&flags[kFlagStatus]) & (1 << (int)LO_ERR_TIMEOUT)) != 0;
}

// Recombination of the pair sums of one output from its per-pair float32
// accumulators: as group_partial in both pair groups, added as integers.
struct PairSums {
  int s[7];        // S_2 .. S_7 (v - 2)
  int s8[2];       // S_8 of pair group 0 and 1
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 7; ++i) s[i] = 0;
    s8[0] = s8[1] = 0;
  }
  __device__ __forceinline__ void add(int t, int u, float x) {
    const int d = __float2int_rn(x * 0x1p48f);
    if (t + u == 8)
      s8[pair_group_has(0, t) ? 0 : 1] += d;
    else
      s[t + u - 2] += d;
  }
  __device__ __forceinline__ double value() const {
    long long rest = (long long)s[1] * (1LL << 37);
    rest += (long long)s[2] * (1LL << 29);
    rest += (long long)s[3] * (1LL << 21);
    rest += (long long)s[4] * (1LL << 13);
    rest += (long long)s[5] * (1LL << 5);
    rest += (long long)((s8[0] + 4) >> 3) + (long long)((s8[1] + 4) >> 3);
    return partial_to_double(s[0], rest);
  }
};

// Read the pair accumulators of NW consecutive output columns (starting at
// column n0 of every pair block) for this thread's TMEM lane and add their
// recombined values to acc[0 .. NW).
template <int NB, int NW>
__device__ __forceinline__ void umma_drain(uint32_t tlane, int n0, double* acc) {
  PairSums ps[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) ps[j].clear();
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t) {
    uint32_t r[8 - 1][NW];
#pragma unroll
    for (int u = 1; u <= 8 - t; ++u) tmem_ld<NW>(tlane + (uint32_t)(umma_col(t, NB) + (u - 1) * NB + n0), r[u - 1]);
    tmem_wait_ld();
#pragma unroll
    for (int u = 1; u <= 8 - t; ++u)
#pragma unroll
      for (int j = 0; j < NW; ++j) ps[j].add(t, u, __uint_as_float(r[u - 1][j]));
  }
#pragma unroll
  for (int j = 0; j < NW; ++j) acc[j] += ps[j].value();
}

// Expand 16 digit bytes d (rows rho = 0..15 of one column) with their sign
// bytes g into 16 fp16 digits: out[0..3] rows 0..7, out[4..7] rows 8..15.
__device__ __forceinline__ void expand16(const uint4& d, const uint4& g, uint4& lo, uint4& hi) {
  lo.x = __byte_perm(d.x, g.x, 0x5140); lo.y = __byte_perm(d.x, g.x, 0x7362);
  lo.z = __byte_perm(d.y, g.y, 0x5140); lo.w = __byte_perm(d.y, g.y, 0x7362);
  hi.x = __byte_perm(d.z, g.z, 0x5140); hi.y = __byte_perm(d.z, g.z, 0x7362);
  hi.z = __byte_perm(d.w, g.w, 0x5140); hi.w = __byte_perm(d.w, g.w, 0x7362);
}

// Split 8 float64 values x[0..7] (8 consecutive rows of one column) against
// exponent e and store their fp16 digits as one 16-byte row of each of the 7
// planes at dst + t * kAPlaneBytes.
__device__ __forceinline__ void split8_store(const double* x, int e, unsigned char* dst, int* flags) {
  unsigned w[kOzDigits][4];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned h0, l0, s0, h1, l1, s1;
    bad |= oz_split(x[2 * i], e, h0, l0, s0);
    bad |= oz_split(x[2 * i + 1], e, h1, l1, s1);
    const unsigned sb = (s0 >> 16) | s1;
#pragma unroll
    for (int t = 1; t <= kOzDigits; ++t) w[t - 1][i] = oz_pack(t, h0, l0, h1, l1, sb);
  }
  if (bad) oz_status(flags, LO_ERR_NONFINITE);
#pragma unroll
  for (int t = 0; t < kOzDigits; ++t)
    *reinterpret_cast<uint4*>(dst + t * kAPlaneBytes) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// ---------------------------------------------------------------------------
// Digit planes of the new panel (slot nb) once stage 2 has fixed its column
// exponents.  One thread per (16-row tile, column): 16 values, 8 planes of 16
// bytes each.
template <int S>
__global__ void __launch_bounds__(256) k_umma_digitize(StepArgs a) {
  __shared__ int ex[S];
  const SlabInfo si = a.slabs[blockIdx.x];
  const int k = a.nb * S;
  if (threadIdx.x < S) ex[threadIdx.x] = a.colexp[(int64_t)(k + threadIdx.x) * a.p + si.chunk];
  __syncthreads();
  const double* slot = a.V + (int64_t)a.nb * a.n * S;
  const int64_t plane = a.dtiles * 16 * S;  // bytes per plane
  uint8_t* base = a.dig + (int64_t)a.nb * 8 * plane;
  const int ntile = (si.rows + 15) / 16;
  for (int i = threadIdx.x; i < ntile * S; i += 256) {
    const int tt = i / S, j = i - tt * S;
    double x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int row = tt * 16 + r;
      x[r] = row < si.rows ? slot[(si.row0 + row) * S + j] : 0.0;
    }
    unsigned wd[kOzDigits][4], wg[4];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned h[4], l[4], g[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) bad |= oz_split(x[4 * q + r], ex[j], h[r], l[r], g[r]);
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) {
        const bool hw = t <= 3;
        const unsigned bi = hw ? (unsigned)(3 - t) : (unsigned)(7 - t);
        const unsigned sel = bi | ((4u + bi) << 4);
        const unsigned w01 = __byte_perm(hw ? h[0] : l[0], hw ? h[1] : l[1], sel);
        const unsigned w23 = __byte_perm(hw ? h[2] : l[2], hw ? h[3] : l[3], sel);
        wd[t - 1][q] = __byte_perm(w01, w23, 0x5410);
      }
      wg[q] = (g[0] >> 24) | (g[1] >> 16) | (g[2] >> 8) | g[3];
    }
    if (bad) oz_status(a.flags, LO_ERR_NONFINITE);
    uint8_t* o = base + ((int64_t)(si.tile0 + tt) * S + j) * 16;
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t)
      *reinterpret_cast<uint4*>(o + t * plane) = make_uint4(wd[t][0], wd[t][1], wd[t][2], wd[t][3]);
    *reinterpret_cast<uint4*>(o + 7 * plane) = make_uint4(wg[0], wg[1], wg[2], wg[3]);
  }
}

// ---------------------------------------------------------------------------
// Stage-1 Gram partial C = [Q_i A]^T A of one slab, for 128 columns of
// [Q_i A] (grid.y) and NB columns of A (grid.z).  MMA: M = columns of [Q_i A],
// N = (u, column of A), K = 16 rows per step.  A operand (K-major, one tile
// per digit t): row m holds the 16 row digits of column m.  B operand
// (K-major): row (u - 1) NB + n holds digit u of column n of A.
template <int S>
struct GramLayout {
  static constexpr int NB = S < 16 ? S : 16, NSPL = S / NB, NP = 128 / S;
  static constexpr int RB = umma_round16(7 * NB);
  static constexpr int STG = 0;                                      // kStages x 16 KB
  static constexpr int ABUF = STG + kStages * kStageBytes;           // 2 x 7 x 4 KB
  static constexpr int BBUF = ABUF + 2 * kOzDigits * kAPlaneBytes;   // 2 x RB x 32 B
  // private cp.async slots of the float64 values a thread splits (3 steps):
  // the block's own columns in the A tile (S threads x 16 rows) and the B
  // operand (4 NB threads x 4 rows)
  static constexpr int SRCA = BBUF + 2 * RB * 32;
  static constexpr int SRCB = SRCA + 3 * S * 16 * 8;
  static constexpr int CTL = SRCB + 3 * 4 * NB * 4 * 8;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;    // + alignment slack
};

template <int S>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_gram(StepArgs a, const double* src, int64_t lds, int pass, const __grid_constant__ CUtensorMap tm) {
  using L = GramLayout<S>;
  constexpr int NB = L::NB, NP = L::NP, RB = L::RB;
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const SlabInfo si = a.slabs[blockIdx.x];
  const int k = a.nb * S, Kt = k + S;
  const int col0 = blockIdx.y * 128, z = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np_q = max(0, min(col0 + 128, k) - col0) / S;  // prior panels in the group
  const int b0 = col0 / S;
  const int nsteps = (si.rows + 15) / 16;
  const uint32_t full0 = su32(&ctl.full[0]), mmad0 = su32(&ctl.mmad[0]);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(full0 + 8 * i, 1);
    mbar_init(mmad0, 1);
    mbar_init(mmad0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
    ctl.issued = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)),
                 "r"(umma_tcols(NB)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < 32) ctl.Hs[tid] = 0;
  // columns past Kt and B pad rows stay zero in both operand buffers
  {
    const int zc0 = max(0, Kt - col0);
    for (int i = tid; i < 2 * kOzDigits * (128 - zc0) * 2; i += kUmmaThreads) {
      const int h = i & 1, rest = i >> 1, m = zc0 + rest % (128 - zc0), bp = rest / (128 - zc0);
      *reinterpret_cast<uint4*>(sm + L::ABUF + bp * kAPlaneBytes + (m & 7) * 16 + (m >> 3) * 256 + h * 128) =
          make_uint4(0u, 0u, 0u, 0u);
    }
    if constexpr (RB > 7 * NB) {
      for (int i = tid; i < 2 * (RB - 7 * NB) * 2; i += kUmmaThreads) {
        const int h = i & 1, rest = i >> 1, r = 7 * NB + rest % (RB - 7 * NB), bb = rest / (RB - 7 * NB);
        *reinterpret_cast<uint4*>(sm + L::BBUF + bb * (RB * 32) + (r & 7) * 16 + (r >> 3) * 256 + h * 128) =
            make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;
  // the ring: TMA loads of steps 0 .. kStages - 2
  if (tid == 0 && np_q > 0) {
    for (int j = 0; j < kStages - 1 && j < nsteps; ++j) {
      mbar_expect_tx(full0 + 8 * j, 8 * NP * 16 * S);
      tma_load_4d(su32(sm + L::STG + j * kStageBytes), &tm, 0, 0, si.tile0 + j, 8 * b0, full0 + 8 * j);
      ctl.issued = j + 1;
    }
  }
  // the pass block's column exponents over this slab
  for (int idx = tid; idx < si.rows * S; idx += kUmmaThreads) {
    const int r = idx / S, l = idx - r * S;
    atomicMax(&ctl.Hs[l], bexp(src[(si.row0 + r) * lds + l]));
  }
  __syncthreads();
  if (blockIdx.y == 0 && z == 0 && tid < S) a.srcexp_slab[(int64_t)blockIdx.x * 32 + tid] = ctl.Hs[tid];
  for (int m = tid; m < 128; m += kUmmaThreads) {
    const int col = col0 + m;
    ctl.Fs[m] = (col < k) ? a.colexp[(int64_t)col * a.p + si.chunk] : (col < Kt ? ctl.Hs[col - k] : 0);
  }
  __syncthreads();

  // roles: threads 0..127 expand column m = tid of the A tile; threads
  // 128 .. 128 + 4 NB - 1 split the B operand: column n, rows 4 q .. 4 q + 3
  const int m = tid, colm = col0 + tid;
  const bool a_q = tid < 128 && colm < k, a_src = tid < 128 && colm >= k && colm < Kt;
  const int bi = tid - 128;
  const bool b_role = bi >= 0 && bi < 4 * NB;
  const int bn = b_role ? bi % NB : 0, bq = b_role ? bi / NB : 0;
  double* xa_slot = reinterpret_cast<double*>(sm + L::SRCA) + (a_src ? (colm - k) : 0) * 16;
  double* xb_slot = reinterpret_cast<double*>(sm + L::SRCB) + (b_role ? bi : 0) * 4;
  // the float64 values this thread splits in step j, into its slot j % 3
  auto load_src = [&](int j) {
    const int r0 = j * 16;
    if (a_src) {
      double* d = xa_slot + (j % 3) * S * 16;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const bool ok = r0 + r < si.rows;
        cp_async8(d + r, src + (si.row0 + (ok ? r0 + r : 0)) * lds + (colm - k), ok);
      }
    }
    if (b_role) {
      double* d = xb_slot + (j % 3) * 4 * NB * 4;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = r0 + 4 * bq + r;
        const bool ok = row < si.rows;
        cp_async8(d + r, src + (si.row0 + (ok ? row : 0)) * lds + z * NB + bn, ok);
      }
    }
    cp_async_commit();
  };
  load_src(0);
  if (nsteps > 1) load_src(1); else cp_async_commit();
  double acc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] = 0.0;
  uint32_t idesc[kOzDigits];
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t) idesc[t - 1] = umma_idesc(128, umma_nt(t, NB), 0, 0);

  for (int st = 0; st < nsteps; ++st) {
    const int s = st % kStages, bb = st & 1;
    // refill the stage consumed in the previous step
    if (tid == 0 && np_q > 0 && !ctl.abort && st + kStages - 1 < nsteps) {
      const int j = st + kStages - 1, sj = j % kStages;
      mbar_expect_tx(full0 + 8 * sj, 8 * NP * 16 * S);
      tma_load_4d(su32(sm + L::STG + sj * kStageBytes), &tm, 0, 0, si.tile0 + j, 8 * b0, full0 + 8 * sj);
      ctl.issued = j + 1;
    }
    if (st + 2 < nsteps) load_src(st + 2); else cp_async_commit();
    asm volatile("cp.async.wait_group 2;" ::: "memory");   // this thread's values of step st
    if (tid < 128 && np_q > 0 && st < ctl.issued) {
      if (!mbar_wait(full0 + 8 * s, (uint32_t)((st / kStages) & 1))) umma_timeout(ctl, a.flags);
    }
    if (st >= 2 && (tid < 128 || b_role) && !ctl.abort) {
      if (!mbar_wait(mmad0 + 8 * bb, (uint32_t)(((st - 2) >> 1) & 1))) umma_timeout(ctl, a.flags);
    }
    unsigned char* abuf = sm + L::ABUF + bb * kOzDigits * kAPlaneBytes;
    const int aoff = (m & 7) * 16 + (m >> 3) * 256;
    if (a_q) {
      const int pi = m / S, j = m - pi * S;
      const unsigned char* sp = sm + L::STG + s * kStageBytes + (pi * 8) * 16 * S + j * 16;
      const uint4 g = *reinterpret_cast<const uint4*>(sp + 7 * 16 * S);
#pragma unroll
      for (int t = 0; t < kOzDigits; ++t) {
        uint4 lo, hi;
        expand16(*reinterpret_cast<const uint4*>(sp + t * 16 * S), g, lo, hi);
        *reinterpret_cast<uint4*>(abuf + t * kAPlaneBytes + aoff) = lo;
        *reinterpret_cast<uint4*>(abuf + t * kAPlaneBytes + aoff + 128) = hi;
      }
    } else if (a_src) {
      const double* x = xa_slot + (st % 3) * S * 16;
      split8_store(x, ctl.Fs[m], abuf + aoff, a.flags);
      split8_store(x + 8, ctl.Fs[m], abuf + aoff + 128, a.flags);
    }
    if (b_role) {
      unsigned h[4], l[4], g[4];
      bool bad = false;
      const int e = ctl.Hs[z * NB + bn];
      const double* x = xb_slot + (st % 3) * 4 * NB * 4;
#pragma unroll
      for (int r = 0; r < 4; ++r) bad |= oz_split(x[r], e, h[r], l[r], g[r]);
      if (bad) oz_status(a.flags, LO_ERR_NONFINITE);
      unsigned char* bbuf = sm + L::BBUF + bb * (RB * 32) + (bq & 1) * 8 + (bq >> 1) * 128;
#pragma unroll
      for (int u = 1; u <= kOzDigits; ++u) {
        const int row = (u - 1) * NB + bn;
        const unsigned w0 = oz_pack(u, h[0], l[0], h[1], l[1], (g[0] >> 16) | g[1]);
        const unsigned w1 = oz_pack(u, h[2], l[2], h[3], l[3], (g[2] >> 16) | g[3]);
        *reinterpret_cast<uint2*>(bbuf + (row & 7) * 16 + (row >> 3) * 256) = make_uint2(w0, w1);
      }
    }
    if (tid == 0 && umma_timed_out(a.flags)) ctl.abort = 1;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && !ctl.abort) {
      tc_fence_after();
      const uint32_t bdesc_addr = su32(sm + L::BBUF + bb * (RB * 32));
      const uint64_t db = umma_sdesc(bdesc_addr, 128, 256);
      const uint32_t accum = (st & 15) ? 1u : 0u;
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) {
        const uint64_t da = umma_sdesc(su32(abuf + (t - 1) * kAPlaneBytes), 128, 256);
        umma_f16(tbase + (uint32_t)umma_col(t, NB), da, db, idesc[t - 1], accum);
      }
      umma_commit(mmad0 + 8 * bb);
    }
    // exact float32 sums cover 16 steps (256 rows): drain the accumulators
    if (((st + 1) & 15) == 0 || st + 1 == nsteps) {
      if (tid < 128 && !ctl.abort) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(mmad0 + 8 * bb, (uint32_t)((st >> 1) & 1)));
        if (!ok) {
          umma_timeout(ctl, a.flags);
        } else {
          tc_fence_after();
          const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll
          for (int c4 = 0; c4 < NB / 4; ++c4) umma_drain<NB, 4>(tlane, c4 * 4, acc + c4 * 4);
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  // partial of this slab: column col0 + m, block columns z NB .. z NB + NB - 1
  if (tid < 128 && colm < Kt && !ctl.abort) {
    double* out = a.part + (int64_t)blockIdx.x * a.Kmax * S + (int64_t)colm * S + z * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) out[j] = scale_exp(acc[j], ctl.Fs[m] + ctl.Hs[z * NB + j] - 2044 - 16);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(umma_tcols(NB)));
  }
}

// ---------------------------------------------------------------------------
// out = [Q_i A] Coef for one slab.  MMA: M = 128 rows (one row tile),
// N = (u, output column) for NB output columns at a time, K = 16 columns of
// [Q_i A] per step.  With more than NB outputs the CTA runs the K loop of a
// row tile once per group of NB outputs and writes the tile only after the
// last group: the pass block may share storage with an output (the new panel
// holds the last iterate; U may alias W), so no row is written before every
// group has read it.  A operand MN-major (a column's 16 row digits are
// contiguous in the planes); B operand: the coefficient image of the step
// (k_oz_coef<UMMA>).  NOUT = 1: the reiteration's new iterate into the new
// panel; NOUT = 2: U_i into the panel and U to the caller, plus the panel's
// column exponents.
template <int S, int NOUT>
struct UpdLayout {
  static constexpr int NC = NOUT * S, NB = NC < 16 ? NC : 16, NSPL = NC / NB;
  static constexpr int SC = S < 16 ? S : 16;  // columns of one TMA inner box
  static constexpr int RB = umma_round16(7 * NB);
  static constexpr int BIMG = RB * 32;
  static constexpr int STG = 0;
  static constexpr int BST = STG + kStages * kStageBytes;
  static constexpr int ABUF = BST + kStages * umma_round16(BIMG / 16) * 16;
  // private cp.async slots (3 steps) of the float64 values of the block's own
  // columns that thread (column kk, tile tau) splits: 128 threads x 16 rows
  static constexpr int SRCU = ABUF + 2 * kOzDigits * kAPlaneBytes;
  static constexpr int CTL = SRCU + 3 * 128 * 16 * 8;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;
};

template <int S, int NOUT>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_update(StepArgs a, const double* src_fixed, int64_t lds_fixed, int pass,
                  const __grid_constant__ CUtensorMap tm) {
  using L = UpdLayout<S, NOUT>;
  constexpr int NC = L::NC, NB = L::NB, SC = L::SC, RB = L::RB, BIMG = L::BIMG;
  if (NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const SlabInfo si = a.slabs[blockIdx.x];
  constexpr int NSPL = L::NSPL;
  const int c = si.chunk, k = a.nb * S, Kt = k + S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* src = src_fixed;
  int64_t lds = lds_fixed;
  double* slot = a.V + (int64_t)a.nb * a.n * S;
  if (NOUT == 2) {
    int Lp = 1;
    for (int t = 2; t <= kMaxPass; ++t)
      if (a.flags[kFlagPass + t - 1]) Lp = t;
    src = (Lp == 1) ? a.W : slot;
    lds = (Lp == 1) ? a.ldw : S;
  }
  const int KS = (Kt + 15) / 16, KSMAX = (a.Kmax + 15) / 16;
  const int ntr = (si.rows + 127) / 128;
  const int nsteps = ntr * NSPL * KS;  // step = (row tile, output group, 16 columns)
  const unsigned char* img = reinterpret_cast<const unsigned char*>(a.coefdig + (int64_t)c * a.coefdig_stride);
  const uint32_t full0 = su32(&ctl.full[0]), mmad0 = su32(&ctl.mmad[0]);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(full0 + 8 * i, 1);
    mbar_init(mmad0, 1);
    mbar_init(mmad0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)),
                 "r"(umma_tcols(NB)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int q = tid; q < Kt; q += kUmmaThreads)
    ctl.Fs[q] = (q < k) ? a.colexp[(int64_t)q * a.p + c] : a.srcexp[(int64_t)c * 32 + (q - k)];
  for (int n = tid; n < 64; n += kUmmaThreads) ctl.Cx[n] = (n < NC) ? a.coefexp[(int64_t)c * 64 + n] : 0;
  if (tid < 32) ctl.Ux[tid] = 0;
  if (tid == 0) ctl.issued = 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;

  // loads of step j: the digit bytes of its prior columns (TMA) and its
  // coefficient image (bulk copy), both on full[j % kStages]
  auto issue = [&](int j) {
    const int sj = j % kStages, rt = (j / (NSPL * KS)) * 128, q0 = (j % KS) * 16, zj = (j / KS) % NSPL;
    const bool has_q = q0 < k;
    mbar_expect_tx(full0 + 8 * sj, (has_q ? kStageBytes : 0) + BIMG);
    if (has_q) {
      const int b = q0 / S, half = (q0 - b * S) / SC;
      tma_load_4d(su32(sm + L::STG + sj * kStageBytes), &tm, 0, half, si.tile0 + rt / 16, 8 * b, full0 + 8 * sj);
    }
    bulk_load(su32(sm + L::BST + sj * umma_round16(BIMG / 16) * 16), img + (int64_t)(zj * KSMAX + j % KS) * BIMG,
              BIMG, full0 + 8 * sj);
    ctl.issued = j + 1;
  };
  // the MMAs read the coefficient image straight from its ring slot, so a slot
  // is refilled only once the MMAs of its previous step are known complete:
  // loads run two steps ahead
  if (tid == 0)
    for (int j = 0; j < 2 && j < nsteps; ++j) issue(j);

  // A roles: thread (column kk = tid % 16 of the step, 16-row tile tau = tid / 16)
  const int kk = tid & 15, tau = tid >> 4;
  // the pass block's values this thread splits in step j, into its slot j % 3
  double* xs_slot = reinterpret_cast<double*>(sm + L::SRCU) + (tid & 127) * 16;
  auto load_src = [&](int j) {
    const int rt = (j / (NSPL * KS)) * 128, q = (j % KS) * 16 + kk;
    if (tid < 128 && q >= k && q < Kt) {
      double* d = xs_slot + (j % 3) * 128 * 16;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int row = rt + 16 * tau + r;
        const bool ok = row < si.rows;
        cp_async8(d + r, src + (si.row0 + (ok ? row : 0)) * lds + (q - k), ok);
      }
    }
    cp_async_commit();
  };
  load_src(0);
  if (nsteps > 1) load_src(1); else cp_async_commit();
  // epilogue roles: warp w drains TMEM lanes 32 (w % 4) .. + 31 and output
  // columns (w / 4) NB / 2 .. + NB / 2 - 1 of the split
  constexpr int NH = NB / 2;
  double acc[NH], res[NSPL][NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) acc[j] = 0.0;
  uint32_t idesc[kOzDigits];
#pragma unroll
  for (int t = 1; t <= kOzDigits; ++t) idesc[t - 1] = umma_idesc(128, umma_nt(t, NB), 1, 0);

  for (int st = 0; st < nsteps; ++st) {
    const int s = st % kStages, bb = st & 1;
    const int rt = (st / (NSPL * KS)) * 128, ks = st % KS, q = ks * 16 + kk, zs = (st / KS) % NSPL;
    if (st + 2 < nsteps) load_src(st + 2); else cp_async_commit();
    asm volatile("cp.async.wait_group 2;" ::: "memory");   // this thread's values of step st
    if (tid < 128) {
      if (st < ctl.issued && !mbar_wait(full0 + 8 * s, (uint32_t)((st / kStages) & 1))) umma_timeout(ctl, a.flags);
      if (st >= 2 && !ctl.abort && !mbar_wait(mmad0 + 8 * bb, (uint32_t)(((st - 2) >> 1) & 1)))
        umma_timeout(ctl, a.flags);
      // the slot of step st + 2 last served step st - 2, whose MMAs are done
      if (tid == 0 && !ctl.abort && st + 2 < nsteps) issue(st + 2);
      unsigned char* abuf = sm + L::ABUF + bb * kOzDigits * kAPlaneBytes;
      // MN-major: rows 16 tau .. +7 and +8 .. +15 of column kk
      const int aoff = (2 * tau) * 128 + (kk & 7) * 16 + (kk >> 3) * 2048;
      if (q < k) {
        const int pp = (S == 8) ? (kk >> 3) * 8 : 0, j = (S == 8) ? (kk & 7) : kk;
        const unsigned char* sp = sm + L::STG + s * kStageBytes + ((pp * 8 + tau) * 16 * SC) + j * 16;
        const uint4 g = *reinterpret_cast<const uint4*>(sp + 7 * 8 * 16 * SC);
#pragma unroll
        for (int t = 0; t < kOzDigits; ++t) {
          uint4 lo, hi;
          expand16(*reinterpret_cast<const uint4*>(sp + t * 8 * 16 * SC), g, lo, hi);
          *reinterpret_cast<uint4*>(abuf + t * kAPlaneBytes + aoff) = lo;
          *reinterpret_cast<uint4*>(abuf + t * kAPlaneBytes + aoff + 128) = hi;
        }
      } else if (q < Kt) {
        const double* x = xs_slot + (st % 3) * 128 * 16;
        split8_store(x, ctl.Fs[q], abuf + aoff, a.flags);
        split8_store(x + 8, ctl.Fs[q], abuf + aoff + 128, a.flags);
      } else {
#pragma unroll
        for (int t = 0; t < kOzDigits; ++t) {
          *reinterpret_cast<uint4*>(abuf + t * kAPlaneBytes + aoff) = make_uint4(0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4*>(abuf + t * kAPlaneBytes + aoff + 128) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    }
    if (tid == 0 && umma_timed_out(a.flags)) ctl.abort = 1;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && !ctl.abort) {
      tc_fence_after();
      const unsigned char* abuf = sm + L::ABUF + bb * kOzDigits * kAPlaneBytes;
      const uint64_t db = umma_sdesc(su32(sm + L::BST + s * umma_round16(BIMG / 16) * 16), 128, 256);
      const uint32_t accum = (ks & 15) ? 1u : 0u;
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) {
        const uint64_t da = umma_sdesc(su32(abuf + (t - 1) * kAPlaneBytes), 2048, 128);
        umma_f16(tbase + (uint32_t)umma_col(t, NB), da, db, idesc[t - 1], accum);
      }
      umma_commit(mmad0 + 8 * bb);
    }
    const bool last_k = (ks + 1 == KS);
    if (((ks + 1) & 15) == 0 || last_k) {  // exact float32 sums cover <= 256 columns
      if (!ctl.abort) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(mmad0 + 8 * bb, (uint32_t)((st >> 1) & 1)));
        if (!ok) {
          umma_timeout(ctl, a.flags);
        } else {
          tc_fence_after();
          const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
          for (int c4 = 0; c4 < NH / 4; ++c4) umma_drain<NB, 4>(tlane, (warp >> 2) * NH + c4 * 4, acc + c4 * 4);
        }
      }
      if (last_k) {
#pragma unroll
        for (int zz = 0; zz < NSPL; ++zz)
          if (zz == zs)
#pragma unroll
            for (int j = 0; j < NH; ++j) res[zz][j] = acc[j];
#pragma unroll
        for (int j = 0; j < NH; ++j) acc[j] = 0.0;
      }
      const int r = rt + (warp & 3) * 32 + lane;
      if (last_k && zs == NSPL - 1 && r < si.rows && !ctl.abort) {
        const int64_t row = si.row0 + r;
#pragma unroll
        for (int zz = 0; zz < NSPL; ++zz)
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            const int n = zz * NB + (warp >> 2) * NH + j;
            const double d = scale_exp(res[zz][j], ctl.Cx[n] - 1022 - 16);
            if (n < S) {
              slot[row * S + n] = d;
              if (NOUT == 2) atomicMax(&ctl.Ux[n], bexp(d));
            } else {
              a.U[row * a.ldu + (n - S)] = d;
            }
          }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  if (NOUT == 2 && tid < S && !ctl.abort) atomicMax(&a.colexp[(int64_t)(k + tid) * a.p + c], ctl.Ux[tid]);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(umma_tcols(NB)));
  }
}

bool g_umma_attr = false;

template <int S>
cudaError_t umma_gram_for(const StepArgs& a, int pass, cudaStream_t st) {
  using L = GramLayout<S>;
  const int Kt = a.nb * S + S;
  dim3 grid(a.nslab, (Kt + 127) / 128, L::NSPL);
  const double* src = (pass == 1) ? a.W : a.V + (int64_t)a.nb * a.n * S;
  const int64_t lds = (pass == 1) ? a.ldw : S;
  k_umma_gram<S><<<grid, kUmmaThreads, L::BYTES, st>>>(a, src, lds, pass, a.maps->gram);
  return cudaGetLastError();
}

template <int S, int NOUT>
cudaError_t umma_update_for(const StepArgs& a, int pass, cudaStream_t st) {
  using L = UpdLayout<S, NOUT>;
  dim3 grid(a.nslab);
  const double* src = nullptr;
  int64_t lds = 0;
  if (NOUT == 1) {
    src = (pass == 2) ? a.W : a.V + (int64_t)a.nb * a.n * S;
    lds = (pass == 2) ? a.ldw : S;
  }
  k_umma_update<S, NOUT><<<grid, kUmmaThreads, L::BYTES, st>>>(a, src, lds, pass, a.maps->upd);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

bool umma_enabled(const StepArgs& a) {
  return a.dig != nullptr && a.nb >= 1 && (a.s == 8 || a.s == 16 || a.s == 32);
}

cudaError_t umma_set_attrs() {
  if (g_umma_attr) return cudaSuccess;
  cudaError_t e;
#define LO_UMMA_ATTR(S)                                                                                          \
  if ((e = cudaFuncSetAttribute(k_umma_gram<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                GramLayout<S>::BYTES)))                                                         \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_umma_update<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                UpdLayout<S, 1>::BYTES)))                                                       \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_umma_update<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                UpdLayout<S, 2>::BYTES)))                                                       \
    return e;
  LO_UMMA_ATTR(8)
  LO_UMMA_ATTR(16)
  LO_UMMA_ATTR(32)
#undef LO_UMMA_ATTR
  g_umma_attr = true;
  return cudaSuccess;
}

cudaError_t launch_umma_gram(const StepArgs& a, int pass, cudaStream_t st) {
  switch (a.s) {
    case 8: return umma_gram_for<8>(a, pass, st);
    case 16: return umma_gram_for<16>(a, pass, st);
    case 32: return umma_gram_for<32>(a, pass, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_umma_update(const StepArgs& a, int nout, int pass, cudaStream_t st) {
  switch (a.s * 4 + nout) {
    case 8 * 4 + 1: return umma_update_for<8, 1>(a, pass, st);
    case 8 * 4 + 2: return umma_update_for<8, 2>(a, pass, st);
    case 16 * 4 + 1: return umma_update_for<16, 1>(a, pass, st);
    case 16 * 4 + 2: return umma_update_for<16, 2>(a, pass, st);
    case 32 * 4 + 1: return umma_update_for<32, 1>(a, pass, st);
    case 32 * 4 + 2: return umma_update_for<32, 2>(a, pass, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_umma_digitize(const StepArgs& a, cudaStream_t st) {
  switch (a.s) {
    case 8: k_umma_digitize<8><<<a.nslab, 256, 0, st>>>(a); break;
    case 16: k_umma_digitize<16><<<a.nslab, 256, 0, st>>>(a); break;
    case 32: k_umma_digitize<32><<<a.nslab, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int64_t umma_coef_words(int Kmax, int s) {
  const int64_t KS = (Kmax + 15) / 16;
  int64_t best = 0;
  for (int nout = 1; nout <= 2; ++nout) {
    const int nc = nout * s, nb = nc < 16 ? nc : 16, nspl = nc / nb, rb = umma_round16(7 * nb);
    const int64_t w = (int64_t)nspl * KS * rb * 32 / 4;
    if (w > best) best = w;
  }
  return best;
}

cudaError_t umma_make_maps(uint8_t* dig, int s, int panels, int64_t dtiles, UmmaMaps* maps) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || fn == nullptr || q != cudaDriverEntryPointSuccess) return e ? e : cudaErrorNotSupported;
  EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
  const int sc = s < 16 ? s : 16;
  // dims (innermost first): the sc columns x 16 rows of one tile, column
  // halves, tiles, planes of all panels
  const cuuint64_t dims[4] = {(cuuint64_t)(16 * sc), (cuuint64_t)(s / sc), (cuuint64_t)dtiles,
                              (cuuint64_t)(8 * panels)};
  const cuuint64_t strides[3] = {(cuuint64_t)(16 * sc), (cuuint64_t)(16 * s), (cuuint64_t)(16 * s) * dtiles};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const cuuint32_t box_gram[4] = {(cuuint32_t)(16 * sc), (cuuint32_t)(s / sc), 1, (cuuint32_t)(8 * (128 / s))};
  const cuuint32_t box_upd[4] = {(cuuint32_t)(16 * sc), 1, 8, (cuuint32_t)(8 * (16 / sc))};
  CUresult r = encode(&maps->gram, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, dig, dims, strides, box_gram, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  r = encode(&maps->upd, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, dig, dims, strides, box_upd, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lo

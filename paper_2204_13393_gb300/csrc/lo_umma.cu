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
//   * the digit planes of prior panels arrive by bulk copies (Gram) or TMA
//     (cp.async.bulk.tensor, assembly) into a 5-stage ring tracked by
//     mbarriers, three steps ahead; the coefficient images of the
//     assembly arrive by cp.async.bulk on the same barriers;
//   * the planes are stored in the canonical no-swizzle UMMA core-matrix
//     order, so the loaded stages are the MMA operands as they are;
//   * the pass block itself (float64) is split on the fly into the stage.
//
// Digit-plane layout (global, fp16 digits with the sign in bit 15): 8-row
// block eta of the slab tiling (rows 8 eta .. 8 eta + 7; a slab's rows start
// at block 2 tile0), 8-column group G of the basis (G = b s / 8 + j / 8 for
// column j of panel b; Gtot = max_blocks s / 8 groups), plane t (digit t + 1),
// column c = j % 8, row r:
//   byte (((eta * Gtot + G) * 7 + t) * 128 + c * 16 + r * 2)
// i.e. 8 x 8 core matrices (one 16-byte row per column).  The Gram's step
// (16 rows x 128 columns) is two contiguous 14 KB runs, loaded with
// cp.async.bulk; the assembly's step (128 rows x 16 columns) is 16 runs of
// 1792 bytes, one 2D TMA box.  In shared memory they are the K-major (Gram)
// and MN-major (assembly) A operands as they are.
//
// Every wait on an mbarrier is bounded: on timeout the kernel records
// LO_ERR_TIMEOUT, stops issuing tensor-core work and drains what it issued.
#include <cfloat>
#include <cstdint>

#include "lo_internal.h"
#include "lo_oz_common.cuh"

namespace lo {
namespace {

constexpr int kUmmaThreads = 288;     // 8 worker warps + 1 issuer warp
constexpr int kIssuer = 256;          // lane 0 of warp 8 issues every load and MMA
constexpr int kStages = 5;            // TMA ring depth
constexpr int kDist = 3;              // steps loaded ahead (a stage is refilled once its MMAs are done)
constexpr int kStageBytes = 28672;    // one step's A operand: 7 digit planes of 128 x 16 fp16
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
__device__ __forceinline__ void mbar_arrive(uint32_t mb) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
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
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(mb)
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
// CTA barrier entered by converged warps (bar.sync counts a diverged warp once).
__device__ __forceinline__ void cta_sync() {
  __syncwarp();
  __syncthreads();
}

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
  uint64_t full[kStages];   // loads of a stage landed (the issuer arms them)
  uint64_t ready[kStages];  // the workers wrote their part of a step's operands (8 warp arrivals)
  uint64_t mmad[2];         // MMAs of a step done (commit), alternating by step parity
  uint64_t empty;           // the accumulators were drained (8 warp arrivals)
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
// exponent e and store their fp16 digits as one 16-byte core-matrix row of
// each of the 7 planes at dst + t * plane.
__device__ __forceinline__ void split8_store(const double* x, int e, unsigned char* dst, int plane, int* flags) {
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
    *reinterpret_cast<uint4*>(dst + t * plane) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// ---------------------------------------------------------------------------
// Digit planes of the new panel (slot nb) once stage 2 has fixed its column
// exponents.  One thread per (16-row tile, column): 16 values, 7 planes of
// two 16-byte core-matrix rows each.
template <int S>
__global__ void __launch_bounds__(256) k_umma_digitize(StepArgs a) {
  __shared__ int ex[S];
  const SlabInfo si = a.slabs[blockIdx.x];
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
}

// Largest biased exponent of each column of a pass block over each slab
// (the Gram's B-operand alignment); the reiteration's new iterate records its
// own in k_umma_update.
template <int S>
__global__ void __launch_bounds__(256) k_umma_srcexp(StepArgs a, const double* src, int64_t lds) {
  __shared__ int hs[S];
  const SlabInfo si = a.slabs[blockIdx.x];
  if (threadIdx.x < S) hs[threadIdx.x] = 0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < si.rows * S; idx += 256) {
    const int r = idx / S, l = idx - r * S;
    atomicMax(&hs[l], bexp(src[(si.row0 + r) * lds + l]));
  }
  __syncthreads();
  if (threadIdx.x < S) a.srcexp_slab[(int64_t)blockIdx.x * 32 + threadIdx.x] = hs[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Stage-1 Gram partial C = [Q_i A]^T A of one slab, for 128 columns of
// [Q_i A] (grid.y) and NB columns of A (grid.z).  MMA: M = columns of [Q_i A],
// N = (u, column of A), K = 16 rows per step.  The A operand of digit t is
// the loaded stage itself ([8-row block][group][t][128 B]: K-major,
// SBO = 7 x 128, LBO = 16 x 7 x 128); the block's own columns are split into
// it after the load.  B
// operand (K-major): row (u - 1) NB + n holds digit u of column n of A.
template <int S>
struct GramLayout {
  static constexpr int NB = S < 16 ? S : 16, NSPL = S / NB;
  static constexpr int RB = umma_round16(7 * NB);
  static constexpr int STG = 0;                                 // kStages x [2][16][7][128 B]
  static constexpr int BBUF = STG + kStages * kStageBytes;      // 2 x RB x 32 B
  // private cp.async slots (3 steps) of the float64 values a thread splits:
  // the block's own columns of the A tile (2 S units of 8 rows) and the B
  // operand (4 NB units of 4 rows)
  static constexpr int SRCA = BBUF + 2 * RB * 32;
  static constexpr int SRCB = SRCA + 3 * 2 * S * 8 * 8;
  static constexpr int CTL = SRCB + 3 * 4 * NB * 4 * 8;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;  // + alignment slack
};

template <int S>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_gram(StepArgs a, const double* src, int64_t lds, int pass) {
  using L = GramLayout<S>;
  constexpr int NB = L::NB, RB = L::RB;
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const SlabInfo si = a.slabs[blockIdx.x];
  const int k = a.nb * S, Kt = k + S;
  const int col0 = blockIdx.y * 128, z = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gtot = a.M * (S / 8), g0 = col0 / 8;
  const int ng = min(16, gtot - g0);            // column groups present in the digit planes
  const bool has_q = k > col0 && ng > 0;        // prior panels in the group: loaded
  const int nsteps = (si.rows + 15) / 16;
  const uint32_t full0 = su32(&ctl.full[0]), ready0 = su32(&ctl.ready[0]), mmad0 = su32(&ctl.mmad[0]);
  const uint32_t empty = su32(&ctl.empty);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(ready0 + 8 * i, 8);
    }
    mbar_init(mmad0, 1);
    mbar_init(mmad0 + 8, 1);
    mbar_init(empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)),
                 "r"(umma_tcols(NB)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < S) ctl.Hs[tid] = a.srcexp_slab[(int64_t)blockIdx.x * 32 + tid];
  for (int m = tid; m < 128; m += kUmmaThreads) {
    const int col = col0 + m;
    ctl.Fs[m] = (col < k) ? a.colexp[(int64_t)col * a.p + si.chunk] : 0;
  }
  if constexpr (RB > 7 * NB) {  // B pad rows stay zero
    for (int i = tid; i < 2 * (RB - 7 * NB) * 2; i += kUmmaThreads) {
      const int h = i & 1, rest = i >> 1, r = 7 * NB + rest % (RB - 7 * NB), bb = rest / (RB - 7 * NB);
      *reinterpret_cast<uint4*>(sm + L::BBUF + bb * (RB * 32) + (r & 7) * 16 + (r >> 3) * 256 + h * 128) =
          make_uint4(0u, 0u, 0u, 0u);
    }
  }
  fence_async_smem();
  tc_fence_before();
  cta_sync();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;

  if (warp == 8) {
    // ---- issuer: loads three steps ahead, one MMA group per step -----------
    if (lane == 0) {
      uint32_t idesc[kOzDigits];
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) idesc[t - 1] = umma_idesc(128, umma_nt(t, NB), 0, 0);
      // descriptors of stage 0 / buffer 0; a stage or buffer only moves the start address
      const uint64_t dA0 = umma_sdesc(su32(sm + L::STG), kStageBytes / 2, kOzDigits * 128);
      const uint64_t dB0 = umma_sdesc(su32(sm + L::BBUF), 128, 256);
      const uint32_t run = (uint32_t)max(ng, 0) * kOzDigits * 128;
      auto issue = [&](int j) {
        const int sj = j % kStages;
        const int64_t eta = 2 * (int64_t)(si.tile0 + j);
        const unsigned char* gsrc = a.dig + (eta * gtot + g0) * (kOzDigits * 128);
        mbar_expect_tx(full0 + 8 * sj, 2 * run);
        bulk_load(su32(sm + L::STG + sj * kStageBytes), gsrc, run, full0 + 8 * sj);
        bulk_load(su32(sm + L::STG + sj * kStageBytes + kStageBytes / 2), gsrc + (int64_t)gtot * kOzDigits * 128,
                  run, full0 + 8 * sj);
      };
      int issued = 0, landed = 0, drains = 0, committed = -1;
      if (has_q)
        for (; issued < kDist && issued < nsteps; ++issued) issue(issued);
      for (int st = 0; st < nsteps; ++st) {
        const int s = st % kStages, bb = st & 1;
        bool ok = true;
        // the stage of step st + kDist last served step st - 2
        if (st >= 2) ok = mbar_wait(mmad0 + 8 * bb, (uint32_t)(((st - 2) >> 1) & 1));
        if (ok && has_q && issued < nsteps && issued == st + kDist) issue(issued++);
        if (ok && has_q) {
          ok = mbar_wait(full0 + 8 * s, (uint32_t)((st / kStages) & 1));
          if (ok) landed = st + 1;
        }
        if (ok) ok = mbar_wait(ready0 + 8 * s, (uint32_t)((st / kStages) & 1));
        if (ok && (st & 15) == 0 && st > 0) ok = mbar_wait(empty, (uint32_t)(drains++ & 1));
        if (!ok || umma_timed_out(a.flags)) {
          umma_timeout(ctl, a.flags);
          break;
        }
        tc_fence_after();
        const uint64_t db = dB0 + (uint64_t)((bb * (RB * 32)) >> 4);
        const uint32_t accum = (st & 15) ? 1u : 0u;
#pragma unroll
        for (int t = 1; t <= kOzDigits; ++t) {
          const uint64_t da = dA0 + (uint64_t)((s * kStageBytes + (t - 1) * 128) >> 4);
          umma_f16(tbase + (uint32_t)umma_col(t, NB), da, db, idesc[t - 1], accum);
        }
        umma_commit(mmad0 + 8 * bb);
        committed = st;
      }
      // drain what is still in flight before the CTA's memory is released
      for (int j = landed; j < issued; ++j) mbar_wait(full0 + 8 * (j % kStages), (uint32_t)((j / kStages) & 1));
      if (committed >= 0) mbar_wait(mmad0 + 8 * (committed & 1), (uint32_t)((committed >> 1) & 1));
    }
    __syncwarp();
  } else {
    // ---- workers (warps 0..7) ------------------------------------------------
    // threads 0 .. 2S - 1 split the block's own columns into the A tile
    // (column l = tid / 2, rows 8 (tid % 2) .. + 7; only in the group that
    // holds them); threads 128 .. 128 + 4 NB - 1 split the B operand (column
    // n, rows 4 q .. 4 q + 3)
    const int al = tid >> 1, ah = tid & 1, am = k - col0 + al;
    const bool a_src = tid < 2 * S && am >= 0 && am < 128;
    const int bi = tid - 128;
    const bool b_role = bi >= 0 && bi < 4 * NB;
    const int bn = b_role ? bi % NB : 0, bq = b_role ? bi / NB : 0;
    double* xa_slot = reinterpret_cast<double*>(sm + L::SRCA) + (a_src ? tid : 0) * 8;
    double* xb_slot = reinterpret_cast<double*>(sm + L::SRCB) + (b_role ? bi : 0) * 4;
    auto load_src = [&](int j) {
      const int r0 = j * 16;
      if (a_src) {
        double* d = xa_slot + (j % 3) * 2 * S * 8;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int row = r0 + 8 * ah + r;
          const bool ok = row < si.rows;
          cp_async8(d + r, src + (si.row0 + (ok ? row : 0)) * lds + al, ok);
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
    double acc[NB / 2];
#pragma unroll
    for (int j = 0; j < NB / 2; ++j) acc[j] = 0.0;
    for (int st = 0; st < nsteps; ++st) {
      const int s = st % kStages, bb = st & 1;
      if (st + 2 < nsteps) load_src(st + 2); else cp_async_commit();
      asm volatile("cp.async.wait_group 2;" ::: "memory");   // this thread's values of step st
      // MMAs of step st - 2 done: B buffer bb is free (and no warp runs ahead)
      if (st >= 2 && !ctl.abort && !mbar_wait(mmad0 + 8 * bb, (uint32_t)(((st - 2) >> 1) & 1)))
        umma_timeout(ctl, a.flags);
      unsigned char* stage = sm + L::STG + s * kStageBytes;
      if (a_src && has_q && !ctl.abort && !mbar_wait(full0 + 8 * s, (uint32_t)((st / kStages) & 1)))
        umma_timeout(ctl, a.flags);
      if (a_src)
        split8_store(xa_slot + (st % 3) * 2 * S * 8, ctl.Hs[al],
                     stage + ah * (kStageBytes / 2) + (am >> 3) * (kOzDigits * 128) + (am & 7) * 16, 128, a.flags);
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
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready0 + 8 * s);
      // exact float32 sums cover 16 steps (256 rows): drain the accumulators;
      // warps w and w + 4 take TMEM lanes 32 (w % 4) .. + 31, halves of the NB columns
      if (((st + 1) & 15) == 0 || st + 1 == nsteps) {
        if (!ctl.abort) {
          const bool ok = __all_sync(0xffffffffu, mbar_wait(mmad0 + 8 * bb, (uint32_t)((st >> 1) & 1)));
          if (!ok) {
            umma_timeout(ctl, a.flags);
          } else {
            tc_fence_after();
            const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
            for (int c4 = 0; c4 < NB / 8; ++c4)
              umma_drain<NB, 4>(tlane, (warp >> 2) * (NB / 2) + c4 * 4, acc + c4 * 4);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(empty);
      }
    }
    // partial of this slab: column col0 + m, block columns z NB + (w / 4) NB / 2 ..
    const int m = (warp & 3) * 32 + lane, colm = col0 + m;
    if (colm < Kt && !ctl.abort) {
      const int n0 = z * NB + (warp >> 2) * (NB / 2);
      const int F = colm < k ? ctl.Fs[m] : ctl.Hs[colm - k];
      double* out = a.part + (int64_t)blockIdx.x * a.Kmax * S + (int64_t)colm * S + n0;
#pragma unroll
      for (int j = 0; j < NB / 2; ++j) out[j] = scale_exp(acc[j], F + ctl.Hs[n0 + j] - 2044 - 16);
    }
  }
  tc_fence_before();
  cta_sync();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(umma_tcols(NB)));
  }
}

// ---------------------------------------------------------------------------
// out = [Q_i A] Coef for one slab.  MMA: M = 128 rows (one row tile),
// N = (u, output column) for NB output columns at a time, K = 16 columns of
// [Q_i A] per step.  The A operand of digit t is the TMA stage itself
// ([8-row block][group][t][128 B]: MN-major, SBO = 2 x 7 x 128,
// LBO = 7 x 128); the block's own columns are split into it.  B operand: the coefficient
// image of the step (k_oz_coef<UMMA>).  With more than NB outputs the CTA
// runs the K loop of a row tile once per group of NB outputs and writes the
// tile only after the last group: the pass block may share storage with an
// output (the new panel holds the last iterate; U may alias W), so no row is
// written before every group has read it.  NOUT = 1: the reiteration's new
// iterate into the new panel, and its column exponents per slab; NOUT = 2:
// U_i into the panel and U to the caller, and the panel's column exponents.
template <int S, int NOUT>
struct UpdLayout {
  static constexpr int NC = NOUT * S, NB = NC < 16 ? NC : 16, NSPL = NC / NB;
  static constexpr int RB = umma_round16(7 * NB);
  static constexpr int BIMG = RB * 32;
  static constexpr int STG = 0;                                        // kStages x [16][2][7][128 B]
  static constexpr int BST = STG + kStages * kStageBytes;              // kStages coefficient images
  // private cp.async slots (3 steps) of the float64 values of the block's own
  // columns that thread (column, tile, half) splits: 256 threads x 8 rows
  static constexpr int SRCU = BST + kStages * umma_round16(BIMG / 16) * 16;
  static constexpr int CTL = SRCU + 3 * 256 * 8 * 8;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;
};

template <int S, int NOUT>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_update(StepArgs a, const double* src_fixed, int64_t lds_fixed, int pass,
                  const __grid_constant__ CUtensorMap tm) {
  using L = UpdLayout<S, NOUT>;
  constexpr int NC = L::NC, NB = L::NB, BIMG = L::BIMG, NSPL = L::NSPL;
  if (NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const SlabInfo si = a.slabs[blockIdx.x];
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
  const uint32_t full0 = su32(&ctl.full[0]), ready0 = su32(&ctl.ready[0]), mmad0 = su32(&ctl.mmad[0]);
  const uint32_t empty = su32(&ctl.empty);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(ready0 + 8 * i, 8);
    }
    mbar_init(mmad0, 1);
    mbar_init(mmad0 + 8, 1);
    mbar_init(empty, 8);
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
  tc_fence_before();
  cta_sync();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;

  if (warp == 8) {
    // ---- issuer: loads three steps ahead, one MMA group per step -----------
    if (lane == 0) {
      uint32_t idesc[kOzDigits];
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) idesc[t - 1] = umma_idesc(128, umma_nt(t, NB), 1, 0);
      const uint64_t dA0 = umma_sdesc(su32(sm + L::STG), kOzDigits * 128, 2 * kOzDigits * 128);
      const uint64_t dB0 = umma_sdesc(su32(sm + L::BST), 128, 256);
      // loads of step j: the digit planes of its prior columns (TMA) and its
      // coefficient image (bulk copy), both on full[j % kStages]
      auto issue = [&](int j) {
        const int sj = j % kStages, rt = (j / (NSPL * KS)) * 128, q0 = (j % KS) * 16, zj = (j / KS) % NSPL;
        const bool hq = q0 < k;
        mbar_expect_tx(full0 + 8 * sj, (hq ? kStageBytes : 0) + BIMG);
        if (hq)
          tma_load_2d(su32(sm + L::STG + sj * kStageBytes), &tm, (q0 / 8) * (kOzDigits * 128 / 8),
                      2 * (si.tile0 + rt / 16), full0 + 8 * sj);
        bulk_load(su32(sm + L::BST + sj * umma_round16(BIMG / 16) * 16), img + (int64_t)(zj * KSMAX + j % KS) * BIMG,
                  BIMG, full0 + 8 * sj);
      };
      int issued = 0, landed = 0, drains = 0, committed = -1;
      for (; issued < kDist && issued < nsteps; ++issued) issue(issued);
      for (int st = 0; st < nsteps; ++st) {
        const int s = st % kStages, bb = st & 1, ks = st % KS;
        bool ok = true;
        // the stage of step st + kDist last served step st - 2
        if (st >= 2) ok = mbar_wait(mmad0 + 8 * bb, (uint32_t)(((st - 2) >> 1) & 1));
        if (ok && issued < nsteps && issued == st + kDist) issue(issued++);
        if (ok) {
          ok = mbar_wait(full0 + 8 * s, (uint32_t)((st / kStages) & 1));
          if (ok) landed = st + 1;
        }
        if (ok) ok = mbar_wait(ready0 + 8 * s, (uint32_t)((st / kStages) & 1));
        // a new accumulation interval starts once the previous one was drained
        if (ok && (ks & 15) == 0 && st > 0) ok = mbar_wait(empty, (uint32_t)(drains++ & 1));
        if (!ok || umma_timed_out(a.flags)) {
          umma_timeout(ctl, a.flags);
          break;
        }
        tc_fence_after();
        const uint64_t db = dB0 + (uint64_t)((s * umma_round16(BIMG / 16) * 16) >> 4);
        const uint32_t accum = (ks & 15) ? 1u : 0u;
#pragma unroll
        for (int t = 1; t <= kOzDigits; ++t) {
          const uint64_t da = dA0 + (uint64_t)((s * kStageBytes + (t - 1) * 128) >> 4);
          umma_f16(tbase + (uint32_t)umma_col(t, NB), da, db, idesc[t - 1], accum);
        }
        umma_commit(mmad0 + 8 * bb);
        committed = st;
      }
      for (int j = landed; j < issued; ++j) mbar_wait(full0 + 8 * (j % kStages), (uint32_t)((j / kStages) & 1));
      if (committed >= 0) mbar_wait(mmad0 + 8 * (committed & 1), (uint32_t)((committed >> 1) & 1));
    }
    __syncwarp();
  } else {
    // ---- workers (warps 0..7): thread (column kk, 16-row tile tau, half h)
    // of a step splits the block's own columns into the stage, and warp w
    // drains TMEM lanes 32 (w % 4) .. + 31 and output columns
    // (w / 4) NB / 2 .. + NB / 2 - 1 of the group
    const int kk = tid & 15, tau = (tid >> 4) & 7, hh = (tid >> 7) & 1;
    double* xs_slot = reinterpret_cast<double*>(sm + L::SRCU) + tid * 8;
    auto load_src = [&](int j) {
      const int rt = (j / (NSPL * KS)) * 128, q = (j % KS) * 16 + kk;
      if (q >= k && q < Kt) {
        double* d = xs_slot + (j % 3) * 256 * 8;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int row = rt + 16 * tau + 8 * hh + r;
          const bool ok = row < si.rows;
          cp_async8(d + r, src + (si.row0 + (ok ? row : 0)) * lds + (q - k), ok);
        }
      }
      cp_async_commit();
    };
    load_src(0);
    if (nsteps > 1) load_src(1); else cp_async_commit();
    constexpr int NH = NB / 2;
    double acc[NH], res[NSPL][NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) acc[j] = 0.0;
    for (int st = 0; st < nsteps; ++st) {
      const int s = st % kStages, bb = st & 1;
      const int rt = (st / (NSPL * KS)) * 128, ks = st % KS, q = ks * 16 + kk, zs = (st / KS) % NSPL;
      if (st + 2 < nsteps) load_src(st + 2); else cp_async_commit();
      asm volatile("cp.async.wait_group 2;" ::: "memory");   // this thread's values of step st
      // no warp runs more than two steps ahead of the MMAs
      if (st >= 2 && !ctl.abort && !mbar_wait(mmad0 + 8 * bb, (uint32_t)(((st - 2) >> 1) & 1)))
        umma_timeout(ctl, a.flags);
      unsigned char* stage = sm + L::STG + s * kStageBytes;
      const bool writes = q >= k;  // the block's own columns, or zeros past Kt
      // the stage's loads landed (its previous step's MMAs finished before they were issued)
      if (!ctl.abort && !mbar_wait(full0 + 8 * s, (uint32_t)((st / kStages) & 1))) umma_timeout(ctl, a.flags);
      if (writes) {
        unsigned char* dst = stage + (2 * tau + hh) * (2 * kOzDigits * 128) + (kk >> 3) * (kOzDigits * 128) + (kk & 7) * 16;
        if (q < Kt) {
          split8_store(xs_slot + (st % 3) * 256 * 8, ctl.Fs[q], dst, 128, a.flags);
        } else {
#pragma unroll
          for (int t = 0; t < kOzDigits; ++t) *reinterpret_cast<uint4*>(dst + t * 128) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready0 + 8 * s);
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
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(empty);
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
                atomicMax(&ctl.Ux[n], bexp(d));
              } else {
                a.U[row * a.ldu + (n - S)] = d;
              }
            }
        }
      }
    }
  }
  tc_fence_before();
  cta_sync();
  if (tid < S && !ctl.abort) {
    if (NOUT == 2)
      atomicMax(&a.colexp[(int64_t)(k + tid) * a.p + c], ctl.Ux[tid]);
    else
      a.srcexp_slab[(int64_t)blockIdx.x * 32 + tid] = ctl.Ux[tid];
  }
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
  // the pass block's exponents per slab: from a small pass over W for pass 1,
  // from the reiteration's assembly (k_umma_update<S, 1>) afterwards
  if (pass == 1) k_umma_srcexp<S><<<a.nslab, 256, 0, st>>>(a, src, lds);
  k_umma_gram<S><<<grid, kUmmaThreads, L::BYTES, st>>>(a, src, lds, pass);
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
  // 2D view in 8-byte elements: an 8-row block's row of all column groups
  // (gtot x 7 x 128 bytes), 8-row blocks; box = 2 groups x 16 blocks
  const cuuint64_t gtot = (cuuint64_t)panels * (s / 8);
  const cuuint64_t dims[2] = {gtot * kOzDigits * 128 / 8, (cuuint64_t)(2 * dtiles)};
  const cuuint64_t strides[1] = {gtot * kOzDigits * 128};
  const cuuint32_t es[2] = {1, 1};
  const cuuint32_t box[2] = {2 * kOzDigits * 128 / 8, 16};
  const CUresult r = encode(&maps->upd, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, dig, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lo

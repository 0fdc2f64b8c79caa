// The two O(n) products of a step (the stage-1 Gram partial of Alg. 7 and the
// assembly products of Sec. 4.1), and the product Q C of apply_Q, on the
// 5th-generation tensor cores, over the digit planes that a tensor-core basis
// keeps for its prior panels.
//
// Digit arithmetic as in lo_ozaki.cu: each float64 value is split exactly into
// 7 8-bit digits aligned to its column's largest exponent, encoded as fp16
// subnormals; the 28 digit pairs (t, u) with t + u <= 8 are multiplied with
// float32 accumulation, exact for up to 256 products, and recombined in 64-bit
// integers.  With prior blocks the Gram and the 8-output assembly give bit
// for bit the results of the mma.sync kernels; the 16-output assembly sums
// the pairs of each of the three lowest classes in one float32 accumulator
// (umma_drain_mc: an error of the size of a float64 dot product's); the k = 0
// assembly rounds each output once (lo_recombine.h).
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

constexpr int kUmmaThreads = 288;     // k = 0 kernels: 8 worker warps + 1 issuer warp
constexpr int kUmma0Threads = 256;    // worker threads of the k = 0 kernels (warps 0..7)
constexpr int kUmmaKThreads = 352;    // k > 0 kernels: 8 worker warps, a load warp and two MMA warps
constexpr int kMmaWarps = 2;          // MMA-issuing warps of the k > 0 kernels (warps 9 and 10)
constexpr int kMmaSplit = 3;          // warp 9 issues digits t <= kMmaSplit (the wider MMAs), warp 10 the rest
constexpr int kStages = 5;            // ring depth: stages, B buffers and step commits (one index)
constexpr int kSrcSlots = 6;          // private cp.async slots of a producer thread (one-slice Gram steps)
constexpr int kMixedDigits = 4;       // leading digits of the mixed form's first Gram (8 bits each)
constexpr int kStageBytes = 28672;    // one step's A operand: 7 digit planes of 128 x 16 fp16
constexpr long long kWaitCycles = 500000000ll;   // ~0.25 s at 2 GHz

__host__ __device__ constexpr int umma_round16(int x) { return (x + 15) / 16 * 16; }
// N of the MMA of digit t (pairs u = 1 .. 8 - t, nb columns each), and its
// first TMEM column.
__host__ __device__ constexpr int umma_nt(int t, int nb, int nd = kOzDigits) { return umma_round16((nd + 1 - t) * nb); }
__host__ __device__ constexpr int umma_col(int t, int nb, int nd = kOzDigits) {
  int c = 0;
  for (int i = 1; i < t; ++i) c += umma_nt(i, nb, nd);
  return c;
}
// TMEM accumulator buffers (256 columns apart) that fit in the 512 columns.
__host__ __device__ constexpr int umma_nacc(int nb, int nd = kOzDigits) { return umma_col(nd + 1, nb, nd) <= 256 ? 2 : 1; }
constexpr int kTmemCols = 512;

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
// The same, also giving up as soon as another role of the CTA set *abort.
__device__ __forceinline__ bool mbar_wait_live(uint32_t mb, uint32_t parity, const int* abort) {
  if (mbar_try(mb, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(mb, parity)) {
    if (*reinterpret_cast<const volatile int*>(abort)) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(mb)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(mb)
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
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t ta, uint32_t (&r)[N]) {
  static_assert(N == 4, "tmem_ld: 4 columns");
  tmem_ld4(ta, r);
}

// Per-CTA control block at the end of dynamic shared memory.
struct UmmaCtl {
  uint64_t full[kStages];   // loads of a stage landed (the load warp arms them every step)
  uint64_t ready[kStages];  // the producer warps wrote their part of a step's operands
  uint64_t mmad[kStages];   // MMAs of a step done (commit): its stage and B buffer are free
  uint64_t empty[2];        // a TMEM accumulator buffer was drained (drainer warp arrivals)
  uint64_t accf[2];         // the last MMAs of an accumulation interval in a buffer are done
  uint64_t fin[kMmaWarps];  // an MMA warp's own MMAs are all done (its teardown)
  uint32_t tslot;           // TMEM base written by tcgen05.alloc
  int abort;                // a bounded wait gave up: no further TMA or MMA is issued
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
// recombined values to acc[0 .. NW) (or set them: the first interval of an
// output, which saves a float64 add).
template <int NB, int NW, int ND = kOzDigits>
__device__ __forceinline__ void umma_drain(uint32_t tlane, int n0, double* acc, bool first) {
  PairSums ps[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) ps[j].clear();
#pragma unroll
  for (int t = 1; t <= ND; ++t) {
    uint32_t r[ND][NW];
#pragma unroll
    for (int u = 1; u <= ND + 1 - t; ++u)
      tmem_ld<NW>(tlane + (uint32_t)(umma_col(t, NB, ND) + (u - 1) * NB + n0), r[u - 1]);
    tmem_wait_ld();
#pragma unroll
    for (int u = 1; u <= ND + 1 - t; ++u)
#pragma unroll
      for (int j = 0; j < NW; ++j) ps[j].add(t, u, __uint_as_float(r[u - 1][j]));
  }
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    const double v = ps[j].value();
    acc[j] = first ? v : acc[j] + v;
  }
}

// Merged-class accumulators of the assembly with 16 outputs per group.  The
// pairs of classes v = t + u <= 5 keep their own exact accumulators (10 pair
// blocks: digit t = 1..4, u = 1..5 - t); the pairs of each class v = 6, 7, 8
// share one float32 accumulator.  Such a class sum takes at most 7 x 16
// roundings per interval, each off by less than one unit in the last place
// (at most 8 units: |sum| < 7 2^24; rounding or truncating accumulation
// alike), under 2^10 units at a weight of at most 2^-32 of class 2: an
// absolute error below 2^-46 of 256 max|q| max|c| (the largest sum an
// interval can hold, in its column alignment), the size of a float64 dot
// product's rounding error over 256 terms near the columns' maxima (256 u =
// 2^-45); tests/test_merged_classes_cpu.py checks it in an exact model.  13
// blocks of 16 columns fit twice in TMEM, so the drain of one interval
// overlaps the next one's MMAs; 28 separate pair blocks (448 columns) allowed
// one set only, and the MMAs waited for every drain.
constexpr int kMcPairBlocks = 10;
__host__ __device__ constexpr int mc_pair_col(int t, int nb) {  // first column of digit t's exact pairs
  return (t == 1 ? 0 : t == 2 ? 4 : t == 3 ? 7 : 9) * nb;
}
__host__ __device__ constexpr int mc_class_col(int v, int nb) { return (kMcPairBlocks + v - 6) * nb; }

// umma_drain for the merged-class layout.
template <int NB, int NW>
__device__ __forceinline__ void umma_drain_mc(uint32_t tlane, int n0, double* acc, bool first) {
  PairSums ps[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) ps[j].clear();
#pragma unroll
  for (int t = 1; t <= 4; ++t) {
    uint32_t r[4][NW];
#pragma unroll
    for (int u = 1; u <= 5 - t; ++u) tmem_ld<NW>(tlane + (uint32_t)(mc_pair_col(t, NB) + (u - 1) * NB + n0), r[u - 1]);
    tmem_wait_ld();
#pragma unroll
    for (int u = 1; u <= 5 - t; ++u)
#pragma unroll
      for (int j = 0; j < NW; ++j) ps[j].add(t, u, __uint_as_float(r[u - 1][j]));
  }
  uint32_t c[3][NW];
#pragma unroll
  for (int v = 6; v <= 8; ++v) tmem_ld<NW>(tlane + (uint32_t)(mc_class_col(v, NB) + n0), c[v - 6]);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    ps[j].s[4] += __float2int_rn(__uint_as_float(c[0][j]) * 0x1p48f);   // S_6
    ps[j].s[5] += __float2int_rn(__uint_as_float(c[1][j]) * 0x1p48f);   // S_7
    ps[j].s8[0] += __float2int_rn(__uint_as_float(c[2][j]) * 0x1p48f);  // S_8 (one accumulator)
    const double v = ps[j].value();
    acc[j] = first ? v : acc[j] + v;
  }
}

// Digit planes of the new panel (slot nb): digitize_slab (lo_oz_common.cuh)
// for every slab.
template <int S>
__global__ void __launch_bounds__(256) k_umma_digitize(StepArgs a) {
  digitize_slab<S>(a, blockIdx.x);
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
  if (a.op_nx) {
    for (int idx = threadIdx.x; idx < si.rows * S; idx += 256) {
      const int r = idx / S, l = idx - r * S;
      atomicMax(&hs[l], bexp(op_value(a, si.row0 + r, l)));
    }
  } else {
    for (int idx = threadIdx.x; idx < si.rows * S; idx += 256) {
      const int r = idx / S, l = idx - r * S;
      atomicMax(&hs[l], bexp(src[(si.row0 + r) * lds + l]));
    }
  }
  __syncthreads();
  if (threadIdx.x < S) a.srcexp_slab[(int64_t)blockIdx.x * 32 + threadIdx.x] = hs[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Stage-1 Gram partials C = [Q_i A]^T A per slab.  Work item = (slab, group
// of 128 columns of [Q_i A], group of NB columns of A); one persistent CTA
// per SM walks its items, with loads running ahead across item boundaries.
// MMA: M = columns of [Q_i A], N = (u, column of A), K = 16 rows per step.
// The A operand of digit t is the loaded stage itself ([8-row block][group]
// [t][128 B]: K-major, SBO = 7 x 128, LBO = 16 x 7 x 128); the block's own
// columns are split into it after the load.  B operand (K-major): row
// (u - 1) NB + n holds digit u of column n of A.
// ND = 7: every digit (float64 accuracy); ND < 7: the leading ND digits of
// both factors and the pairs t + u <= ND + 1 (an 8 ND-bit split: the first
// pass of the mixed form), which reads ND of the 7 planes.
template <int S, int ND = kOzDigits>
struct GramLayout {
  static constexpr int NB = S < 16 ? S : 16, NSPL = S / NB;
  static constexpr int RB = umma_round16(ND * NB);
  static constexpr int STAGE = ND * 4096;                       // one K-slice: [2][16][ND][128 B]
  // K-slices of 16 rows per step: two for S <= 16 (the per-step barrier and
  // loop work of the MMA warps then covers 32 rows), in a ring of NST steps
  static constexpr int SL = S <= 16 ? 2 : 1;
  static constexpr int NST = SL == 2 ? 3 : kStages;
  static constexpr int IS = 16 / SL;                            // steps per exact float32 interval
  // private cp.async slots (SLOTS steps) of the float64 values each of the 128
  // producer threads splits, and of the exponents it splits them against: VA
  // values of the block's own columns (the A tile: S x 16 per slice) and VB
  // values of the B operand (NB x 16 per slice), per slice
  static constexpr int SLOTS = S <= 8 ? 4 : (S == 16 ? 3 : kSrcSlots);
  static constexpr int VA = S / 8, VB = NB / 8;
  static constexpr int STG = 0;                                 // NST x SL slices
  static constexpr int BBUF = STG + NST * SL * STAGE;           // NST x SL x RB x 32 B
  static constexpr int SRCA = BBUF + NST * SL * RB * 32;
  static constexpr int SRCB = SRCA + SLOTS * 128 * SL * VA * 8;
  static constexpr int EXA = SRCB + SLOTS * 128 * SL * VB * 8;
  static constexpr int EXB = EXA + SLOTS * 128 * 4;
  static constexpr int CTL = EXB + SLOTS * 128 * 4;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;  // + alignment slack
};

// One Gram work item and the walk over a CTA's items (w = blockIdx.x,
// blockIdx.x + gridDim.x, ...), step by step (SL slices of 16 rows each).
template <int SL>
struct GramCursor {
  int w, st, nsteps, slab, rows, tile0, chunk, col0, z;
  int64_t row0;
  bool valid;
  __device__ __forceinline__ void load(const StepArgs& a, int nitems, int ngroups) {
    valid = w < nitems;
    if (!valid) return;
    slab = w % a.nslab;
    const int rest = w / a.nslab;
    col0 = (rest % ngroups) * 128;
    z = rest / ngroups;
    const SlabInfo si = a.slabs[slab];
    row0 = si.row0;
    rows = si.rows;
    tile0 = si.tile0;
    chunk = si.chunk;
    nsteps = (rows + 16 * SL - 1) / (16 * SL);
  }
  // slices of the current step inside the slab (a prefix of 1 .. SL)
  __device__ __forceinline__ int slices() const {
    const int left = rows - st * 16 * SL;
    return left >= 16 * SL ? SL : (left + 15) / 16;
  }
  __device__ __forceinline__ void start(const StepArgs& a, int nitems, int ngroups) {
    w = blockIdx.x;
    st = 0;
    load(a, nitems, ngroups);
  }
  __device__ __forceinline__ void next(const StepArgs& a, int nitems, int ngroups) {
    if (++st < nsteps) return;
    w += gridDim.x;
    st = 0;
    load(a, nitems, ngroups);
  }
};

// The role of a thread of the persistent k > 0 kernels: warps 0..3 split the
// pass block into the operands of each step (producers), warps 4..7 read the
// accumulators of each finished interval back from TMEM (drainers), lane 0
// of warp 8 issues the loads of each step as soon as its stage is free (load
// warp) and lanes 0 of warps 9 and 10 issue its MMAs (MMA warps: digits t <=
// 3 and t > 3 of the streamed operand).  One thread issuing loads and MMAs
// spent about 2000 cycles per step on the serial chain of barrier waits,
// copy and MMA instructions (about 100 cycles per tcgen05.mma); split, the
// chains overlap.  mmad[s], the commits of a step's MMAs by both MMA warps,
// frees its stage (for the load warp) and its B buffer (for the producers);
// no role runs more than kStages steps ahead of the MMAs, so no barrier is
// waited on more than one phase late.  Drainers wait on accf, the commits of
// the interval's last MMAs into that TMEM buffer.

// Whether step st (of nsteps in its item) closes an accumulation interval:
// exact float32 sums cover 256 rows, IS steps.
template <int IS>
__device__ __forceinline__ bool interval_end(int st, int nsteps) { return (st + 1) % IS == 0 || st + 1 == nsteps; }

// The values a Gram producer thread loads for one step when the pass block is
// the step's operator applied to its input: rows r0 + ar0 .. + va - 1 of
// column al (A tile) and rows r0 + br0 .. + vb - 1 of column n0 + bn (B
// operand); the first column group also keeps the latter in U for the later
// passes.
__device__ __noinline__ void gram_op_values(const StepArgs& a, int64_t row0, int rows, int r0, int col0, int n0,
                                            bool asrc, int al, int ar0, int va, double* da, int bn, int br0, int vb,
                                            double* db) {
  if (asrc)
    for (int i = 0; i < va; ++i) {
      const int row = r0 + ar0 + i;
      da[i] = row < rows ? op_value(a, row0 + row, al) : 0.0;
    }
  for (int i = 0; i < vb; ++i) {
    const int row = r0 + br0 + i;
    const bool ok = row < rows;
    const double v = ok ? op_value(a, row0 + row, n0 + bn) : 0.0;
    db[i] = v;
    if (ok && col0 == 0) a.U[(row0 + row) * a.ldu + n0 + bn] = v;
  }
}

template <int S, int ND>
__global__ void __launch_bounds__(kUmmaKThreads, 1)
    k_umma_gram(StepArgs a, const double* src, int64_t lds, int pass, const __grid_constant__ CUtensorMap tm) {
  using L = GramLayout<S, ND>;
  constexpr int NB = L::NB, RB = L::RB, NSPL = L::NSPL, NACC = umma_nacc(NB, ND), STAGE = L::STAGE;
  constexpr int SL = L::SL, NST = L::NST, IS = L::IS;
  using Cursor = GramCursor<SL>;
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const int k = a.nb * S, Kt = k + S;
  const int ngroups = (Kt + 127) / 128, nitems = a.nslab * ngroups * NSPL;
  const int gtot = a.M * (S / 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = su32(&ctl.full[0]), ready0 = su32(&ctl.ready[0]), mmad0 = su32(&ctl.mmad[0]);
  const uint32_t empty0 = su32(&ctl.empty[0]), accf0 = su32(&ctl.accf[0]);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(ready0 + 8 * i, 4);
    }
    for (int i = 0; i < kStages; ++i) mbar_init(mmad0 + 8 * i, kMmaWarps);
    for (int i = 0; i < 2; ++i) {
      mbar_init(empty0 + 8 * i, 4);
      mbar_init(accf0 + 8 * i, kMmaWarps);
    }
    for (int i = 0; i < kMmaWarps; ++i) mbar_init(su32(&ctl.fin[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if constexpr (RB > ND * NB) {  // B pad rows stay zero
    for (int i = tid; i < NST * SL * (RB - ND * NB) * 2; i += kUmmaKThreads) {
      const int h = i & 1, rest = i >> 1, r = ND * NB + rest % (RB - ND * NB), bb = rest / (RB - ND * NB);
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
    // ---- load warp: the digit planes of each step once its stage is free ----
    // (the test hook withholds the loads and the MMAs: every bounded wait
    // then expires)
    if (lane == 0 && a.test_stall != 1) {
      // loads of global step j (cursor c): the digit planes of the group's prior
      // panels (all 7: two contiguous runs of the k / 8 - g0 prior column
      // groups only; the leading ND: one 3D TMA box that skips the other
      // planes of every group), or a bare arrival when it has none.  Stage
      // rows of the block's own columns are split in by the producers; rows
      // past them keep what the stage held and only reach accumulator rows
      // (columns >= k + S) that the drainers never read.
      // (per slice of the step inside the slab: slices past the slab's rows
      // are neither loaded nor multiplied)
      auto issue = [&](const Cursor& c, int j) {
        const int sj = j % NST, g0 = c.col0 / 8, ng = min(16, k / 8 - g0), nsl = c.slices();
        if (ng > 0) {
          if constexpr (ND == kOzDigits) {
            const uint32_t run = (uint32_t)ng * kOzDigits * 128;
            mbar_expect_tx(full0 + 8 * sj, (uint32_t)nsl * 2 * run);
            for (int h = 0; h < nsl; ++h) {
              const int64_t eta = 2 * (int64_t)(c.tile0 + c.st * SL + h);
              const unsigned char* gsrc = a.dig + (eta * gtot + g0) * (kOzDigits * 128);
              unsigned char* dst = sm + L::STG + (sj * SL + h) * STAGE;
              bulk_load(su32(dst), gsrc, run, full0 + 8 * sj);
              bulk_load(su32(dst + STAGE / 2), gsrc + (int64_t)gtot * kOzDigits * 128, run, full0 + 8 * sj);
            }
          } else {
            // whole boxes (groups past gtot arrive as zeros)
            mbar_expect_tx(full0 + 8 * sj, (uint32_t)(nsl * STAGE));
            for (int h = 0; h < nsl; ++h)
              tma_load_3d(su32(sm + L::STG + (sj * SL + h) * STAGE), &tm, 0, g0, (int)(2 * (c.tile0 + c.st * SL + h)),
                          full0 + 8 * sj);
          }
        } else {
          mbar_arrive(full0 + 8 * sj);
        }
      };
      Cursor ld;
      ld.start(a, nitems, ngroups);
      int issued = 0;
      for (; ld.valid; ++issued, ld.next(a, nitems, ngroups)) {
        const int sj = issued % NST;
        // the stage last served step issued - NST
        if (issued >= NST &&
            !mbar_wait_live(mmad0 + 8 * sj, (uint32_t)(((issued - NST) / NST) & 1), &ctl.abort)) {
          umma_timeout(ctl, a.flags);
          break;
        }
        if (*reinterpret_cast<volatile int*>(&ctl.abort)) break;
        issue(ld, issued);
      }
      // the copies in flight land before the CTA's memory is released (the
      // last load into each stage: no later phase exists)
      for (int j = issued > NST ? issued - NST : 0; j < issued; ++j)
        mbar_wait(full0 + 8 * (j % NST), (uint32_t)((j / NST) & 1));
    }
    __syncwarp();
  } else if (warp == 9 || warp == 10) {
    // ---- MMA warps: digits t0 .. t1 of each step ---------------------------------
    const int mw = warp - 9, t0 = mw ? kMmaSplit + 1 : 1, t1 = mw ? ND : kMmaSplit;
    if (lane == 0 && a.test_stall != 1) {
      uint32_t idesc[ND];
#pragma unroll
      for (int t = 1; t <= ND; ++t) idesc[t - 1] = umma_idesc(128, umma_nt(t, NB, ND), 0, 0);
      // descriptors of stage 0 / buffer 0; a stage or buffer only moves the start address
      const uint64_t dA0 = umma_sdesc(su32(sm + L::STG), STAGE / 2, ND * 128);
      const uint64_t dB0 = umma_sdesc(su32(sm + L::BBUF), 128, 256);
      Cursor cur;
      cur.start(a, nitems, ngroups);
      int intervals = 0;
      int64_t committed = -1;
      for (int g = 0; cur.valid; ++g, cur.next(a, nitems, ngroups)) {
        const int s = g % NST;
        const uint32_t par = (uint32_t)((g / NST) & 1);
        bool ok = mbar_wait_live(full0 + 8 * s, par, &ctl.abort);
        if (ok) ok = mbar_wait_live(ready0 + 8 * s, par, &ctl.abort);
        if (cur.st % IS == 0) {  // a new accumulation interval: its buffer must be drained
          const int b = intervals % NACC;
          if (ok && intervals >= NACC)
            ok = mbar_wait_live(empty0 + 8 * b, (uint32_t)(((intervals / NACC) - 1) & 1), &ctl.abort);
          ++intervals;
        }
        const int buf = (intervals - 1) % NACC;
        if (!ok || *reinterpret_cast<volatile int*>(&ctl.abort)) {
          umma_timeout(ctl, a.flags);
          break;
        }
        tc_fence_after();
        const int nsl = cur.slices();
#pragma unroll
        for (int h = 0; h < SL; ++h) {
          if (h >= nsl) break;
          const uint64_t db = dB0 + (uint64_t)((((s * SL + h) * RB) * 32) >> 4);
          const uint32_t accum = (cur.st % IS != 0 || h > 0) ? 1u : 0u;
#pragma unroll
          for (int t = 1; t <= ND; ++t) {
            if (t < t0 || t > t1) continue;
            const uint64_t da = dA0 + (uint64_t)(((s * SL + h) * STAGE + (t - 1) * 128) >> 4);
            umma_f16(tbase + (uint32_t)(buf * 256 + umma_col(t, NB, ND)), da, db, idesc[t - 1], accum);
          }
        }
        umma_commit(mmad0 + 8 * s);
        if (interval_end<IS>(cur.st, cur.nsteps)) umma_commit(accf0 + 8 * buf);
        committed = g;
      }
      // this warp's MMAs in flight complete before the CTA's memory is released
      if (committed >= 0) {
        umma_commit(su32(&ctl.fin[mw]));
        mbar_wait(su32(&ctl.fin[mw]), 0);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---- producers (warps 0..3) -----------------------------------------------
    // in every slice of a step each thread splits VA rows a_r0 .. of the
    // block's own column a_l into the A tile (only in the column group that
    // holds them) and VB rows b_r0 .. of column z NB + b_n into the slice's B
    // buffer.  Its values and the slab exponents it splits them against
    // arrive by cp.async AH steps ahead.
    constexpr int VA = L::VA, VB = L::VB, SLOTS = L::SLOTS, AH = SLOTS - 1;
    // S <= 16 (one group of block columns): the block's own columns of the A
    // tile are the B operand's columns, thread for thread (same values, same
    // exponents), so their split is done once and stored twice
    constexpr bool SAMEAB = NSPL == 1;
    const int a_l = tid / (16 / VA), a_r0 = (tid % (16 / VA)) * VA;
    const int b_n = tid / (16 / VB), b_r0 = (tid % (16 / VB)) * VB;
    double* xa_slot = reinterpret_cast<double*>(sm + L::SRCA) + tid * SL * VA;
    double* xb_slot = reinterpret_cast<double*>(sm + L::SRCB) + tid * SL * VB;
    int* ea_slot = reinterpret_cast<int*>(sm + L::EXA) + tid;
    int* eb_slot = reinterpret_cast<int*>(sm + L::EXB) + tid;
    auto is_asrc = [&](const Cursor& c) {
      const int am = k - c.col0 + a_l;
      return am >= 0 && am < 128;
    };
    // the float64 values this thread splits in global step j (cursor c), and
    // their exponents, into slot j % SLOTS (rows past the slab read as zeros)
    auto load_src = [&](const Cursor& c, int j) {
      if (c.valid) {
        const int sl = j % SLOTS;
        const int* hs = a.srcexp_slab + (int64_t)c.slab * 32;
        const bool asrc = is_asrc(c) && !SAMEAB;
        if (asrc) cp_async4(ea_slot + sl * 128, hs + a_l);
        cp_async4(eb_slot + sl * 128, hs + c.z * NB + b_n);
#pragma unroll
        for (int h = 0; h < SL; ++h) {
          const int r0 = (c.st * SL + h) * 16;
          double* da = xa_slot + (sl * 128 * SL + h) * VA;
          double* db = xb_slot + (sl * 128 * SL + h) * VB;
          if (a.op_nx) {
            // the operator's block, formed from its input (off the hot loop: the
            // stencil's index arithmetic stays out of the common path)
            gram_op_values(a, c.row0, c.rows, r0, c.col0, c.z * NB, asrc, a_l, a_r0, VA, da, b_n, b_r0, VB, db);
          } else {
            if (asrc) {
#pragma unroll
              for (int i = 0; i < VA; ++i) {
                const int row = r0 + a_r0 + i;
                const bool ok = row < c.rows;
                cp_async8(da + i, src + (c.row0 + (ok ? row : 0)) * lds + a_l, ok);
              }
            }
#pragma unroll
            for (int i = 0; i < VB; ++i) {
              const int row = r0 + b_r0 + i;
              const bool ok = row < c.rows;
              cp_async8(db + i, src + (c.row0 + (ok ? row : 0)) * lds + c.z * NB + b_n, ok);
            }
          }
        }
      }
      cp_async_commit();
    };
    Cursor ahead, cur;
    ahead.start(a, nitems, ngroups);
    cur.start(a, nitems, ngroups);
#pragma unroll
    for (int j = 0; j < AH; ++j) {
      load_src(ahead, j);
      ahead.next(a, nitems, ngroups);
    }
    // B buffer position of rows b_r0 .. of column b_n (digit 1; the planes are NB * 32 bytes apart)
    const int b_off = (b_n & 7) * 16 + (b_n >> 3) * 256 + (b_r0 & 7) * 2 + (b_r0 >> 3) * 128;
    for (int g = 0; cur.valid; ++g, cur.next(a, nitems, ngroups)) {
      const int s = g % NST, sl = g % SLOTS;
      load_src(ahead, g + AH);
      ahead.next(a, nitems, ngroups);
      asm volatile("cp.async.wait_group %0;" ::"n"(AH) : "memory");   // this thread's values of step g
      // MMAs of step g - NST done: the B buffers and stage s are free (and no
      // warp runs further ahead)
      if (g >= NST && !ctl.abort &&
          !mbar_wait_live(mmad0 + 8 * s, (uint32_t)(((g - NST) / NST) & 1), &ctl.abort))
        umma_timeout(ctl, a.flags);
      const bool asrc = is_asrc(cur);
      // the 7-plane loads never cover the block's own columns; the leading-
      // digit box does, so its producers write only after it landed
      if (asrc && ND != kOzDigits && !ctl.abort &&
          !mbar_wait_live(full0 + 8 * s, (uint32_t)((g / NST) & 1), &ctl.abort))
        umma_timeout(ctl, a.flags);
#pragma unroll
      for (int h = 0; h < SL; ++h) {
        unsigned char* bdst = sm + L::BBUF + (s * SL + h) * (RB * 32) + b_off;
        const int am = k - cur.col0 + a_l;
        unsigned char* adst = sm + L::STG + (s * SL + h) * STAGE + (a_r0 >> 3) * (STAGE / 2) +
                              (am >> 3) * (ND * 128) + (am & 7) * 16 + (a_r0 & 7) * 2;
        if (SAMEAB && asrc) {
          split_rows_store2<VB, ND>(xb_slot + (sl * 128 * SL + h) * VB, eb_slot[sl * 128], bdst, NB * 32, adst, 128,
                                    a.flags);
        } else {
          if (asrc)
            split_rows_store<VA, ND>(xa_slot + (sl * 128 * SL + h) * VA, ea_slot[sl * 128], adst, 128, a.flags);
          split_rows_store<VB, ND>(xb_slot + (sl * 128 * SL + h) * VB, eb_slot[sl * 128], bdst, NB * 32, a.flags);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready0 + 8 * s);
    }
  } else {
    // ---- drainers (warps 4..7): TMEM lanes 32 (w % 4) .. + 31 = columns
    // col0 + m of the item, all NB block columns, once per interval ----------
    Cursor cur;
    cur.start(a, nitems, ngroups);
    double acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = 0.0;
    int intervals = 0;
    for (; cur.valid; cur.next(a, nitems, ngroups)) {
      if (!interval_end<IS>(cur.st, cur.nsteps)) continue;
      const int buf = intervals % NACC;
      const uint32_t use = (uint32_t)(intervals / NACC);
      ++intervals;
      // warp-uniform decisions around the warp-collective TMEM loads
      bool alive = __all_sync(0xffffffffu, ctl.abort == 0);
      if (alive) {
        alive = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * buf, use & 1));
        if (!alive) {
          umma_timeout(ctl, a.flags);
        } else {
          tc_fence_after();
          const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(buf * 256);
          const bool first = cur.st < IS;  // the item's first interval
#pragma unroll
          for (int c4 = 0; c4 < NB / 4; ++c4) umma_drain<NB, 4, ND>(tlane, c4 * 4, acc + c4 * 4, first);
        }
      }
      tc_fence_before();
      __syncwarp();
      // (test hook 2: the drained buffer is never released, so the issuer's
      // wait for it expires with loads and MMAs already issued)
      if (lane == 0 && a.test_stall != 2) mbar_arrive(empty0 + 8 * buf);
      if (cur.st + 1 == cur.nsteps) {
        // partial of this slab: column col0 + m, block columns z NB .. z NB + NB - 1
        const int m = (warp & 3) * 32 + lane, colm = cur.col0 + m;
        if (colm < Kt && alive) {
          const int n0 = cur.z * NB;
          const int* hs = a.srcexp_slab + (int64_t)cur.slab * 32;
          const int F = colm < k ? a.colexp[(int64_t)colm * a.p + cur.chunk] : hs[colm - k];
          double* out = a.part + (int64_t)cur.slab * a.Kmax * S + (int64_t)colm * S + n0;
#pragma unroll
          for (int j = 0; j < NB; ++j) out[j] = scale_exp(acc[j], F + hs[n0 + j] - 2044 - 16);
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = 0.0;
      }
    }
  }
  tc_fence_before();
  cta_sync();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// out = [Q_i A] Coef per slab; one persistent CTA per SM walks its slabs.
// MMA: M = 128 rows (one row tile), N = (u, output column) for NB output
// columns at a time, K = 16 columns of [Q_i A] per step.  The A operand of
// digit t is the TMA stage itself ([8-row block][group][t][128 B]: MN-major,
// SBO = 2 x 7 x 128, LBO = 7 x 128); the block's own columns are split into
// it.  B operand: the coefficient image of the step (k_oz_coef<UMMA>; for
// apply_Q, k_apply_coef).  With
// more than NB outputs the K loop of a row tile runs once per group of NB
// outputs and the tile is written only after the last group: the pass block
// may share storage with an output (the new panel holds the last iterate;
// U may alias W), so no row is written before every group has read it.
// NOUT = 1: the reiteration's new iterate into the new panel, and its column
// exponents per slab; NOUT = 2: U_i into the panel and U to the caller, and
// the panel's column exponents.  APPLY (apply_Q, NOUT = 1, a.apply_y set):
// [Q_i A] is the basis itself -- A the last panel, whose digits are never
// stored -- and the coefficient T_i C; the result goes to the caller's Y.
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

// The walk over a CTA's slabs, step by step: step = (row tile, output
// group, 16 columns).
struct UpdCursor {
  int w, st, nsteps, rows, tile0, chunk;
  int64_t row0;
  bool valid;
  __device__ __forceinline__ void load(const StepArgs& a, int per_tile) {
    valid = w < a.nslab;
    if (!valid) return;
    const SlabInfo si = a.slabs[w];
    row0 = si.row0;
    rows = si.rows;
    tile0 = si.tile0;
    chunk = si.chunk;
    nsteps = ((rows + 127) / 128) * per_tile;
  }
  __device__ __forceinline__ void start(const StepArgs& a, int per_tile) {
    w = blockIdx.x;
    st = 0;
    load(a, per_tile);
  }
  __device__ __forceinline__ void next(const StepArgs& a, int per_tile) {
    if (++st < nsteps) return;
    w += gridDim.x;
    st = 0;
    load(a, per_tile);
  }
};

template <int S, int NOUT, bool APPLY = false>
__global__ void __launch_bounds__(kUmmaKThreads, 1)
    k_umma_update(StepArgs a, const double* src_fixed, int64_t lds_fixed, int pass,
                  const __grid_constant__ CUtensorMap tm) {
  using L = UpdLayout<S, NOUT>;
  // 16 outputs per group: merged classes 6..8 (umma_drain_mc), two accumulator sets
  constexpr int NB = L::NB, BIMG = L::BIMG, NSPL = L::NSPL;
  constexpr bool MC = NB == 16;
  constexpr int NACC = MC ? 2 : umma_nacc(NB);
  static_assert(!MC || 2 * (kMcPairBlocks + 3) * NB <= kTmemCols, "merged-class accumulators: two sets");
  static_assert(!APPLY || NOUT == 1, "apply_Q has one output");
  if (!APPLY && NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const int k = a.nb * S, Kt = k + S;
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
  const int KS = (Kt + 15) / 16, KSMAX = (a.Kmax + 15) / 16, per_tile = NSPL * KS;
  const uint32_t full0 = su32(&ctl.full[0]), ready0 = su32(&ctl.ready[0]), mmad0 = su32(&ctl.mmad[0]);
  const uint32_t empty0 = su32(&ctl.empty[0]), accf0 = su32(&ctl.accf[0]);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(ready0 + 8 * i, 4);
    }
    for (int i = 0; i < kStages; ++i) mbar_init(mmad0 + 8 * i, kMmaWarps);
    for (int i = 0; i < 2; ++i) {
      mbar_init(empty0 + 8 * i, 4);
      mbar_init(accf0 + 8 * i, kMmaWarps);
    }
    for (int i = 0; i < kMmaWarps; ++i) mbar_init(su32(&ctl.fin[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  cta_sync();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;
  // a step closes an accumulation interval: exact float32 sums cover 256 columns
  auto closes = [&](const UpdCursor& c) {
    const int ks = c.st % KS;
    return ((ks + 1) & 15) == 0 || ks + 1 == KS;
  };

  if (warp == 8) {
    // ---- load warp: each step's planes and coefficient image once its stage is free
    if (lane == 0) {
      // loads of global step j (cursor c): the digit planes of its prior
      // columns (TMA) and its coefficient image (bulk copy), on full[j % kStages]
      auto issue = [&](const UpdCursor& c, int j) {
        const int sj = j % kStages, rt = (c.st / per_tile) * 128, ks = c.st % KS, zj = (c.st / KS) % NSPL;
        const int q0 = ks * 16;
        const bool hq = q0 < k;
        mbar_expect_tx(full0 + 8 * sj, (hq ? kStageBytes : 0) + BIMG);
        if (hq)
          tma_load_2d(su32(sm + L::STG + sj * kStageBytes), &tm, (q0 / 8) * (kOzDigits * 128 / 8),
                      2 * (c.tile0 + rt / 16), full0 + 8 * sj);
        const unsigned char* img =
            reinterpret_cast<const unsigned char*>(a.coefdig + (int64_t)c.chunk * a.coefdig_stride);
        bulk_load(su32(sm + L::BST + sj * umma_round16(BIMG / 16) * 16), img + (int64_t)(zj * KSMAX + ks) * BIMG,
                  BIMG, full0 + 8 * sj);
      };
      UpdCursor ld;
      ld.start(a, per_tile);
      int issued = 0;
      for (; ld.valid; ++issued, ld.next(a, per_tile)) {
        const int sj = issued % kStages;
        // the stage last served step issued - kStages
        if (issued >= kStages &&
            !mbar_wait_live(mmad0 + 8 * sj, (uint32_t)(((issued - kStages) / kStages) & 1), &ctl.abort)) {
          umma_timeout(ctl, a.flags);
          break;
        }
        if (*reinterpret_cast<volatile int*>(&ctl.abort)) break;
        issue(ld, issued);
      }
      // the copies in flight land before the CTA's memory is released
      for (int j = issued > kStages ? issued - kStages : 0; j < issued; ++j)
        mbar_wait(full0 + 8 * (j % kStages), (uint32_t)((j / kStages) & 1));
    }
    __syncwarp();
  } else if (warp == 9 || warp == 10) {
    // ---- MMA warps: digits t0 .. t1 of each step ---------------------------------
    const int mw = warp - 9, t0 = mw ? kMmaSplit + 1 : 1, t1 = mw ? kOzDigits : kMmaSplit;
    if (lane == 0) {
      uint32_t idesc[kOzDigits];
#pragma unroll
      for (int t = 1; t <= kOzDigits; ++t) idesc[t - 1] = umma_idesc(128, umma_nt(t, NB), 1, 0);
      const uint64_t dA0 = umma_sdesc(su32(sm + L::STG), kOzDigits * 128, 2 * kOzDigits * 128);
      const uint64_t dB0 = umma_sdesc(su32(sm + L::BST), 128, 256);
      UpdCursor cur;
      cur.start(a, per_tile);
      int intervals = 0;
      int64_t committed = -1;
      for (int g = 0; cur.valid; ++g, cur.next(a, per_tile)) {
        const int s = g % kStages, ks = cur.st % KS;
        const uint32_t par = (uint32_t)((g / kStages) & 1);
        bool ok = mbar_wait_live(full0 + 8 * s, par, &ctl.abort);
        if (ok) ok = mbar_wait_live(ready0 + 8 * s, par, &ctl.abort);
        if ((ks & 15) == 0) {  // a new accumulation interval: its buffer must be drained
          const int b = intervals % NACC;
          if (ok && intervals >= NACC)
            ok = mbar_wait_live(empty0 + 8 * b, (uint32_t)(((intervals / NACC) - 1) & 1), &ctl.abort);
          ++intervals;
        }
        const int buf = (intervals - 1) % NACC;
        if (!ok || *reinterpret_cast<volatile int*>(&ctl.abort)) {
          umma_timeout(ctl, a.flags);
          break;
        }
        tc_fence_after();
        const uint64_t db = dB0 + (uint64_t)((s * umma_round16(BIMG / 16) * 16) >> 4);
        const uint32_t accum = (ks & 15) ? 1u : 0u;
        if constexpr (MC) {
          if (mw == 0) {
            // the exact pairs of digits t = 1..4 (u = 1..5 - t): their own blocks
#pragma unroll
            for (int t = 1; t <= 4; ++t) {
              const uint64_t da = dA0 + (uint64_t)((s * kStageBytes + (t - 1) * 128) >> 4);
              umma_f16(tbase + (uint32_t)(buf * 256 + mc_pair_col(t, NB)), da, db,
                       umma_idesc(128, (5 - t) * NB, 1, 0), accum);
            }
          } else {
            // every digit's pairs of classes 6..8 (u = max(1, 6 - t) .. 8 - t),
            // all from this thread in a fixed order: the shared accumulators
            // see the same sequence of additions in every run
#pragma unroll
            for (int t = 1; t <= kOzDigits; ++t) {
              const int u0 = t <= 5 ? 6 - t : 1, nu = 9 - t - u0;
              const uint64_t da = dA0 + (uint64_t)((s * kStageBytes + (t - 1) * 128) >> 4);
              const uint64_t dbu = db + (uint64_t)((((u0 - 1) * NB / 8) * 256) >> 4);
              umma_f16(tbase + (uint32_t)(buf * 256 + mc_class_col(t + u0, NB)), da, dbu,
                       umma_idesc(128, nu * NB, 1, 0), (accum || t > 1) ? 1u : 0u);
            }
          }
        } else {
#pragma unroll
          for (int t = 1; t <= kOzDigits; ++t) {
            if (t < t0 || t > t1) continue;
            const uint64_t da = dA0 + (uint64_t)((s * kStageBytes + (t - 1) * 128) >> 4);
            umma_f16(tbase + (uint32_t)(buf * 256 + umma_col(t, NB)), da, db, idesc[t - 1], accum);
          }
        }
        umma_commit(mmad0 + 8 * s);
        if (closes(cur)) umma_commit(accf0 + 8 * buf);
        committed = g;
      }
      if (committed >= 0) {
        umma_commit(su32(&ctl.fin[mw]));
        mbar_wait(su32(&ctl.fin[mw]), 0);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---- producers (warps 0..3): thread (column kk, 16-row tile tau) of a
    // step splits the block's own columns, both 8-row halves, into the stage
    const int kk = tid & 15, tau = (tid >> 4) & 7;
    auto xs_slot = [&](int hh, int j) {
      return reinterpret_cast<double*>(sm + L::SRCU) + (j % 3) * 256 * 8 + (tid + 128 * hh) * 8;
    };
    auto load_src = [&](const UpdCursor& c, int j) {
      if (c.valid) {
        const int rt = (c.st / per_tile) * 128, q = (c.st % KS) * 16 + kk;
        if (q >= k && q < Kt) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            double* d = xs_slot(hh, j);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              const int row = rt + 16 * tau + 8 * hh + r;
              const bool ok = row < c.rows;
              cp_async8(d + r, src + (c.row0 + (ok ? row : 0)) * lds + (q - k), ok);
            }
          }
        }
      }
      cp_async_commit();
    };
    UpdCursor ahead, cur;
    ahead.start(a, per_tile);
    cur.start(a, per_tile);
    load_src(ahead, 0);
    ahead.next(a, per_tile);
    load_src(ahead, 1);
    ahead.next(a, per_tile);
    for (int g = 0; cur.valid; ++g, cur.next(a, per_tile)) {
      const int s = g % kStages;
      const int ks = cur.st % KS, q = ks * 16 + kk;
      load_src(ahead, g + 2);
      ahead.next(a, per_tile);
      asm volatile("cp.async.wait_group 2;" ::: "memory");   // this thread's values of step g
      // no warp runs more than kStages steps ahead of the MMAs
      if (g >= kStages && !ctl.abort &&
          !mbar_wait_live(mmad0 + 8 * s, (uint32_t)(((g - kStages) / kStages) & 1), &ctl.abort))
        umma_timeout(ctl, a.flags);
      if (q >= k) {  // the block's own columns, or zeros past Kt, once the stage's loads landed
        if (!ctl.abort && !mbar_wait_live(full0 + 8 * s, (uint32_t)((g / kStages) & 1), &ctl.abort))
          umma_timeout(ctl, a.flags);
        unsigned char* stage = sm + L::STG + s * kStageBytes;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          unsigned char* dst =
              stage + (2 * tau + hh) * (2 * kOzDigits * 128) + (kk >> 3) * (kOzDigits * 128) + (kk & 7) * 16;
          if (q < Kt) {
            split8_store(xs_slot(hh, g), a.srcexp[(int64_t)cur.chunk * 32 + (q - k)], dst, 128, a.flags);
          } else {
#pragma unroll
            for (int t = 0; t < kOzDigits; ++t) *reinterpret_cast<uint4*>(dst + t * 128) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready0 + 8 * s);
    }
  } else {
    // ---- drainers (warps 4..7): TMEM lanes 32 (w % 4) .. + 31 = rows of the
    // tile, all NB output columns of the group, once per interval; the tile
    // is written after the last group -------------------------------------
    UpdCursor cur;
    cur.start(a, per_tile);
    double acc[NB], res[NSPL][NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = 0.0;
    int intervals = 0;
    for (; cur.valid; cur.next(a, per_tile)) {
      if (!closes(cur)) continue;
      const int rt = (cur.st / per_tile) * 128, ks = cur.st % KS, zs = (cur.st / KS) % NSPL;
      const int buf = intervals % NACC;
      const uint32_t use = (uint32_t)(intervals / NACC);
      ++intervals;
      // warp-uniform decisions around the warp-collective operations
      bool alive = __all_sync(0xffffffffu, ctl.abort == 0);
      if (alive) {
        alive = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * buf, use & 1));
        if (!alive) {
          umma_timeout(ctl, a.flags);
        } else {
          tc_fence_after();
          const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(buf * 256);
          const bool first = ks < 16;  // the output group's first interval
#pragma unroll
          for (int c4 = 0; c4 < NB / 4; ++c4) {
            if constexpr (MC)
              umma_drain_mc<NB, 4>(tlane, c4 * 4, acc + c4 * 4, first);
            else
              umma_drain<NB, 4>(tlane, c4 * 4, acc + c4 * 4, first);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * buf);
      if (ks + 1 == KS) {
#pragma unroll
        for (int zz = 0; zz < NSPL; ++zz)
          if (zz == zs)
#pragma unroll
            for (int j = 0; j < NB; ++j) res[zz][j] = acc[j];
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[j] = 0.0;
        if (zs == NSPL - 1 && alive) {
          const int r = rt + (warp & 3) * 32 + lane;
          const bool in = r < cur.rows;
          const int64_t row = cur.row0 + (in ? r : 0);
#pragma unroll
          for (int zz = 0; zz < NSPL; ++zz)
#pragma unroll
            for (int j = 0; j < NB; ++j) {
              const int n = zz * NB + j;
              const double d = scale_exp(res[zz][j], a.coefexp[(int64_t)cur.chunk * 64 + n] - 1022 - 16);
              if constexpr (APPLY) {  // apply_Q: the caller's Y, no exponent bookkeeping
                if (in && a.apply_n0 + n < a.apply_m) a.apply_y[row * a.apply_ldy + a.apply_n0 + n] = d;
              } else if (n < S) {
                if (in) slot[row * S + n] = d;
                // the column's largest exponent over the slab (NOUT = 1) or chunk (NOUT = 2)
                const int ex = __reduce_max_sync(0xffffffffu, in ? bexp(d) : 0);
                if (lane == 0) {
                  if (NOUT == 2)
                    atomicMax(&a.colexp[(int64_t)(k + n) * a.p + cur.chunk], ex);
                  else
                    atomicMax(&a.srcexp_slab[(int64_t)cur.w * 32 + n], ex);
                }
              } else if (in) {
                a.U[row * a.ldu + (n - S)] = d;
              }
            }
        }
      }
    }
  }
  tc_fence_before();
  cta_sync();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// Steps without prior blocks (k = 0, Kt = S), s in {8, 16}: the per-digit
// forms above would spend a whole 128-row M tile and seven MMAs on S
// columns.  Here the digit index moves into the MMA dimensions instead, and
// each slab is staged whole in shared memory (its exponents come from there).

// Gram of the block A over one slab: the stacked tile T (row (t - 1) S + q
// = digit t of column q, K = 16 rows per step, K-major) is both operands of
// one MMA per 16 rows: D[(t, q)][(u, n)] = sum_rows d_t(A_q) d_u(A_n), M = 7 S
// rows padded to 64 / 128, N = 7 S.  The pairs t + u <= 8 are summed per
// (q, n) into the integer pair sums of the recombination.
// Shared-memory layout of k_umma_gram0.  A slab's digits (K = its rows, M = N
// = (digit t, column q)) are 16 steps of 16 rows; a step tile holds the BLK
// digit rows of one step (7 S used, the rest zero) as 8 x 16-byte core
// matrices, K-major, 256 bytes apart along M.  At s = 8 one MMA takes two
// consecutive steps (M = N = 128, the two 64-row halves being the two steps'
// digits) and only its two diagonal 64 x 64 blocks are kept; at s = 16 one
// MMA takes one step (M = 128, N = 112).  A slab's 16 steps are written as
// two halves of 8 steps into two tile buffers, each released by the commit
// of its own MMAs.
template <int S>
struct Gram0Layout {
  static constexpr int BLK = S == 8 ? 64 : 128;   // digit rows of one step
  static constexpr int CH = 128 / BLK;             // steps per MMA
  static constexpr int N = CH == 2 ? 128 : 7 * S;  // MMA N (a multiple of 16)
  static constexpr int TILE = BLK * 32;            // bytes of one step tile (16 rows of K)
  static constexpr int HALF = 8 * TILE;            // 8 steps
  static constexpr int NX = 3, DIST = 2;           // float64 slab ring, slabs loaded ahead
  static constexpr int SS = S * S;
  static constexpr int CS = 28 * SS + 16;          // int stride of a step set in the pair sums
  static constexpr int X = 0;                      // NX slabs x 256 rows x S float64
  static constexpr int TL = X + NX * 256 * S * 8;  // 2 half-slab tile buffers
  static constexpr int P = TL + 2 * HALF;          // pair sums: CH x 28 pairs x S x S ints
  static constexpr int HW = P + CH * CS * 4;       // per-warp column exponents: 2 x 8 x S ints
  static constexpr int HS = HW + 2 * 8 * S * 4;    // slab column exponents: 2 x S ints
  static constexpr int CTL = HS + 2 * S * 4;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;
};

// The values of column q, rows r0 .. r0 + R - 1 of both 128-row halves of a
// slab (rows past the slab zero): each thread stages exactly what it reads.
template <int S, int R>
__device__ __forceinline__ void stage_cols(double* X, const SlabInfo& si, const double* src, int64_t lds, int q,
                                           int r0) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int r = 128 * h + r0 + i;
      const bool ok = r < si.rows;
      cp_async8(X + r * S + q, src + (si.row0 + (ok ? r : 0)) * lds + q, ok);
    }
}

// CTAs of the k = 0 kernels per SM: two at s = 8 (registers, shared memory
// and TMEM allow it), so one CTA's phases overlap the other's.
__host__ __device__ constexpr int umma0_ctas(int s, int nout) { return s == 8 ? 2 : 1; }

// Barrier of the 256 worker threads (warps 0..7); warp 8 issues the MMAs.
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Index of digit pair (t, u), t + u <= 8, among the 28 pairs (t-major).
__host__ __device__ constexpr int pair_index(int t, int u) { return (t - 1) * 8 - (t - 1) * t / 2 + (u - 1); }

// Contiguous slab range of CTA `cta` among `ctas`.
__device__ __forceinline__ void slab_range(int nslab, int cta, int ctas, int& w0, int& w1) {
  w0 = (int)((int64_t)nslab * cta / ctas);
  w1 = (int)((int64_t)nslab * (cta + 1) / ctas);
}

// Gram partial of every slab of the step without prior blocks (Alg. 7 stage
// 1, k = 0): part[slab] = X_slab^T X_slab in the digit arithmetic, with the
// slab's column exponents in srcexp_slab.  Worker warps 0..7 stage the
// slabs (cp.async, DIST ahead), take the column exponents, split the digits
// into the step tiles, and drain the accumulators of the previous slab; lane
// 0 of warp 8 issues the MMAs of each half slab as soon as its tiles are
// written.
template <int S>
__global__ void __launch_bounds__(kUmmaThreads, umma0_ctas(S, 1)) k_umma_gram0(StepArgs a, const double* src,
                                                                                int64_t lds, int pass) {
  using L = Gram0Layout<S>;
  constexpr int BLK = L::BLK, CH = L::CH, TILE = L::TILE, NX = L::NX, DIST = L::DIST, SS = L::SS, CS = L::CS;
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  int* P = reinterpret_cast<int*>(sm + L::P);
  int* Hw = reinterpret_cast<int*>(sm + L::HW);
  int* Hs = reinterpret_cast<int*>(sm + L::HS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ready[h]: half h of a slab's tiles written (8 warp arrivals); full[h]:
  // the MMAs reading half h are done; mmad[b]: the MMAs of a slab are done
  const uint32_t ready0 = su32(&ctl.ready[0]), free0 = su32(&ctl.full[0]), mmad0 = su32(&ctl.mmad[0]);
  if (tid == 0) {
    for (int h = 0; h < 2; ++h) {
      mbar_init(ready0 + 8 * h, 8);
      mbar_init(free0 + 8 * h, 1);
      mbar_init(mmad0 + 8 * h, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // digit rows past 7 S of every step tile stay zero
  for (int i = tid; i < 2 * 8 * (BLK - 7 * S) * 2; i += kUmmaThreads) {
    const int kh = i & 1, rest = i >> 1, r = 7 * S + rest % (BLK - 7 * S), tl = rest / (BLK - 7 * S);
    *reinterpret_cast<uint4*>(sm + L::TL + tl * TILE + (r & 7) * 16 + (r >> 3) * 256 + kh * 128) = make_uint4(0u, 0u, 0u, 0u);
  }
  int w0, w1;
  slab_range(a.nslab, blockIdx.x, gridDim.x, w0, w1);
  // split item of a worker: column q, rows r0 .. r0 + R - 1 of each half (R = S / 2)
  constexpr int R = S / 2;
  const int q = tid % S, r0 = (tid / S) * R;
  SlabInfo pf{};  // slab info of the next slab to stage
  if (tid < kUmma0Threads) {
    for (int d = 0; d < DIST; ++d) {
      if (w0 + d < w1)
        stage_cols<S, R>(reinterpret_cast<double*>(sm + L::X) + d * 256 * S, a.slabs[w0 + d], src, lds, q, r0);
      cp_async_commit();
    }
    if (w0 + DIST < w1) pf = a.slabs[w0 + DIST];
  }
  fence_async_smem();
  tc_fence_before();
  cta_sync();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;

  if (warp == 8) {
    // MMA issuer: per slab, half 0 then half 1 as their tiles are ready
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(128, L::N, 0, 0);
      const uint64_t d0 = umma_sdesc(su32(sm + L::TL), 128, 256);
      int rows_next = w0 < w1 ? a.slabs[w0].rows : 0;
      for (int j = 0, w = w0; w < w1; ++j, ++w) {
        const int nsteps = (rows_next + 15) / 16;
        if (w + 1 < w1) rows_next = a.slabs[w + 1].rows;
        const uint32_t acc_col = (uint32_t)((j & 1) * 128);
        int issued = 0;
        for (int h = 0; h < 2; ++h) {
          const bool ok = ctl.abort ? false : mbar_wait(ready0 + 8 * h, (uint32_t)(j & 1));
          if (!ok && !ctl.abort) umma_timeout(ctl, a.flags);
          tc_fence_after();
          if (!ctl.abort) {
            for (int st = 8 * h; st < 8 * h + 8 && st < nsteps; st += CH) {
              const uint64_t d = d0 + (uint64_t)((h * L::HALF + (st - 8 * h) * TILE) >> 4);
              umma_f16(tbase + acc_col, d, d, idesc, issued > 0 ? 1u : 0u);
              ++issued;
            }
          }
          umma_commit(free0 + 8 * h);
        }
        umma_commit(mmad0 + 8 * (j & 1));
      }
    }
  } else {
    // ---- workers ----
    const int qq = warp & 3, hcol = warp >> 2;
    // drain role: TMEM lanes 32 qq + lane = digit row (step set c, t, q)
    const int mrow = 32 * qq + lane, dc = mrow / BLK, dr = mrow % BLK, dt = dr / S + 1, dq = dr % S;
    auto drain = [&](int wp, int jj) {
      const int b = jj & 1;
      const bool ok = __all_sync(0xffffffffu, ctl.abort ? true : mbar_wait(mmad0 + 8 * b, (uint32_t)((jj >> 1) & 1)));
      if (!ok) umma_timeout(ctl, a.flags);
      tc_fence_after();
      if (__all_sync(0xffffffffu, ctl.abort == 0)) {  // warp-uniform around the TMEM loads
        // columns (u, n) of this warp's half: u = 4 hcol + 1 .. 4 hcol + NU
        constexpr int NU0 = 4;
        const uint32_t ta = tbase + ((uint32_t)(32 * qq) << 16) + (uint32_t)(b * 128 + dc * BLK + hcol * NU0 * S);
        uint32_t r[NU0 * S];
#pragma unroll
        for (int c8 = 0; c8 < NU0 * S / 8; ++c8) {
          if (hcol == 0 || c8 < 3 * S / 8)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[c8 * 8 + 0]), "=r"(r[c8 * 8 + 1]), "=r"(r[c8 * 8 + 2]), "=r"(r[c8 * 8 + 3]),
                           "=r"(r[c8 * 8 + 4]), "=r"(r[c8 * 8 + 5]), "=r"(r[c8 * 8 + 6]), "=r"(r[c8 * 8 + 7])
                         : "r"(ta + (uint32_t)(c8 * 8)));
        }
        tmem_wait_ld();
#pragma unroll
        for (int ui = 0; ui < NU0; ++ui) {
          const int u = hcol * NU0 + ui + 1;
          if (u <= 7 && dt <= 7 && dt + u <= 8) {
            int* dst = P + dc * CS + pair_index(dt, u) * SS + dq * S;
#pragma unroll
            for (int n4 = 0; n4 < S / 4; ++n4) {
              int4 v;
              v.x = __float2int_rn(__uint_as_float(r[ui * S + 4 * n4 + 0]) * 0x1p48f);
              v.y = __float2int_rn(__uint_as_float(r[ui * S + 4 * n4 + 1]) * 0x1p48f);
              v.z = __float2int_rn(__uint_as_float(r[ui * S + 4 * n4 + 2]) * 0x1p48f);
              v.w = __float2int_rn(__uint_as_float(r[ui * S + 4 * n4 + 3]) * 0x1p48f);
              reinterpret_cast<int4*>(dst)[n4] = v;
            }
          }
        }
      }
      tc_fence_before();
      workers_sync();
      // pair sums S_v of output (qo, no), one step set per thread, then added
      const bool alive = __all_sync(0xffffffffu, ctl.abort == 0);
      if (tid < CH * SS && alive) {
        const int qn = CH == 2 ? tid >> 1 : tid, c = CH == 2 ? tid & 1 : 0;
        int sv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) sv[i] = 0;
#pragma unroll
        for (int t = 1; t <= 7; ++t)
#pragma unroll
          for (int u = 1; u + t <= 8; ++u) {
            const int x = P[c * CS + pair_index(t, u) * SS + qn];
            sv[t + u < 8 ? t + u - 2 : (pair_group_has(0, t) ? 6 : 7)] += x;
          }
        if (CH == 2) {
#pragma unroll
          for (int i = 0; i < 8; ++i) sv[i] += __shfl_xor_sync(0xffffffffu, sv[i], 1);
        }
        if (c == 0) {
          const int qo = qn / S, no = qn % S;
          long long rest = (long long)sv[1] * (1LL << 37);
          rest += (long long)sv[2] * (1LL << 29);
          rest += (long long)sv[3] * (1LL << 21);
          rest += (long long)sv[4] * (1LL << 13);
          rest += (long long)sv[5] * (1LL << 5);
          rest += (long long)((sv[6] + 4) >> 3) + (long long)((sv[7] + 4) >> 3);
          const int* hs = Hs + S * b;
          a.part[(int64_t)wp * a.Kmax * S + qo * S + no] = oz_recombine(sv[0], rest, hs[qo] + hs[no] - 2044 - 16);
        }
      }
      if (tid < S && alive) a.srcexp_slab[(int64_t)wp * 32 + tid] = Hs[S * b + tid];
    };

    for (int j = 0, w = w0; w < w1; ++j, ++w) {
      const int b = j & 1;
      asm volatile("cp.async.wait_group %0;" ::"n"(DIST - 1) : "memory");  // own copies of slab j
      if (w + DIST < w1) {
        stage_cols<S, R>(reinterpret_cast<double*>(sm + L::X) + ((j + DIST) % NX) * 256 * S, pf, src, lds, q, r0);
        if (w + DIST + 1 < w1) pf = a.slabs[w + DIST + 1];
      }
      cp_async_commit();
      const double* X = reinterpret_cast<const double*>(sm + L::X) + (j % NX) * 256 * S;
      double x[2][R];
      int mx = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int i = 0; i < R; ++i) {
          x[h][i] = X[(128 * h + r0 + i) * S + q];
          mx = max(mx, bexp(x[h][i]));
        }
#pragma unroll
      for (int o = S; o < 32; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane < S) Hw[(b * 8 + warp) * S + lane] = mx;
      workers_sync();
      int e = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) e = max(e, Hw[(b * 8 + i) * S + q]);
      if (tid < S) Hs[S * b + tid] = e;
      // the digits, half by half, each once the MMAs of slab j - 1 that read
      // its tile buffer are done
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (j > 0 && !ctl.abort) {
          const bool ok = __all_sync(0xffffffffu, mbar_wait(free0 + 8 * h, (uint32_t)((j - 1) & 1)));
          if (!ok) umma_timeout(ctl, a.flags);
        }
        unsigned hh[R], ll[R], gg[R];
        bool bad = false;
#pragma unroll
        for (int i = 0; i < R; ++i) bad |= oz_split(x[h][i], e, hh[i], ll[i], gg[i]);
        if (bad) oz_status(a.flags, LO_ERR_NONFINITE);
        // rows r0 .. r0 + R - 1: step r0 / 16, K offset r0 % 16
        unsigned char* tb = sm + L::TL + h * L::HALF + (r0 >> 4) * TILE + ((r0 >> 3) & 1) * 128 + (r0 & 7) * 2;
#pragma unroll
        for (int t = 1; t <= kOzDigits; ++t) {
          const int m = (t - 1) * S + q;
          unsigned char* dst = tb + (m & 7) * 16 + (m >> 3) * 256;
          if constexpr (R == 4) {
            const unsigned wa = oz_pack(t, hh[0], ll[0], hh[1], ll[1], (gg[0] >> 16) | gg[1]);
            const unsigned wb = oz_pack(t, hh[2], ll[2], hh[3], ll[3], (gg[2] >> 16) | gg[3]);
            *reinterpret_cast<uint2*>(dst) = make_uint2(wa, wb);
          } else {
            uint4 v;
            v.x = oz_pack(t, hh[0], ll[0], hh[1], ll[1], (gg[0] >> 16) | gg[1]);
            v.y = oz_pack(t, hh[2], ll[2], hh[3], ll[3], (gg[2] >> 16) | gg[3]);
            v.z = oz_pack(t, hh[4], ll[4], hh[5], ll[5], (gg[4] >> 16) | gg[5]);
            v.w = oz_pack(t, hh[6], ll[6], hh[7], ll[7], (gg[6] >> 16) | gg[7]);
            *reinterpret_cast<uint4*>(dst) = v;
          }
        }
        fence_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready0 + 8 * h);
      }
      // the previous slab's accumulators, while these MMAs run
      if (j > 0) drain(w - 1, j - 1);
    }
    if (w1 > w0) {
      workers_sync();
      drain(w1 - 1, w1 - w0 - 1);
    }
  }
  tc_fence_before();
  cta_sync();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(256));
  }
}

// out = A Coef over one slab without prior blocks: K = (digit t, column q)
// = 7 S values per row (padded to KK), N = (class j, output n) = 8 NC with
// the coefficient image of k_oz_coef<MODE 2>, M = 128 rows per MMA group of
// KK / 16 instructions.  D[row][(j, n)] is the pair sum S_v (v = j + 2, or
// the two pair groups of v = 8) of the recombination, exact since it adds at
// most 7 S digit products.
template <int S, int NOUT>
struct Upd0Layout {
  static constexpr int NC = NOUT * S, KK = umma_round16(7 * S), NCOL = 8 * NC;
  static constexpr int SBO = (KK / 8) * 128, ATILE = 16 * SBO, BIMG = NC * SBO;
  static constexpr int TBUF = NCOL <= 128 ? 128 : 256;  // TMEM columns of one half's accumulators
  static constexpr int NX = 3, DIST = 2;                 // float64 slab ring, slabs loaded ahead
  static constexpr int X = 0;                            // NX slabs x 256 rows x S float64
  static constexpr int AT = X + NX * 256 * S * 8;        // A tiles of the two 128-row halves
  static constexpr int BI = AT + 2 * ATILE;              // the chunk's coefficient image
  static constexpr int CTL = BI + BIMG;
  static constexpr int BYTES = CTL + (int)sizeof(UmmaCtl) + 1024;
};

// Row `row` of slab si, float64, into X (zero past the slab), by its own thread.
template <int S>
__device__ __forceinline__ void stage_row(double* X, const SlabInfo& si, const double* src, int64_t lds, int row,
                                          bool vec16) {
  const bool ok = row < si.rows;
  const double* g = src + (si.row0 + (ok ? row : 0)) * lds;
  if (vec16) {
#pragma unroll
    for (int c = 0; c < S; c += 2) cp_async16(X + row * S + c, g + c, ok);
  } else {
#pragma unroll
    for (int c = 0; c < S; ++c) cp_async8(X + row * S + c, g + c, ok);
  }
}

// Assembly products of the step without prior blocks: out = X Coef per slab
// (NOUT = 1: the pass product into the basis slot; NOUT = 2: the slot and U).
// Worker thread i owns row i of every slab of its CTA: it stages the row
// (cp.async, DIST slabs ahead), splits it into the A tile of its 128-row half
// (K-major digits), and reads its outputs back from TMEM lane i % 128 of the
// half's accumulators one slab later; no barrier joins the workers.  Lane 0
// of warp 8 issues the KK / 16 MMAs of each half as its 4 warps finish, with
// the chunk's coefficient image resident until the chunk changes.
template <int S, int NOUT>
__global__ void __launch_bounds__(kUmmaThreads, umma0_ctas(S, NOUT)) k_umma_update0(StepArgs a, const double* src_fixed,
                                                                                     int64_t lds_fixed, int pass) {
  using L = Upd0Layout<S, NOUT>;
  constexpr int NC = L::NC, KK = L::KK, NCOL = L::NCOL, SBO = L::SBO, ATILE = L::ATILE, BIMG = L::BIMG;
  constexpr int TBUF = L::TBUF, TCOLS = 2 * TBUF, NX = L::NX, DIST = L::DIST;
  if (NOUT == 1 && !a.flags[kFlagPass + pass - 1]) return;
  if (umma_timed_out(a.flags)) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  UmmaCtl& ctl = *reinterpret_cast<UmmaCtl*>(sm + L::CTL);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* src = src_fixed;
  int64_t lds = lds_fixed;
  double* slot = a.V;  // nb = 0
  if (NOUT == 2) {
    int Lp = 1;
    for (int t = 2; t <= kMaxPass; ++t)
      if (a.flags[kFlagPass + t - 1]) Lp = t;
    src = (Lp == 1) ? a.W : slot;
    lds = (Lp == 1) ? a.ldw : S;
  }
  // ready[h]: the 4 warps of half h wrote its A tile; mmad[h]: its MMAs are
  // done; empty[0]: every MMA issued so far is done (before a new image)
  const uint32_t ready0 = su32(&ctl.ready[0]), mmad0 = su32(&ctl.mmad[0]), cfree = su32(&ctl.empty[0]);
  if (tid == 0) {
    for (int h = 0; h < 2; ++h) {
      mbar_init(ready0 + 8 * h, 4);
      mbar_init(mmad0 + 8 * h, 1);
    }
    mbar_init(cfree, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl.tslot)), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if constexpr (KK > 7 * S) {  // K pad columns of both A tiles stay zero
    static_assert(KK - 7 * S == 8, "one 16-byte pad row");
    for (int i = tid; i < 2 * 128; i += kUmmaThreads) {
      const int tl = i >> 7, m = i & 127;
      *reinterpret_cast<uint4*>(sm + L::AT + tl * ATILE + (m & 7) * 16 + (m >> 3) * SBO + (7 * S / 8) * 128) =
          make_uint4(0u, 0u, 0u, 0u);
    }
  }
  int w0, w1;
  slab_range(a.nslab, blockIdx.x, gridDim.x, w0, w1);
  const bool vec16 = ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && ((lds & 1) == 0);
  SlabInfo pf{};  // the next slab to stage
  if (tid < kUmma0Threads) {
    for (int d = 0; d < DIST; ++d) {
      if (w0 + d < w1) stage_row<S>(reinterpret_cast<double*>(sm + L::X) + d * 256 * S, a.slabs[w0 + d], src, lds, tid, vec16);
      cp_async_commit();
    }
    if (w0 + DIST < w1) pf = a.slabs[w0 + DIST];
  }
  fence_async_smem();
  tc_fence_before();
  cta_sync();
  tc_fence_after();
  const uint32_t tbase = ctl.tslot;

  if (warp == 8) {
    // ---- MMA issuer (lane 0; the warp copies coefficient images) ----
    const uint32_t idesc = umma_idesc(128, NCOL, 0, 0);
    const uint64_t db0 = umma_sdesc(su32(sm + L::BI), 128, SBO);
    int chunk = -1;
    uint32_t nimg = 0;
    SlabInfo nxt{};
    if (w0 < w1) nxt = a.slabs[w0];
    for (int j = 0, w = w0; w < w1; ++j, ++w) {
      const SlabInfo si = nxt;
      if (w + 1 < w1) nxt = a.slabs[w + 1];
      if (si.chunk != chunk) {
        if (chunk >= 0) {  // the MMAs reading the old image are done
          if (lane == 0) umma_commit(cfree);
          __syncwarp();
          const bool ok = __all_sync(0xffffffffu, ctl.abort ? true : mbar_wait(cfree, nimg & 1));
          if (!ok && lane == 0) umma_timeout(ctl, a.flags);
          ++nimg;
        }
        const uint4* g = reinterpret_cast<const uint4*>(a.coefdig + (int64_t)si.chunk * a.coefdig_stride);
        for (int i = lane; i < BIMG / 16; i += 32) reinterpret_cast<uint4*>(sm + L::BI)[i] = g[i];
        fence_async_smem();
        __syncwarp();
        chunk = si.chunk;
      }
      for (int h = 0; h < 2; ++h) {
        if (lane == 0) {
          const bool ok = ctl.abort ? false : mbar_wait(ready0 + 8 * h, (uint32_t)(j & 1));
          if (!ok && !ctl.abort) umma_timeout(ctl, a.flags);
          tc_fence_after();
          if (!ctl.abort && 128 * h < si.rows) {
            const uint64_t da0 = umma_sdesc(su32(sm + L::AT + h * ATILE), 128, SBO);
#pragma unroll
            for (int kb = 0; kb < KK / 16; ++kb)
              umma_f16(tbase + (uint32_t)(h * TBUF), da0 + (uint64_t)((kb * 256) >> 4),
                       db0 + (uint64_t)((kb * 256) >> 4), idesc, kb > 0 ? 1u : 0u);
          }
          umma_commit(mmad0 + 8 * h);
        }
        __syncwarp();
      }
    }
  } else {
    // ---- workers: thread tid owns row tid of each slab ----
    const int h = warp >> 2, m = tid & 127;
    const uint32_t tl = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * TBUF);
    unsigned char* arow = sm + L::AT + h * ATILE + (m & 7) * 16 + (m >> 3) * SBO;
    int ex[S];            // split exponents of the current chunk's columns
    int xchunk = -1;
    // outputs of row tid of slab sd (its accumulators in this half's TMEM)
    auto drain = [&](const SlabInfo& sd, int wd) {
      const bool in = tid < sd.rows;
      const int64_t row = sd.row0 + (in ? tid : 0);
#pragma unroll
      for (int g4 = 0; g4 < NC / 4; ++g4) {
        uint32_t x[8][4];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) tmem_ld4(tl + (uint32_t)(jj * NC + 4 * g4), x[jj]);
        tmem_wait_ld();
        double val[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int d[8];
          // a class sums at most 6 S digit products (< 2^22 at s = 8)
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            d[jj] = S == 8 ? oz_f2i_small(__uint_as_float(x[jj][e])) : __float2int_rn(__uint_as_float(x[jj][e]) * 0x1p48f);
          // recombination rounded once: the two exact halves of the integer
          // sum built from their bits and added in one float64 operation
          // (|class sum| <= 6 S digit products < 2^23 - 2^16 at s <= 16)
          val[e] = oz_recombine8_add(d, a.coefexp[(int64_t)sd.chunk * 64 + 4 * g4 + e] - 1022 - 16);
        }
        if (4 * g4 < S) {
          if (in) {
            double2* o = reinterpret_cast<double2*>(slot + row * S + 4 * g4);
            o[0] = make_double2(val[0], val[1]);
            o[1] = make_double2(val[2], val[3]);
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int mx = __reduce_max_sync(0xffffffffu, in ? bexp(val[e]) : 0);
            if (lane == 0) {
              if (NOUT == 2)
                atomicMax(&a.colexp[(int64_t)(4 * g4 + e) * a.p + sd.chunk], mx);
              else
                atomicMax(&a.srcexp_slab[(int64_t)wd * 32 + 4 * g4 + e], mx);
            }
          }
        } else if (in) {
#pragma unroll
          for (int e = 0; e < 4; ++e) a.U[row * a.ldu + (4 * g4 + e - S)] = val[e];
        }
      }
    };
    SlabInfo cur{}, prev{};
    if (w0 < w1) cur = a.slabs[w0];
    for (int j = 0, w = w0; w < w1; ++j, ++w) {
      const SlabInfo si = cur;
      if (w + 1 < w1) cur = a.slabs[w + 1];
      asm volatile("cp.async.wait_group %0;" ::"n"(DIST - 1) : "memory");  // own row of slab j
      if (w + DIST < w1) {
        stage_row<S>(reinterpret_cast<double*>(sm + L::X) + ((j + DIST) % NX) * 256 * S, pf, src, lds, tid, vec16);
        if (w + DIST + 1 < w1) pf = a.slabs[w + DIST + 1];
      }
      cp_async_commit();
      if (si.chunk != xchunk) {
#pragma unroll
        for (int c = 0; c < S; ++c) ex[c] = a.srcexp[(int64_t)si.chunk * 32 + c];
        xchunk = si.chunk;
      }
      // the A tile and the accumulators of this half are free once the MMAs
      // of slab j - 1 are done; its outputs first
      if (j > 0) {
        const bool ok = __all_sync(0xffffffffu, ctl.abort ? true : mbar_wait(mmad0 + 8 * h, (uint32_t)((j - 1) & 1)));
        if (!ok) umma_timeout(ctl, a.flags);
        tc_fence_after();
        if (__all_sync(0xffffffffu, ctl.abort == 0)) drain(prev, w - 1);
      }
      const double* xr = reinterpret_cast<const double*>(sm + L::X) + (j % NX) * 256 * S + tid * S;
      bool bad = false;
#pragma unroll
      for (int c8 = 0; c8 < S / 8; ++c8) {
        unsigned hh[8], ll[8], gg[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) bad |= oz_split(xr[8 * c8 + i], ex[8 * c8 + i], hh[i], ll[i], gg[i]);
#pragma unroll
        for (int t = 1; t <= kOzDigits; ++t) {
          uint4 v;
          v.x = oz_pack(t, hh[0], ll[0], hh[1], ll[1], (gg[0] >> 16) | gg[1]);
          v.y = oz_pack(t, hh[2], ll[2], hh[3], ll[3], (gg[2] >> 16) | gg[3]);
          v.z = oz_pack(t, hh[4], ll[4], hh[5], ll[5], (gg[4] >> 16) | gg[5]);
          v.w = oz_pack(t, hh[6], ll[6], hh[7], ll[7], (gg[6] >> 16) | gg[7]);
          *reinterpret_cast<uint4*>(arow + ((t - 1) * (S / 8) + c8) * 128) = v;
        }
      }
      if (bad) oz_status(a.flags, LO_ERR_NONFINITE);
      fence_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready0 + 8 * h);
      prev = si;
    }
    if (w1 > w0) {
      const int j = w1 - w0;
      const bool ok = __all_sync(0xffffffffu, ctl.abort ? true : mbar_wait(mmad0 + 8 * h, (uint32_t)((j - 1) & 1)));
      if (!ok) umma_timeout(ctl, a.flags);
      tc_fence_after();
      if (__all_sync(0xffffffffu, ctl.abort == 0)) drain(prev, w1 - 1);
    }
  }
  tc_fence_before();
  cta_sync();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
  }
}

bool g_umma_attr = false;

int umma_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  return sms;
}

template <int S, int ND = kOzDigits>
cudaError_t umma_gram_for(const StepArgs& a, int pass, cudaStream_t st) {
  using L = GramLayout<S, ND>;
  const int Kt = a.nb * S + S;
  const int nitems = a.nslab * ((Kt + 127) / 128) * L::NSPL;
  dim3 grid(nitems < umma_sms() ? nitems : umma_sms());
  const double* src = (pass == 1) ? a.W : a.V + (int64_t)a.nb * a.n * S;
  const int64_t lds = (pass == 1) ? a.ldw : S;
  // the pass block's exponents per slab: from a small pass over W for pass 1,
  // from the reiteration's assembly (k_umma_update<S, 1>) afterwards
  if (pass == 1) k_umma_srcexp<S><<<a.nslab, 256, 0, st>>>(a, src, lds);
  k_umma_gram<S, ND><<<grid, kUmmaKThreads, L::BYTES, st>>>(a, src, lds, pass, a.maps->gram_lead);
  return cudaGetLastError();
}

template <int S, int NOUT>
cudaError_t umma_update_for(const StepArgs& a, int pass, cudaStream_t st) {
  using L = UpdLayout<S, NOUT>;
  dim3 grid(a.nslab < umma_sms() ? a.nslab : umma_sms());
  const double* src = nullptr;
  int64_t lds = 0;
  if (NOUT == 1) {
    src = (pass == 2) ? a.W : a.V + (int64_t)a.nb * a.n * S;
    lds = (pass == 2) ? a.ldw : S;
  }
  k_umma_update<S, NOUT><<<grid, kUmmaKThreads, L::BYTES, st>>>(a, src, lds, pass, a.maps->upd);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// apply_Q on the tensor cores (Sec. 5.1, the product Q C, chunk-wise as
// Y_i = Q_i (T_i C)): the coefficient of chunk c for the output columns
// apply_n0 .. + S - 1 is Z_c = T_c C (Kt x S, Kt = (a.nb + 1) S: a.nb panels
// with digit planes and the last panel), each row scaled by the exponent its
// local column is aligned to, split into the image k_umma_update reads.  The
// last panel is the assembly's own block: its per-chunk column exponents go
// to srcexp, from where the producers split it.
template <int S>
__global__ void __launch_bounds__(256) k_apply_coef(StepArgs a, const double* C, int64_t ldc) {
  extern __shared__ __align__(16) double smc[];
  const int c = blockIdx.x, nbf = a.nb + 1, Kt = nbf * S, k = a.nb * S, tid = threadIdx.x;
  const double* Tc = a.T + (int64_t)c * a.tstride;
  double* Cf = smc;                                       // Kt x S
  int* Gs = reinterpret_cast<int*>(Cf + (size_t)Kt * S);  // S
  if (tid < S) {
    Gs[tid] = 0;
    a.srcexp[(int64_t)c * 32 + tid] = a.colexp[(int64_t)(k + tid) * a.p + c];
  }
  __syncthreads();
  for (int e = tid; e < Kt * S; e += 256) {
    const int r = e / S, j = e - r * S, col = a.apply_n0 + j;
    double v = 0.0;
    if (col < a.apply_m)
      for (int cb = r / S; cb < nbf; ++cb) {  // T_c is block upper triangular
        const double* Tb = Tc + tblock_offset(cb, S);
        for (int qq = 0; qq < S; ++qq) v += Tb[r * S + qq] * C[(int64_t)(cb * S + qq) * ldc + col];
      }
    const int F = a.colexp[(int64_t)r * a.p + c];
    v = (F == 0 || v == 0.0) ? 0.0 : scale2(v, F - 1022);
    Cf[e] = v;
    atomicMax(&Gs[j], bexp(v));
  }
  __syncthreads();
  umma_coef_image<S>(Cf, Gs, Kt, (a.Kmax + 15) / 16,
                     reinterpret_cast<unsigned char*>(a.coefdig + (int64_t)c * a.coefdig_stride), a.flags);
  if (tid < S) a.coefexp[(int64_t)c * 64 + tid] = Gs[tid];
}

template <int S>
size_t apply_coef_smem(int Kt) {
  return sizeof(double) * (size_t)Kt * S + sizeof(int) * 64;
}

template <int S>
cudaError_t umma_apply_for(const StepArgs& a0, const double* C, int64_t ldc, int m, double* Y, int64_t ldy,
                           cudaStream_t st) {
  using L = UpdLayout<S, 1>;
  StepArgs a = a0;
  a.nb = a0.nb - 1;  // panels with digit planes; the last is split on the fly
  a.apply_y = Y;
  a.apply_ldy = ldy;
  a.apply_m = m;
  const double* last = a0.V + (int64_t)(a0.nb - 1) * a0.n * S;
  dim3 grid(a.nslab < umma_sms() ? a.nslab : umma_sms());
  for (int n0 = 0; n0 < m; n0 += S) {
    a.apply_n0 = n0;
    k_apply_coef<S><<<a.p, 256, apply_coef_smem<S>(a0.nb * S), st>>>(a, C, ldc);
    k_umma_update<S, 1, true><<<grid, kUmmaKThreads, L::BYTES, st>>>(a, last, S, 0, a.maps->upd);
  }
  return cudaGetLastError();
}

}  // namespace

bool umma_op_supported(const StepArgs& a) { return a.precision == LO_PREC_FP64_TC && umma_enabled(a); }

bool umma_enabled(const StepArgs& a) {
  return a.dig != nullptr && a.nb >= 1 && (a.s == 8 || a.s == 16 || a.s == 32);
}

bool umma_apply_supported(const StepArgs& a) {
  return a.dig != nullptr && a.colexp != nullptr && a.maps != nullptr && a.nb >= 2 &&
         (a.s == 8 || a.s == 16 || a.s == 32);
}

cudaError_t launch_umma_apply(const StepArgs& a, const double* C, int64_t ldc, int m, double* Y, int64_t ldy,
                              cudaStream_t st) {
  switch (a.s) {
    case 8: return umma_apply_for<8>(a, C, ldc, m, Y, ldy, st);
    case 16: return umma_apply_for<16>(a, C, ldc, m, Y, ldy, st);
    case 32: return umma_apply_for<32>(a, C, ldc, m, Y, ldy, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t umma_set_attrs() {
  if (g_umma_attr) return cudaSuccess;
  cudaError_t e;
#define LO_UMMA_ATTR(S)                                                                                          \
  if ((e = cudaFuncSetAttribute(k_umma_gram<S, kOzDigits>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                GramLayout<S, kOzDigits>::BYTES)))                                              \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_umma_gram<S, kMixedDigits>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                GramLayout<S, kMixedDigits>::BYTES)))                                           \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_umma_update<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                UpdLayout<S, 1>::BYTES)))                                                       \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_umma_update<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                UpdLayout<S, 2>::BYTES)))                                                       \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_umma_update<S, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                UpdLayout<S, 1>::BYTES)))                                                       \
    return e;                                                                                                   \
  if ((e = cudaFuncSetAttribute(k_apply_coef<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                (int)apply_coef_smem<S>(kMaxKS / S))))                                          \
    return e;
  LO_UMMA_ATTR(8)
  LO_UMMA_ATTR(16)
  LO_UMMA_ATTR(32)
#undef LO_UMMA_ATTR
  if ((e = cudaFuncSetAttribute(k_umma_gram0<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, Gram0Layout<8>::BYTES)))
    return e;
  if ((e = cudaFuncSetAttribute(k_umma_gram0<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, Gram0Layout<16>::BYTES)))
    return e;
  if ((e = cudaFuncSetAttribute(k_umma_update0<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Upd0Layout<8, 1>::BYTES)))
    return e;
  if ((e = cudaFuncSetAttribute(k_umma_update0<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Upd0Layout<8, 2>::BYTES)))
    return e;
  if ((e = cudaFuncSetAttribute(k_umma_update0<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Upd0Layout<16, 1>::BYTES)))
    return e;
  if ((e = cudaFuncSetAttribute(k_umma_update0<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Upd0Layout<16, 2>::BYTES)))
    return e;
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

cudaError_t launch_umma_gram_mixed(const StepArgs& a, cudaStream_t st) {
  switch (a.s) {
    case 8: return umma_gram_for<8, kMixedDigits>(a, 1, st);
    case 16: return umma_gram_for<16, kMixedDigits>(a, 1, st);
    case 32: return umma_gram_for<32, kMixedDigits>(a, 1, st);
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

bool umma0_enabled(const StepArgs& a) { return a.nb == 0 && (a.s == 8 || a.s == 16); }

template <int S>
cudaError_t umma_gram0_for(const StepArgs& a, int pass, cudaStream_t st) {
  const double* src = (pass == 1) ? a.W : a.V;
  const int64_t lds = (pass == 1) ? a.ldw : S;
  const int ctas = umma_sms() * umma0_ctas(S, 1);
  dim3 grid(a.nslab < ctas ? a.nslab : ctas);
  k_umma_gram0<S><<<grid, kUmmaThreads, Gram0Layout<S>::BYTES, st>>>(a, src, lds, pass);
  return cudaGetLastError();
}

template <int S, int NOUT>
cudaError_t umma_update0_for(const StepArgs& a, int pass, cudaStream_t st) {
  const double* src = nullptr;
  int64_t lds = 0;
  if (NOUT == 1) {
    src = (pass == 2) ? a.W : a.V;
    lds = (pass == 2) ? a.ldw : S;
  }
  const int ctas = umma_sms() * umma0_ctas(S, NOUT);
  dim3 grid(a.nslab < ctas ? a.nslab : ctas);
  k_umma_update0<S, NOUT><<<grid, kUmmaThreads, Upd0Layout<S, NOUT>::BYTES, st>>>(a, src, lds, pass);
  return cudaGetLastError();
}

cudaError_t launch_umma_gram0(const StepArgs& a, int pass, cudaStream_t st) {
  switch (a.s) {
    case 8: return umma_gram0_for<8>(a, pass, st);
    case 16: return umma_gram0_for<16>(a, pass, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_umma_update0(const StepArgs& a, int nout, int pass, cudaStream_t st) {
  switch (a.s * 4 + nout) {
    case 8 * 4 + 1: return umma_update0_for<8, 1>(a, pass, st);
    case 8 * 4 + 2: return umma_update0_for<8, 2>(a, pass, st);
    case 16 * 4 + 1: return umma_update0_for<16, 1>(a, pass, st);
    case 16 * 4 + 2: return umma_update0_for<16, 2>(a, pass, st);
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
  if (s == 8 || s == 16)  // the image of the step without prior blocks (k_umma_update0)
    best = (int64_t)2 * s * (umma_round16(7 * s) / 8) * 128 / 4;
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
  CUresult r = encode(&maps->upd, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, dig, dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // 3D view for the mixed Gram's leading digits: (the 7 x 128 bytes of one
  // group of one 8-row block, groups, 8-row blocks); box = the first
  // kMixedDigits x 128 bytes of 16 groups of 2 blocks (one 16-row step of 128
  // columns)
  const cuuint64_t dims3[3] = {kOzDigits * 128 / 8, gtot, (cuuint64_t)(2 * dtiles)};
  const cuuint64_t strides3[2] = {kOzDigits * 128, gtot * kOzDigits * 128};
  const cuuint32_t es3[3] = {1, 1, 1};
  const cuuint32_t box3[3] = {kMixedDigits * 128 / 8, 16, 2};
  r = encode(&maps->gram_lead, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, dig, dims3, strides3, box3, es3,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lo

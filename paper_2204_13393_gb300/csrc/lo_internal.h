// Internal declarations shared by the host orchestration (lo_api.cu) and the
// kernels (lo_kernels.cu).  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lo.h"

namespace lo {

constexpr int kMaxS = 32;        // block width limit (one warp per column set)
constexpr int kMaxK = 1024;      // max_blocks * s
constexpr int kMaxKS = 8192;     // (k + s) * s entries of one Gram tile
constexpr int kThreads = 256;    // threads of the streaming kernels
constexpr int kMaxPass = 3;      // local Gram passes (PIP, PIP+, one more)
constexpr int kMaxTreeIter = 3;  // reduction iterations
constexpr int kTreeGroup = 16;   // chunks summed per CTA in the tree's first level (more CTAs: float64 adds)
constexpr int kHHThreads = 256;  // threads of the Householder leaf (one CTA per chunk)
constexpr int kHHTileBytes = 200 * 1024;  // shared memory for one chunk tile of the Householder leaf
// Rows of the Householder leaf's sub-tiles when a chunk exceeds one tile: the
// largest power of two T with (T + s) s doubles in the tile budget.
inline int hh_subtile_rows(int s) {
  int T = 1 << 14;
  while (T > s && (int64_t)(T + s) * s * 8 > kHHTileBytes) T >>= 1;
  return T;
}

// Flag words (int) in device memory.
enum Flag : int {
  kFlagStatus = 0,        // lo_status bits (OR of 1 << status) latched by kernels
  kFlagPass = 1,          // [1 .. kMaxPass]: pass t requested (1) or not (0)
  kFlagTree = 1 + kMaxPass + 1,  // [.. + kMaxTreeIter]: tree iteration requested
  kFlagCount = 16
};

// One row slab of one chunk: the unit of work of the streaming kernels.
struct SlabInfo {
  int64_t row0;
  int32_t rows;
  int32_t chunk;
  int32_t tile0;   // first 16-row tile of the slab in the digit planes (slabs start new tiles)
  int32_t pad_;
};

// Per-chunk small-matrix scratch, offsets in doubles (Kmax = M * s).
struct SmallLayout {
  int64_t P_last, P_comb, P_hat, Z;          // Kmax x s each
  int64_t N_last, Ninv_last, N_comb, N_hat;  // s x s each
  int64_t stride;
  __host__ __device__ static SmallLayout make(int Kmax, int s) {
    SmallLayout L;
    int64_t ks = (int64_t)Kmax * s, ss = (int64_t)s * s;
    L.P_last = 0;
    L.P_comb = ks;
    L.P_hat = 2 * ks;
    L.Z = 3 * ks;
    L.N_last = 4 * ks;
    L.Ninv_last = L.N_last + ss;
    L.N_comb = L.N_last + 2 * ss;
    L.N_hat = L.N_last + 3 * ss;
    L.stride = L.N_last + 4 * ss;
    return L;
  }
};

// Global small-matrix scratch, offsets in doubles.
struct GlobLayout {
  int64_t P_it, N_it, Ninv_it;   // this tree iteration: Kmax x s, s x s, s x s
  int64_t P_acc, N_acc;          // combined over iterations (the outputs H, R)
  int64_t Zsum;                  // Kmax x s, the summed contributions
  int64_t scal;                  // 8 scalars: [0] = |W|_F^2 of the step (tree), [1] = the same from the
                                 // pass-1 Gram partials (deflation thresholds of the local leaves)
  int64_t stride;
  __host__ __device__ static GlobLayout make(int Kmax, int s) {
    GlobLayout L;
    int64_t ks = (int64_t)Kmax * s, ss = (int64_t)s * s;
    L.P_it = 0;
    L.N_it = ks;
    L.Ninv_it = ks + ss;
    L.P_acc = ks + 2 * ss;
    L.N_acc = 2 * ks + 2 * ss;
    L.Zsum = 2 * ks + 3 * ss;
    L.scal = 3 * ks + 3 * ss;
    L.stride = 3 * ks + 3 * ss + 8;
    return L;
  }
};

// Everything a kernel needs to know about a basis and the current step.
struct StepArgs {
  int64_t n;
  int s, M, p, nb;          // nb = blocks already in the basis (k = nb * s)
  int Kmax;
  double* V;                // local panels: panel b at V + b * n * s, row-major n x s
  double* T;                // tree factors, chunk stride tstride
  int64_t tstride;
  double* part;             // Gram partials: nslab x Kmax x s
  double* small;            // per-chunk scratch, SmallLayout
  double* glob;             // global scratch, GlobLayout
  double* tsum;             // tree first-level sums: ngroups x Kmax x s
  int* flags;
  int* tree_ticket;         // one int, zero between steps: chunks done in a ticketed reduction round
  const SlabInfo* slabs;
  const int32_t* chunk_slab0;   // first slab of chunk c (p + 1 entries)
  const int64_t* chunk_row0;    // first row of chunk c (p + 1 entries)
  int nslab;
  int slab_rows;
  int max_chunk_rows;       // rows of the largest chunk (the last one holds the remainder)
  // Householder leaf over chunks larger than one tile (FlatTSPQR inside the
  // chunk): sub-tile rows, stages per chunk, and per chunk and stage the
  // reflectors' parts on the carried rows (s x s) and their tau (s)
  int hh_T, hh_stages;
  double* hh_scratch;
  int precision;
  int leaf;
  int reduction;
  double refine_tol;
  double deflation_tol;     // delta of the deflated PQR (0: off)
  // the step's block and outputs
  const double* W;
  int64_t ldw;
  double* U;
  int64_t ldu;
  // the block as an operator applied to a device block: W = L V for the 2D
  // 5-point Laplacian on an op_nx x op_ny grid (op_nx = 0: none).  The first
  // Gram pass forms W from V on the fly and writes it into U (W = U then for
  // the rest of the step).
  int op_nx, op_ny;
  const double* op_V;
  int64_t op_ldv;
  // float64-accurate tensor-core form (LO_PREC_FP64_TC); null otherwise
  int* colexp;               // [Kmax][p]: largest biased exponent of each local column per chunk
  int* srcexp_slab;          // [nslab][32]: the same for the block of the current pass, per slab
  int* srcexp;               // [p][32]: ... per chunk
  uint32_t* coefdig;         // [p][coefdig_stride]: digit planes of the scaled coefficients
  int* coefexp;              // [p][64]: exponent of each coefficient column
  int64_t coefdig_stride;    // uint32 words per chunk
  // digit planes of the local panels (tensor-core forms, s in {8, 16, 32}); null when off.
  // fp16 digit t + 1 (t = 0..6, sign in bit 15) of the value in column j of
  // panel b, row 8 eta + r of the slab tiling (a slab starts at eta = 2 tile0),
  // aligned to colexp of its chunk, at byte
  //   (((eta * Gtot + G) * 7 + t) * 128 + (j % 8) * 16 + r * 2),  G = b s / 8 + j / 8,
  // Gtot = M s / 8 (8 x 8 core matrices of the tcgen05 operand layouts); rows
  // past a slab's end are zero.
  uint8_t* dig;
  int64_t dtiles;            // 16-row tiles of the slab tiling
  const struct UmmaMaps* maps;  // host-side TMA descriptors of dig (lo_umma.cu)
  int32_t test_stall;           // test hook (lo_options): 1 the k > 0 tensor-core Gram issues nothing,
                                // 2 its drainers never release a drained accumulator buffer
  // apply_Q on the tensor cores: k_umma_update<S, 1> writes columns
  // apply_n0 .. apply_n0 + S - 1 (those below apply_m) of Y = apply_y (device,
  // row stride apply_ldy) instead of the new panel; null in the steps
  double* apply_y;
  int64_t apply_ldy;
  int apply_m, apply_n0;
};

// One instance of a persistent batched launch (k_batch_step).
struct BatchInst {
  StepArgs a;
  int* tick;        // ticket area of the instance (TickLayout, 4 p + 4 ints)
  double* H;        // device outputs (or null)
  double* R;
  int tile_g;       // tile rows of the generic Gram (pass 2, and pass 1 without gram1)
  int tile_u;       // tile rows of the assembly
  int gram1;        // pass 1 by the register-tiled Gram (s in {1, 2, 4, 8, 16, 32})
  int digitize;     // write the digit planes of the new panel
};

// Entry (row, l) of L V for the 2D 5-point Dirichlet Laplacian of the step's
// operator (grid points row-major, n = op_nx op_ny): the same expression, in
// the same order, as k_laplace5, so a fused pass sees bit for bit the block
// the operator kernel would have written.
__device__ __forceinline__ double op_value(const StepArgs& a, int64_t row, int l) {
  const int nx = a.op_nx;
  const int64_t iy = row / nx;
  const int ix = (int)(row - iy * nx);
  const double* V = a.op_V;
  const int64_t ld = a.op_ldv;
  double v = 4.0 * V[row * ld + l];
  if (ix > 0) v -= V[(row - 1) * ld + l];
  if (ix < nx - 1) v -= V[(row + 1) * ld + l];
  if (iy > 0) v -= V[(row - nx) * ld + l];
  if (iy < a.op_ny - 1) v -= V[(row + nx) * ld + l];
  return v;
}

// TMA descriptors of a basis's digit planes: one box shape per kernel.
struct UmmaMaps {
  CUtensorMap upd;    // 16 8-row blocks (128 rows) of the 16 columns of one step, all planes
  CUtensorMap gram_lead;  // 2 8-row blocks of 16 column groups, the mixed Gram's leading planes
};

// Digit planes of the tensor-core form: 7 planes of 8-bit digits per value.
constexpr int kOzDigits = 7;
// uint32 words of one chunk's coefficient planes for Kmax rows and `ncols` columns.
__host__ __device__ inline int64_t oz_coef_words(int Kmax, int ncols) {
  const int ksteps = (Kmax + 15) / 16, ntiles = (ncols + 7) / 8;
  return (int64_t)ksteps * ntiles * kOzDigits * 64;
}

// Offset (in doubles) of column block c inside one chunk's tree factor.
__host__ __device__ inline int64_t tblock_offset(int c, int s) {
  return (int64_t)s * s * c * (c + 1) / 2;
}

// Kernel groups timed by the optional profiling hook (lo_basis_set_profiling).
enum KernelKind : int {
  kKindGram = 0,     // stage-1 Gram pass 1
  kKindLeaf = 1,     // per-chunk leaf factorizations
  kKindTree = 2,     // reduction (tree combine)
  kKindUpdate = 3,   // stage-2 assembly of U and of the new local block
  kKindApply = 4,    // apply_Q
  kKindRefine = 5,   // reiteration passes (new iterate + its Gram), passes >= 2
  kKindCount = 6
};

// Records a CUDA event before/after each kernel group when profiling is on.
struct ProfHook {
  virtual void mark(int kind, bool begin, cudaStream_t st) = 0;
  virtual ~ProfHook() {}
};

// Number of kernels this library has launched in this process.
long long launches();
void count_launches(int k);

// One-time function attributes of every kernel (call before stream capture).
cudaError_t launch_prepare();
// Fill X[0:count) with a deterministic synthetic pattern (chunk-size tuner only).
cudaError_t launch_fill_pattern(double* X, int64_t count, cudaStream_t st);

// Launchers (lo_kernels.cu).  All enqueue on `st` and return the launch error.
cudaError_t launch_step(const StepArgs& a, cudaStream_t st, ProfHook* hook);
// Y = Q C on the tensor cores (digit planes of every panel but the last, which
// is split on the fly); false when the basis has no such form (then the
// float64 kernels run).
bool umma_apply_supported(const StepArgs& a);
cudaError_t launch_umma_apply(const StepArgs& a, const double* C, int64_t ldc, int m, double* Y, int64_t ldy,
                              cudaStream_t st);
cudaError_t launch_apply_q(const StepArgs& a, const double* C, int m, int64_t ldc, double* Z,
                           double* Y, int64_t ldy, cudaStream_t st, ProfHook* hook);
// Tensor-core (Ozaki) launchers (lo_ozaki.cu).
cudaError_t launch_oz_gram(const StepArgs& a, int pass, cudaStream_t st);
cudaError_t launch_oz_ypass(const StepArgs& a, int pass, cudaStream_t st);
cudaError_t launch_oz_stage2(const StepArgs& a, cudaStream_t st);
bool oz_planes_supported(int s);
// Coefficients of an assembly product as tcgen05 B-operand images (lo_ozaki.cu).
// mode 1: images of k_umma_update; mode 2: the image of k_umma_update0.
cudaError_t launch_oz_coef_umma(const StepArgs& a, int nout, int pass, int mode, cudaStream_t st);
// tcgen05 forms over digit planes (lo_umma.cu): used when a.dig is set and the
// step has prior blocks (nb >= 1).
bool umma_enabled(const StepArgs& a);
// Whether the tensor-core Gram of pass 1 can form the operator's block on the fly.
bool umma_op_supported(const StepArgs& a);
cudaError_t launch_umma_gram(const StepArgs& a, int pass, cudaStream_t st);
// The mixed form's first Gram pass: the leading digits of both factors.
cudaError_t launch_umma_gram_mixed(const StepArgs& a, cudaStream_t st);
cudaError_t launch_umma_update(const StepArgs& a, int nout, int pass, cudaStream_t st);
// tcgen05 forms of a step without prior blocks (k = 0, s in {8, 16}); no digit planes needed.
bool umma0_enabled(const StepArgs& a);
cudaError_t launch_umma_gram0(const StepArgs& a, int pass, cudaStream_t st);
cudaError_t launch_umma_update0(const StepArgs& a, int nout, int pass, cudaStream_t st);
// Digit planes of the panel written by stage 2.
cudaError_t launch_umma_digitize(const StepArgs& a, cudaStream_t st);
cudaError_t umma_set_attrs();
// Host: TMA descriptors over a digit-plane array of `panels` panels.
cudaError_t umma_make_maps(uint8_t* dig, int s, int panels, int64_t dtiles, UmmaMaps* maps);
// uint32 words of one chunk's coefficient images (both assembly products).
int64_t umma_coef_words(int Kmax, int s);
bool oz_supported(int s);
// Widest block of a one-block basis that the tensor-core forms leave to the
// native float64 kernels.
constexpr int kNativeMaxS = 4;
cudaError_t oz_set_attrs();

cudaError_t launch_laplace5(int nx, int ny, int s, const double* X, int64_t ldx, double* Y,
                            int64_t ldy, cudaStream_t st);

// Persistent batched launch (lo_kernels.cu).  batch_fill: fill the host
// descriptor of one instance (tile rows, route flags) and return whether the
// persistent kernel can run it; batch_tick_ints: its ticket area size;
// launch_batch: init + the persistent kernel over d_insts (device copies),
// pref the phase-major item prefix (6 x (ninst + 1) ints, device), counters
// 2 ints (device).  smem: dynamic shared memory of the kernel.
bool batch_fill(BatchInst* bi);
int batch_tick_ints(int p);
size_t batch_smem(const BatchInst* insts, int ninst);
cudaError_t launch_batch(BatchInst* d_insts, int ninst, const int* d_pref, int* d_counters, size_t smem,
                         cudaStream_t st);

}  // namespace lo

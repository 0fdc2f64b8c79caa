/*
 * lo.h — C ABI of the GB300 block-orthogonalization library (liblo).
 *
 * Implements the project-and-normalize (PQR) step of block Arnoldi / block
 * GMRes as TreeTSPQR on a locally orthogonal basis, after Dreier & Engwer,
 * "A Hardware-aware and Stable Orthogonalization Framework", arXiv 2204.13393:
 *
 *   PQR problem, eq. (pqr), Sec. 1: for orthonormal Q (n x k) and a new block
 *   X (n x s) find orthonormal U (n x s) with Q^T U = 0, P (k x s) and upper
 *   triangular N (s x s, positive diagonal) such that
 *        [Q X] = [Q U] [[I, P], [0, N]].
 *   In block Arnoldi (Alg. 1) P and N are the new column block of the block
 *   Hessenberg matrix; this API returns them as H (= P) and R (= N).
 *
 *   Locally orthogonal representation, Sec. 4.1: the basis is never stored
 *   explicitly; it is Q = diag(Q_1 .. Q_p) [T_1; ..; T_p] with local
 *   orthonormal Q_i (one per row chunk) and upper-triangular tree factors T_i
 *   whose stack is orthonormal.
 *
 *   TreeTSPQR, Alg. 9: a local PQR per chunk (BCGS-PIP, Alg. 7, reiterated as
 *   BCGS-PIP+, Alg. 8: by default always, optionally only when the block is
 *   ill-conditioned), a reduction PQR of the stacked small factors
 *   (BCGS-PIP+), and the assembly of U from the block-wise products of
 *   Sec. 4.1.
 *
 * Conventions for every entry point:
 *   - All matrices are float64, row-major.  "ld" is the row stride in
 *     elements (ld >= number of columns).
 *   - Device work is enqueued on the stream given at lo_basis_create.
 *   - Pointers to n-row matrices (W, U, Y) may be device pointers or host
 *     pointers (pageable or pinned); host data is staged through device
 *     buffers owned by the basis, with the copies on the basis stream.
 *   - The small outputs H and R are written to device or host memory as the
 *     pointer's kind says.
 *   - Functions return an lo_status; they never abort or throw across the ABI.
 *   - The library allocates only in lo_basis_create, and lazily the host
 *     staging buffers and apply_Q's scratch (grown to the largest m seen).
 *     Calls on one basis are not thread-safe.
 */
#ifndef LO_H_
#define LO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lo_status {
  LO_OK = 0,
  LO_ERR_INVALID_ARG = 1,      /* bad pointer, size, stride or option           */
  LO_ERR_CAPACITY = 2,         /* basis already holds max_blocks blocks         */
  LO_ERR_CHUNK_TOO_SMALL = 3,  /* chunk_rows < max_blocks*s or n < max_blocks*s */
  LO_ERR_BREAKDOWN = 4,        /* a Cholesky pivot <= tolerance: the new block  */
                               /* is (numerically) rank deficient against the   */
                               /* basis and deflation (lo_options.deflation_tol,*/
                               /* Sec. 3) is off.  Exact zeros on some chunks   */
                               /* are not a breakdown (see lo_orthogonalize)    */
  LO_ERR_NONFINITE = 5,        /* NaN or Inf reached a small factor             */
  LO_ERR_TIMEOUT = 6,          /* a bounded device wait gave up                 */
  LO_ERR_CUDA = 7,             /* a CUDA runtime call failed                    */
  LO_ERR_OOM = 8,              /* device or pinned allocation failed            */
  LO_ERR_UNSUPPORTED = 9       /* option combination not implemented            */
} lo_status;

/* Arithmetic of the O(n) passes. */
typedef enum lo_precision {
  LO_PREC_FP64 = 0,        /* every product in native float64                    */
  LO_PREC_MIXED_FP32 = 1,  /* first-pass Gram/projection in float32 (each column */
                           /* of W scaled per slab by a power of two), then      */
                           /* float64 shifted Cholesky, one float64 CholeskyQR2- */
                           /* style refinement pass, float64 tree and update     */
                           /* (Alg. 8 pattern)                                    */
  LO_PREC_FP64_TC = 2,     /* float64-accurate products of the O(n) passes on the */
                           /* tensor cores: every float64 value is split into 7   */
                           /* 8-bit digits against its column's largest exponent */
                           /* (error-free splitting of Ozaki et al., Numer.      */
                           /* Algorithms 59, 2012), the 28 significant digit      */
                           /* products run as fp16 mma with exact float32        */
                           /* accumulation, and are recombined in 64-bit         */
                           /* integers.  Small factors stay float64.  Requires   */
                           /* s in {1, 2, 4, 8, 16, 32} (any s <= 4 when         */
                           /* max_blocks = 1); values below 2^-1022              */
                           /* (subnormals) count as zero.  A one-block basis     */
                           /* (max_blocks = 1) with s <= 4 runs the native       */
                           /* float64 kernels (its products are too narrow for   */
                           /* the tensor cores to pay)                           */
  LO_PREC_MIXED_TC = 3     /* mixed form on the tensor-core path: the first Gram */
                           /* pass reduced (with digit planes and prior blocks:  */
                           /* the leading four digits of both factors on the     */
                           /* tensor cores, a 32-bit split, unshifted float64    */
                           /* Cholesky with a shifted retry on breakdown; else   */
                           /* float32 with a fixed shift), every further pass    */
                           /* and the assembly as LO_PREC_FP64_TC                */
                           /* (max_blocks = 1, s <= 4: as LO_PREC_MIXED_FP32)    */
} lo_precision;

/* Local sub-algorithm (the "local subalgorithm" of Alg. 9). */
typedef enum lo_leaf {
  LO_LEAF_AUTO = 0,        /* BCGS-PIP, plus the PIP+ reiteration when the local */
                           /* condition estimate says the single pass would lose */
                           /* orthogonality (decided on the device; no host      */
                           /* synchronization).  Suited to well-conditioned,     */
                           /* independent blocks; in a Krylov sequence the local */
                           /* losses below the estimate accumulate.               */
  LO_LEAF_PIP = 1,         /* BCGS-PIP, Alg. 7: one Gram pass                    */
  LO_LEAF_PIP2 = 2,        /* BCGS-PIP+, Alg. 8: two Gram passes (the default),  */
                           /* a third when the estimate still asks for it; a     */
                           /* first-pass breakdown retries with the shift of     */
                           /* shifted CholeskyQR3 and forces two more passes     */
  LO_LEAF_HH = 3           /* Householder QR (Alg. 6, sign rule sigma = -sgn of  */
                           /* the pivot) of each chunk in the step without prior */
                           /* blocks (k = 0, the tall-skinny QR): one CTA per    */
                           /* chunk, the chunk tile in shared memory, so the     */
                           /* block is read once and no Gram matrix is formed    */
                           /* (stable at any condition number, no shifted        */
                           /* retry).  A chunk larger than one tile (rows * s * 8*/
                           /* above 200 KiB) is walked as sub-tiles in the order */
                           /* of FlatTSPQR (Alg. 10: each sub-tile factored      */
                           /* stacked under the previous R, the local factor     */
                           /* formed backwards), so the recursion has three      */
                           /* levels: sub-tiles, chunk, reduction tree.  The     */
                           /* reduction stays BCGS-PIP+ (the paper's choice at   */
                           /* the level above the node, Sec. 5.3) and the local  */
                           /* panel is the explicit Householder Q_i.  Steps with */
                           /* prior blocks run BCGS-PIP+                         */
} lo_leaf;

/*
 * Storage of the local panels for the tensor-core forms (LO_PREC_FP64_TC,
 * LO_PREC_MIXED_TC).  Both products of a step read every earlier local panel
 * once per pass; the tensor cores take each float64 value as 7 exact 8-bit
 * digits aligned to its column's largest exponent.  With digit planes the
 * digits are made once, when the panel is created, and kept beside the
 * float64 values as fp16 digits (7 per value, the sign in each, 14 bytes per
 * value) in the tensor cores' operand order: the panels take 2.75 times the
 * memory of float64 alone and the passes stream MMA operands instead of
 * re-splitting float64 values.  LO_PREC_FP64_TC gives bitwise the same
 * results either way; LO_PREC_MIXED_TC's first pass needs the planes for its
 * 32-bit digit split and otherwise runs in float32.
 * Memory per basis with planes: max_blocks * s * (8 + 14) bytes per row.
 */
typedef enum lo_digit_planes {
  LO_PLANES_AUTO = 0, /* planes for the tensor-core forms when s is 8, 16 or 32  */
  LO_PLANES_OFF = 1   /* split the float64 panels again in every pass           */
} lo_digit_planes;

typedef struct lo_options {
  int32_t precision;   /* lo_precision, default LO_PREC_FP64                     */
  int32_t leaf;        /* lo_leaf, default LO_LEAF_PIP2                          */
  int32_t reduction;   /* reduction sub-algorithm: 0 = AUTO (BCGS-PIP+, plus a   */
                       /* third iteration when the estimate below asks for it), */
                       /* 1 = BCGS-PIP (one iteration), 2 = BCGS-PIP+ exactly.  */
                       /* Default 0                                              */
  int32_t sync;        /* 1 (default): lo_orthogonalize waits for its device     */
                       /* work and returns the device status.  0: asynchronous;  */
                       /* a device error is latched and returned by the next     */
                       /* call or by lo_basis_sync.                              */
  double refine_tol;   /* reiterate when eps * kappa^2 exceeds this, where       */
                       /* kappa = ||X||_F ||N^{-1}||_F for the block X and its  */
                       /* normalizer N (the Gram cancellation factor).          */
                       /* <= 0 selects the default 1e-13.                        */
  int32_t digit_planes;  /* lo_digit_planes, default LO_PLANES_AUTO              */
  int32_t test_stall;    /* test hook, default 0.  1: in a step with prior       */
                         /* blocks, the tensor-core Gram's issuing thread issues */
                         /* no loads and no MMAs, so the kernel's bounded waits  */
                         /* (about 0.25 s each) expire and the step returns      */
                         /* LO_ERR_TIMEOUT with the basis unchanged (the timeout */
                         /* path; no fault, nothing left in flight).  2: the     */
                         /* Gram's drainer warps never release a drained         */
                         /* accumulator buffer, so the issuer's wait for it      */
                         /* expires after loads and MMAs were issued; it drains  */
                         /* them and the step returns LO_ERR_TIMEOUT likewise    */
  double deflation_tol;  /* delta >= 0, default 0 (off).  delta > 0: the        */
                         /* deflated PQR of Sec. 3 (t < s), kept as t = s: a    */
                         /* column of W whose distance to the span of the basis */
                         /* and of the earlier kept columns is at most          */
                         /* delta ||W||_F is dropped -- its column of U is zero */
                         /* and its row of R is zero -- instead of reporting    */
                         /* LO_ERR_BREAKDOWN.  Decided by the Cholesky pivots   */
                         /* (squared distances) of the local first pass and of  */
                         /* the reduction against max(delta^2, 64 s eps)        */
                         /* ||W||_F^2: the Gram pivots carry rounding noise of  */
                         /* order eps ||W||_F^2, so delta below about 3e-7 acts */
                         /* as that floor.  No shifted retry then.  Float64     */
                         /* forms only (LO_PREC_FP64, LO_PREC_FP64_TC); the     */
                         /* mixed forms return LO_ERR_UNSUPPORTED.  A deflated  */
                         /* block still takes a slot of the basis (its dropped  */
                         /* columns are zero columns of Q).                     */
} lo_options;

typedef struct lo_basis lo_basis;

/* Fill *opt with the defaults. */
void lo_options_default(lo_options* opt);

/*
 * Create an empty basis for n-row blocks of width s, holding up to max_blocks
 * blocks, with local row chunks of chunk_rows rows (p = max(1, n / chunk_rows)
 * chunks; the remainder rows join the last chunk).  The basis is the locally
 * orthogonal representation of Sec. 4.1 (one local factor Q_i per row chunk,
 * the tree factors T_i), split into the local subproblems of Sec. 5.1.3
 * (p = n / local size); the chunk size is the local problem size that
 * Sec. 6.2 studies.  Every chunk must have at least max_blocks*s rows so that
 * each local problem has full rank (LO_ERR_CHUNK_TOO_SMALL otherwise).
 * Requires 1 <= s <= 32 and max_blocks*s <= 1024.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream) of the current device.  opt may
 * be NULL (defaults).  Allocates all device memory of the basis (local panels
 * n*max_blocks*s doubles, tree factors, scratch).  On failure *out is NULL.
 */
lo_status lo_basis_create(int64_t n, int32_t s, int32_t max_blocks, int32_t chunk_rows,
                          const lo_options* opt, void* cuda_stream, lo_basis** out);

/* Free everything owned by the basis.  NULL-safe. */
void lo_basis_destroy(lo_basis* b);

/* Drop all blocks (e.g. at a GMRes restart); keeps the allocations. */
lo_status lo_basis_reset(lo_basis* b);

/* Number of blocks currently in the basis (k = blocks * s columns): the
 * number of PQR steps of Alg. 2 / Alg. 1 solved so far since create, reset or
 * truncate.  -1 for NULL. */
int32_t lo_basis_num_blocks(const lo_basis* b);

/* Number of local chunks p. */
int32_t lo_basis_num_chunks(const lo_basis* b);

/*
 * One PQR step (Alg. 9): orthogonalize the n x s block W (row stride ldw)
 * against the current basis (k = num_blocks*s columns).  Writes
 *   U (n x s, row stride ldu)  the new orthonormal block, explicit (Sec. 1:
 *                              U is needed explicitly to apply the operator),
 *   H (k x s, row-major)       the projection P = Q^T W (may be NULL if k = 0),
 *   R (s x s, row-major)       the normalizer N, upper triangular, diag > 0,
 * and appends the block to the basis.  U may alias W (same pointer, same ld).
 * H and R may be NULL if not wanted.  On any error the basis is unchanged
 * (its block count is not advanced) and U, H, R are undefined.  A block that
 * is exactly zero on some chunks, or in some of its columns there, is
 * supported as long as it has full rank against the basis overall: the
 * chunk's local panel then keeps zero columns (Sec. 3, t = s with the rank
 * deficiency carried in the normalizer).  The results are homogeneous in W:
 * W scaled by 2^j gives the same U and H, R scaled by 2^j, bit for bit.
 */
lo_status lo_orthogonalize(lo_basis* b, const double* W, int64_t ldw,
                           double* U, int64_t ldu, double* H, double* R);

/*
 * One PQR step of block Arnoldi (Alg. 1) with the operator fused into the
 * step: orthogonalize W = L V, where L is the 2D 5-point Dirichlet Laplacian
 * on an nx x ny grid (the operator of lo_laplace5_apply, n = nx ny) and V the
 * previous basis block, against the current basis.  The first Gram pass reads
 * V and forms each value of W from the stencil as it needs it (no separate
 * operator pass: the Gram does not read a materialized W), writing W once
 * into U, where the later passes and the assembly read it; U then receives
 * the new orthonormal block as in lo_orthogonalize.  The result is bit for
 * bit that of lo_laplace5_apply followed by lo_orthogonalize.  Forms whose
 * first pass cannot form the block on the fly (the mixed forms, the
 * tensor-core form without digit planes, a step without prior blocks, the
 * Householder leaf) apply the operator into U first.
 *   V  device, n x s, row stride ldv >= s (read only);
 *   U  device, n x s, row stride ldu >= s; must not overlap V;
 *   H, R as in lo_orthogonalize (host or device, may be NULL).
 */
lo_status lo_orthogonalize_laplace5(lo_basis* b, int32_t nx, int32_t ny, const double* V, int64_t ldv, double* U,
                                    int64_t ldu, double* H, double* R);

/*
 * Y = Q C for the current basis (Sec. 5.1: the product QC of the second
 * stage), computed chunk-wise as Y_i = Q_i (T_i C).  C is k x m row-major
 * (k = num_blocks*s, row stride ldc >= m), host or device; Y is n x m
 * (row stride ldy >= m), host or device.  With C = I_k this materializes the
 * explicit basis.  1 <= m <= 1024.  A basis with digit planes (tensor-core
 * forms, s in {8, 16, 32}, at least two blocks) computes the products on the
 * tensor cores with float64 accuracy, one assembly per s columns of C; other
 * bases use float64 arithmetic.  Errors latched by the device (a non-finite C:
 * LO_ERR_NONFINITE; LO_ERR_TIMEOUT) are returned when the call synchronizes
 * (host Y or the sync option), else by the next call or lo_basis_sync.
 */
lo_status lo_apply_Q(lo_basis* b, const double* C, int32_t m, int64_t ldc,
                     double* Y, int64_t ldy);

/*
 * Orthogonalize count independent problems (uneven n, s, k), one block each:
 * for j < count, the same as lo_orthogonalize(bases[j], W[j], ldw[j], U[j],
 * ldu[j], H[j], R[j]) -- one PQR step (eq. (pqr), Alg. 9) per problem.  The
 * paper solves one problem at a time; running many small ones together is
 * this library's answer to Sec. 6.2's observation that small local problems
 * leave the hardware idle.  The steps of all problems are captured once into
 * one CUDA graph whose branches run concurrently (a fork over 8 internal
 * streams, joined back into the stream of bases[0]); the graph is cached under
 * the call's arguments (each basis by a process-unique id, its block count,
 * the buffers and strides) and a repeat call with the same arguments is a
 * single graph launch.  Destroying a basis evicts every cached graph that
 * names it.  All bases must live on the same device and be distinct.  W, U,
 * H, R may be device or host pointers, as in lo_orthogonalize (host W is
 * staged through the basis's device buffer before the graph runs; host U, H,
 * R are copied out after it, on the stream of bases[0]); H, R, H[j], R[j] may
 * be NULL.  Waits for the work.  Returns the first error; bases without error
 * advance, the others are unchanged.
 */
lo_status lo_orthogonalize_batched(lo_basis* const* bases, int32_t count,
                                   const double* const* W, const int64_t* ldw,
                                   double* const* U, const int64_t* ldu,
                                   double* const* H, double* const* R);

/*
 * Route of lo_orthogonalize_batched's instances (process-wide; part of the
 * cached graphs' key):
 *   0 (default) auto: an instance of the native float64 form
 *     (LO_PREC_FP64) of at most 4e6 n (k + s) that the persistent launch can
 *     run goes into it, every other one gets its own branch of the graph (on
 *     GB300 the tensor-core forms' own kernels beat the float64 pipe the
 *     persistent launch computes on);
 *   1: the persistent launch for every instance it can run;
 *   2: graph branches only (each instance's own kernel sequence).
 * The persistent launch is one kernel (after a small init kernel) over a work
 * list of (instance, row slab) and (instance, chunk) items of all its
 * instances, with per-chunk and per-instance tickets handing the leaf and
 * reduction factorizations to the CTA that finishes last (TreeTSPQR, Alg. 9,
 * BCGS-PIP+ local and reduction solvers, float64 arithmetic on the CUDA cores;
 * for a tensor-core basis the new panel's exponents and digit planes are
 * kept current).  It runs instances created with the float64 forms
 * (LO_PREC_FP64, LO_PREC_FP64_TC), the BCGS-PIP+ leaf (or the Householder
 * leaf past the first block), a reiterating reduction, no deflation, and
 * device buffers; an instance whose estimate asks for a third local pass or
 * reduction iteration (or the shifted retry) is redone on the regular path
 * within the same call.  Sec. 6.2 finds small local problems leave the
 * hardware idle; many such steps fill it together.
 * lo_batched_persistent_count: instances the last used cached graph runs in
 * the persistent launch (for tests and the benchmark).
 */
lo_status lo_set_batched_route(int32_t mode);
int32_t lo_batched_persistent_count(void);

/*
 * Drop the trailing blocks so that num_blocks (<= the current count) remain.
 * The representation of the first num_blocks blocks is not affected by later
 * steps, so this is exact (a truncated restart, or re-running a step).
 */
lo_status lo_basis_truncate(lo_basis* b, int32_t num_blocks);

/*
 * Autotuner: time one step at half capacity for every candidate chunk size
 * (powers of two from max(256, max_blocks*s) up to n) on a synthetic block of
 * this shape and return the fastest in *chunk_rows.  Allocates temporary
 * device memory; results are memoized per (log2 n in quarter steps, s,
 * max_blocks, precision, leaf).  opt may be NULL.
 */
lo_status lo_tune_chunk_rows(int64_t n, int32_t s, int32_t max_blocks, const lo_options* opt,
                             void* cuda_stream, int32_t* chunk_rows);

/*
 * Inspection of the batched graph cache (for tests): lo_basis_id returns the
 * basis's process-unique id (0 for NULL; ids are never reused);
 * lo_batched_cache_entries returns how many cached graphs name the basis with
 * that id (basis_id = 0: all cached graphs).  Host-only, no device work.
 */
uint64_t lo_basis_id(const lo_basis* b);
int32_t lo_batched_cache_entries(uint64_t basis_id);

/*
 * Autotuner of the leaf: the chunk size of each leaf from lo_tune_chunk_rows
 * (BCGS-PIP+; the Householder leaf for a one-block basis), then the step
 * without prior blocks (k = 0, where the two leaves differ) timed with each on
 * a synthetic block of this shape; *leaf and *chunk_rows receive the faster
 * pair (for a basis of several blocks the chunk size is BCGS-PIP+'s, which its
 * later steps want).  The paper chooses the sub-algorithm per hardware level
 * (Sec. 5.3); here the choice is measured.  Both leaves are stable, so the
 * choice is on speed alone.  Allocates temporary device memory.
 */
lo_status lo_tune_leaf(int64_t n, int32_t s, int32_t max_blocks, const lo_options* opt, void* cuda_stream,
                       int32_t* leaf, int32_t* chunk_rows);

/* Wait for the basis stream and return (and clear) any latched device error. */
lo_status lo_basis_sync(lo_basis* b);

/*
 * Copy the local factor of chunk i (its rows of the local panels, n_i x k,
 * row-major with row stride k) and its tree factor T_i (k x k, row-major,
 * zeros below the diagonal) to host memory.  For tests and inspection.
 * Either destination may be NULL.  *rows receives n_i if rows != NULL.
 */
lo_status lo_basis_export_chunk(lo_basis* b, int32_t chunk, double* Qi_host,
                                double* Ti_host, int64_t* rows);

/* y = L x for the 2D 5-point Dirichlet Laplacian on an nx x ny grid
 * (row-major grid points, n = nx*ny), applied to s columns at once: X and Y
 * are n x s row-major device arrays with row strides ldx, ldy.  This is the
 * operator of the block-GMRes test workload, not part of the PQR step. */
lo_status lo_laplace5_apply(int32_t nx, int32_t ny, int32_t s, const double* X, int64_t ldx,
                            double* Y, int64_t ldy, void* cuda_stream);

/*
 * Measurement hooks (used by the benchmark; not needed for normal use).
 * lo_launch_count: number of kernels the library has launched in this process.
 * lo_basis_set_profiling: when enabled, every group of kernels of this basis
 *   (0 stage-1 Gram pass 1, 1 leaf factorizations, 2 reduction, 3 stage-2
 *   update, 4 apply_Q, 5 reiteration passes) is bracketed by CUDA events on the
 *   basis stream.
 * lo_basis_profile_read: waits for the recorded events and returns, per group,
 *   the summed elapsed milliseconds and the number of bracketed intervals since
 *   the last read (nkinds >= 6 entries in both arrays).
 */
long long lo_launch_count(void);
/* Rank t of the last step's normalizer R (the nonzero diagonal entries; t < s
 * only with deflation).  Waits for the step. */
lo_status lo_basis_last_rank(lo_basis* b, int32_t* rank);
/* Local Gram passes and reduction iterations the last step ran (waits for it). */
lo_status lo_basis_last_step_info(lo_basis* b, int32_t* passes, int32_t* tree_iterations);
lo_status lo_basis_set_profiling(lo_basis* b, int32_t enable);
lo_status lo_basis_profile_read(lo_basis* b, double* ms, int64_t* intervals, int32_t nkinds);

/*
 * Allocation-free tall-skinny QR: W = U R with the first step of the method
 * (empty basis, k = 0: local Gram per chunk, leaf Cholesky with the BCGS-PIP+
 * reiteration -- the library's default leaf, LO_LEAF_PIP2 --, reduction of the
 * stacked factors, assembly of U), for callers that cannot allocate device
 * memory: code that runs where the memory budget is fixed up front (an
 * application that owns every device allocation through its own pool, a
 * process that must not grow its footprint after start-up) or a host thread
 * for which cudaMalloc/cudaFree, with their implicit device synchronization,
 * are not permitted.  The paper has no counterpart; it is an interface
 * variant of the k = 0 step of lo_orthogonalize.
 *
 *   n, s, chunk_rows  as for lo_basis_create with max_blocks = 1 (1 <= s <= 32,
 *                     every chunk at least s rows);
 *   W                 device, n x s, row stride ldw >= s (read only);
 *   U                 device, n x s, row stride s (written; it is also the
 *                     working panel of the step).  U may equal W when
 *                     ldw == s (in place); otherwise they must not overlap;
 *   R                 device, s x s row-major, upper triangular, diag > 0;
 *   cuda_stream       cudaStream_t of the current device (NULL = default).
 *
 * It allocates nothing: all scratch is one fixed 16 MiB array in device
 * memory that every device loading the library holds until the process exits.
 * A problem whose scratch does not fit (lo_tsqr_noalloc_scratch gives the
 * size: roughly p chunks * (8 s^2 + 1) doubles plus one s x s tile per
 * 256-row slab) returns LO_ERR_CAPACITY before any CUDA call.  Every call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress; after a device reset the module is reloaded, possibly
 * elsewhere); the first call on a device also loads the module, so make it
 * before any stream capture.  Every call shares the array and leaves its
 * contents behind, so calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialized by the caller.  The call waits
 * for its stream and returns the step's status (LO_ERR_BREAKDOWN for a
 * numerically rank-deficient W, LO_ERR_NONFINITE for NaN/Inf).
 */
lo_status lo_tsqr_noalloc(int64_t n, int32_t s, int32_t chunk_rows, const double* W, int64_t ldw,
                          double* U, double* R, void* cuda_stream);

/*
 * Host-only size query for lo_tsqr_noalloc (no CUDA call): *need_bytes gets
 * the scratch the problem (n, s, chunk_rows) needs, *capacity_bytes the size
 * of the fixed array (either may be NULL).  Returns LO_OK if it fits,
 * LO_ERR_CAPACITY if not, and the argument errors of lo_tsqr_noalloc
 * (LO_ERR_INVALID_ARG, LO_ERR_CHUNK_TOO_SMALL) for bad sizes.
 */
lo_status lo_tsqr_noalloc_scratch(int64_t n, int32_t s, int32_t chunk_rows, uint64_t* need_bytes,
                                  uint64_t* capacity_bytes);

/* Human-readable name of a status code (static string). */
const char* lo_status_string(lo_status st);

#ifdef __cplusplus
}
#endif

#endif /* LO_H_ */

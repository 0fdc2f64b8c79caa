// Float64 kernels of one TreeTSPQR step (Alg. 9) on the locally orthogonal
// basis of Sec. 4.1, plus apply_Q and the 5-point Laplacian of the test
// workload.
//
// Step = stage 1 (Gram passes + local leaf factorizations), reduction
// (tree combine of the stacked small factors), stage 2 (assembly of U and of
// the new local block).  Every reduction has a fixed order, so two runs give
// bit-identical results.  No kernel waits on another CTA; breakdowns are
// reported through the status flag word, never by trapping.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cstdint>

#include "lo_internal.h"
#include "lo_oz_common.cuh"
#include "lo_recombine.h"

namespace lo {
namespace {

__device__ __forceinline__ void set_status(int* flags, lo_status st) {
  atomicOr(&flags[kFlagStatus], 1 << (int)st);
}

__device__ __forceinline__ double* chunk_small(const StepArgs& a, int c) {
  return a.small + (int64_t)c * SmallLayout::make(a.Kmax, a.s).stride;
}

__device__ __forceinline__ int passes_run(const StepArgs& a) {
  int L = 1;
  for (int t = 2; t <= kMaxPass; ++t)
    if (a.flags[kFlagPass + t - 1]) L = t;
  return L;
}

// ---------------------------------------------------------------------------
// Small dense helpers executed by a whole CTA on shared-memory matrices.

// In-place upper Cholesky of the s x s symmetric matrix M (row-major, smem):
// afterwards the upper triangle holds N with N^T N = M, the lower is zero.
// A pivot that is exactly zero with the rest of its row exactly zero (the
// block is exactly zero in that component, e.g. a column that vanishes on a
// chunk) leaves a zero row of N: Sec. 3 allows keeping t = s and carrying the
// rank deficiency in N.  Any other pivot <= tol (or non-finite) sets *fail
// (shared memory, zeroed by the caller) and, when flags is not null, latches
// LO_ERR_BREAKDOWN / LO_ERR_NONFINITE; the pivot is replaced by 1 so that no
// NaN propagates.
//
// defl > 0 (the deflated PQR of Sec. 3): a finite pivot d <= defl (the squared
// distance of column i to the span of what precedes it) is deflated as well:
// row i of N is set to zero and eliminates nothing.
__device__ void cta_cholesky(double* M, int s, double tol, int* flags, int* fail, double defl = 0.0) {
  for (int i = 0; i < s; ++i) {
    if (threadIdx.x == 0) {
      double d = M[i * s + i];
      bool zero_row = d == 0.0;
      for (int j = i + 1; j < s && zero_row; ++j) zero_row = M[i * s + j] == 0.0;
      if (!zero_row && defl > 0.0 && isfinite(d) && d <= defl) {
        for (int j = i + 1; j < s; ++j) M[i * s + j] = 0.0;
        zero_row = true;
      }
      if (zero_row) {
        d = 0.0;
      } else if (!isfinite(d)) {
        if (flags) set_status(flags, LO_ERR_NONFINITE);
        *fail = 1;
        d = 1.0;
      } else if (!(d > tol)) {
        if (flags) set_status(flags, LO_ERR_BREAKDOWN);
        *fail = 1;
        d = 1.0;
      }
      M[i * s + i] = sqrt(d);
    }
    __syncthreads();
    const double piv = M[i * s + i];
    if (piv == 0.0) {  // zero row: nothing to divide, nothing to eliminate
      __syncthreads();
      continue;
    }
    for (int j = i + 1 + threadIdx.x; j < s; j += blockDim.x) M[i * s + j] /= piv;
    __syncthreads();
    const int rem = s - i - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int j = i + 1 + e / rem, l = i + 1 + e % rem;
      if (l >= j) M[j * s + l] -= M[i * s + j] * M[i * s + l];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < s * s; e += blockDim.x)
    if (e / s > e % s) M[e] = 0.0;
  __syncthreads();
}

// Cholesky of M with the shifted retry of shifted CholeskyQR3 (Fukaya,
// Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 42, 2020):
// when allow_shift is set and the plain factorization breaks down (the block
// is ill-conditioned beyond eps*kappa^2 < 1), factor M + sigma*I with
// sigma = 11 (rows*s + s(s+1)) eps trace(G) instead and return true; the
// caller then forces two further reiterations.  Without allow_shift a
// breakdown latches the status.  save: s*s shared scratch.
__device__ bool cta_cholesky_shifted(double* M, double* save, int s, double tol, double sigma, bool allow_shift,
                                     int* flags, int* fail, double defl = 0.0) {
  if (threadIdx.x == 0) *fail = 0;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) save[e] = M[e];
  __syncthreads();
  cta_cholesky(M, s, tol, allow_shift ? nullptr : flags, fail, defl);
  const bool failed = *fail != 0;
  __syncthreads();
  if (!failed || !allow_shift) return false;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) M[e] = save[e] + ((e / s == e % s) ? sigma : 0.0);
  if (threadIdx.x == 0) *fail = 0;
  __syncthreads();
  cta_cholesky(M, s, tol, flags, fail);
  return true;
}

// X = N^{-1} for upper-triangular N (smem), column by column.  Zero rows of
// N (exactly zero components, see cta_cholesky) give zero rows and columns
// of X: X = (N + E)^{-1} with those columns cleared (E: ones on the zero
// rows' diagonal), so that Y X has zero columns there and Y X N = Y for Y in
// the row space of N.
__device__ void cta_upper_inverse(const double* N, double* X, int s) {
  for (int l = threadIdx.x; l < s; l += blockDim.x) {
    const bool zero_col = N[l * s + l] == 0.0;
    for (int i = s - 1; i >= 0; --i) {
      double v = (i == l) ? 1.0 : 0.0;
      if (i <= l && !zero_col && N[i * s + i] != 0.0) {
        for (int j = i + 1; j <= l; ++j) v -= N[i * s + j] * X[j * s + l];
        v /= N[i * s + i];
      } else {
        v = 0.0;
      }
      X[i * s + l] = v;
    }
  }
  __syncthreads();
}

// C = A B for s x s matrices in smem (C must not alias A or B).
__device__ void cta_matmul_ss(const double* A, const double* B, double* C, int s) {
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e / s, j = e % s;
    double v = 0.0;
    for (int q = 0; q < s; ++q) v += A[i * s + q] * B[q * s + j];
    C[e] = v;
  }
  __syncthreads();
}

// Amplification estimate of a BCGS-PIP solve: kappa = ||X||_F ||N^{-1}||_F with
// ||X||_F^2 = trace(G).  The Gram G - P^T P loses about eps * kappa^2 of its
// relative accuracy to cancellation (the block's norm against its part
// orthogonal to the basis), which is the orthogonality the single pass loses
// (Sec. 3: O(eps kappa^2)); ||N||_F alone would miss the cancellation.
__device__ double cta_pip_kappa(double trG, const double* Ninv, int s, double* red) {
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int e = 0; e < s * s; ++e) b += Ninv[e] * Ninv[e];
    red[0] = sqrt(trG) * sqrt(b);
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Step bookkeeping: which passes / tree iterations are forced.

__global__ void k_step_begin(int* flags, int force_pass2, int force_tree2) {
  if (threadIdx.x == 0) {
    for (int t = 1; t <= kMaxPass; ++t) flags[kFlagPass + t - 1] = (t == 1) || (t == 2 && force_pass2);
    for (int t = 1; t <= kMaxTreeIter; ++t) flags[kFlagTree + t - 1] = (t == 1) || (t == 2 && force_tree2);
  }
}

// float64 -> float32 with integer operations only (round toward zero; |x| below
// 2^-126 flushes to a signed zero, above the float32 range becomes a signed
// infinity).  Used by the float32 first pass of the mixed form so that it never
// issues work to GB300's narrow float64 pipe.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned r = sign | ((unsigned)(e - 896) << 23) | mant;
  if (e < 897) r = sign;
  if (e > 1150) r = sign | 0x7F800000u;
  return __uint_as_float(r);
}

// f32_trunc(x * 2^sh) for an integer sh, by moving the exponent field
// (zero and subnormal x give a signed zero).  The float32 first pass scales
// each column of the block by a power of two so that its largest entry on
// the slab lies in [1, 2): the float32 products then neither overflow nor
// underflow whatever the block's magnitude, and the scaling is undone
// exactly in float64 on the partial.
__device__ __forceinline__ float f32_trunc_shift(double x, int sh) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu), es = e + sh;
  if (e == 0 || es < 897) return __uint_as_float(sign);
  if (es > 1150) return __uint_as_float(sign | 0x7F800000u);
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  return __uint_as_float(sign | ((unsigned)(es - 896) << 23) | mant);
}

// Largest biased exponent of each of the S columns of the block over the
// slab's rows (0 for a zero column), into hs[0 .. S).  Whole CTA.
template <typename F>
__device__ __forceinline__ void slab_col_exponents(int* hs, int S, int rows, F&& value) {
  if ((int)threadIdx.x < S) hs[threadIdx.x] = 0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < rows * S; idx += blockDim.x) {
    const int r = idx / S, l = idx - r * S;
    atomicMax(&hs[l], (int)((((unsigned long long)__double_as_longlong(value(r, l))) >> 52) & 0x7FF));
  }
  __syncthreads();
}

// The shift that brings a column with largest biased exponent h to [1, 2).
__device__ __forceinline__ int col_shift(int h) { return h == 0 ? 0 : 1023 - h; }

template <typename Acc>
__device__ __forceinline__ Acc load_as(const double* p);
template <>
__device__ __forceinline__ double load_as<double>(const double* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_as<float>(const double* p) { return f32_trunc(__ldg(p)); }
template <typename Acc>
__device__ __forceinline__ Acc load_scaled(const double* p, int sh);
template <>
__device__ __forceinline__ double load_scaled<double>(const double* p, int) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_scaled<float>(const double* p, int sh) { return f32_trunc_shift(__ldg(p), sh); }

// ---------------------------------------------------------------------------
// Stage 1, Gram pass `pass` over one row slab of one chunk (Alg. 7 first line,
// "at once"): the partial of C_i = [Q_i A_i]^T A_i where A_i is the block of
// this pass: W_i for pass 1; for pass t >= 2 the previous iterate
// Y = (A_prev - Q_i P_last) N_last^{-1} (Alg. 8, U_1), which is also written
// into the new local panel so that the next stage reads it instead of
// recomputing it.  TileT/Acc = float for the first pass of the mixed form.
template <typename TileT, typename Acc>
__device__ void gram_slab(const StepArgs& a, int pass, int tile_rows, int slab, unsigned char* smem_raw) {
  const SlabInfo si = a.slabs[slab];
  const int s = a.s, k = a.nb * s, Kt = k + s, E = Kt * s;
  TileT* A = reinterpret_cast<TileT*>(smem_raw);  // tile_rows x Kt
  const size_t tm_off = (sizeof(TileT) * (size_t)tile_rows * Kt + 15) & ~(size_t)15;
  double* Tm = reinterpret_cast<double*>(smem_raw + tm_off);  // tile_rows x s
  const int tid = threadIdx.x;
  // thread -> (output entry, row group)
  const int G = (E >= kThreads) ? 1 : kThreads / E;
  const int J = (E + kThreads - 1) / kThreads;  // entries per thread when G == 1
  const int g = (G == 1) ? 0 : tid / E;
  const bool active = (G == 1) || (tid < G * E);
  Acc acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = Acc(0);

  const double* smallc = chunk_small(a, si.chunk);
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  const double* Plast = smallc + SL.P_last;
  const double* Ninv = smallc + SL.Ninv_last;
  double* slot = a.V + (int64_t)a.nb * a.n * s;
  // float32 first pass: the block's columns scaled per slab (see f32_trunc_shift)
  constexpr bool kF32 = sizeof(TileT) == 4;
  __shared__ int hs[32];
  if (kF32) slab_col_exponents(hs, s, si.rows, [&](int r, int l) { return a.W[(si.row0 + r) * a.ldw + l]; });
  auto out_scale = [&](int e) { return kF32 ? -col_shift(hs[e % s]) - (e / s >= k ? col_shift(hs[e / s - k]) : 0) : 0; };

  for (int r0 = 0; r0 < si.rows; r0 += tile_rows) {
    const int rows = min(tile_rows, si.rows - r0);
    const int64_t grow0 = si.row0 + r0;
    // Q_i rows: each panel's rows are contiguous (rows * s doubles)
    for (int idx = tid; idx < rows * k; idx += kThreads) {
      const int b = idx / (rows * s), rem = idx - b * rows * s, r = rem / s, j = rem - r * s;
      A[r * Kt + b * s + j] = (TileT)a.V[(int64_t)b * a.n * s + (grow0 + r) * s + j];
    }
    if (pass == 1) {
      for (int idx = tid; idx < rows * s; idx += kThreads) {
        const int r = idx / s, l = idx - r * s;
        double w;
        if (a.op_nx) {  // the operator's block, formed here and kept in U for the later passes
          w = op_value(a, grow0 + r, l);
          a.U[(grow0 + r) * a.ldu + l] = w;
        } else {
          w = a.W[(grow0 + r) * a.ldw + l];
        }
        A[r * Kt + k + l] = kF32 ? (TileT)f32_trunc_shift(w, col_shift(hs[l])) : (TileT)w;
      }
    } else {
      __syncthreads();
      const double* src = (pass == 2) ? a.W : slot;
      const int64_t lds = (pass == 2) ? a.ldw : s;
      for (int idx = tid; idx < rows * s; idx += kThreads) {
        const int r = idx / s, l = idx - r * s;
        double t = src[(grow0 + r) * lds + l];
        for (int q = 0; q < k; ++q) t -= (double)A[r * Kt + q] * Plast[q * s + l];
        Tm[r * s + l] = t;
      }
      __syncthreads();
      for (int idx = tid; idx < rows * s; idx += kThreads) {
        const int r = idx / s, l = idx - r * s;
        double y = 0.0;
        for (int j = 0; j <= l; ++j) y += Tm[r * s + j] * Ninv[j * s + l];
        A[r * Kt + k + l] = (TileT)y;
        slot[(grow0 + r) * s + l] = y;
      }
    }
    __syncthreads();
    if (active) {
      for (int r = g; r < rows; r += G) {
        const TileT* Ar = A + r * Kt;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j < J) {
            const int e = (G == 1) ? tid + j * kThreads : tid - g * E;
            if (e < E) {
              const int q = e / s, l = e - q * s;
              acc[j] += (Acc)Ar[q] * (Acc)Ar[k + l];
            }
          }
        }
      }
    }
    __syncthreads();
  }
  double* out = a.part + (int64_t)slab * a.Kmax * s;
  if (G == 1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int e = tid + j * kThreads;
      if (j < J && e < E) out[e] = kF32 ? scale2((double)acc[j], out_scale(e)) : (double)acc[j];
    }
  } else {
    // fixed-order sum over the G row groups
    double* red = reinterpret_cast<double*>(smem_raw);
    if (active) red[tid] = (double)acc[0];
    __syncthreads();
    if (tid < E) {
      double v = 0.0;
      for (int gg = 0; gg < G; ++gg) v += red[gg * E + tid];
      out[tid] = kF32 ? scale2(v, out_scale(tid)) : v;
    }
  }
}

template <typename TileT, typename Acc>
__global__ void __launch_bounds__(kThreads) k_gram(StepArgs a, int pass, int tile_rows) {
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gram_slab<TileT, Acc>(a, pass, tile_rows, blockIdx.x, smem_raw);
}

// Stage 1, first Gram pass, for block widths S in {1, 2, 4, 8, 16, 32}: the
// partial of C_i = [Q_i W_i]^T W_i over one slab.  Each thread keeps a
// TQ x S register tile of C (TQ = 32 / S columns of [Q_i W_i]); T threads
// cover the k + S columns and G = 256 / T row groups split the slab's rows;
// the groups are summed in a fixed order at the end.
template <int S, typename Acc>
__device__ void gram1_slab(const StepArgs& a, int slab, double* red) {
  constexpr int TQ = (32 / S) > 0 ? 32 / S : 1;
  const SlabInfo si = a.slabs[slab];
  const int k = a.nb * S, Kt = k + S;
  const int T = (Kt + TQ - 1) / TQ;
  const int G = kThreads / T;
  const int tid = threadIdx.x, g = tid / T, t = tid - g * T;
  const bool active = g < G;
  const int q0 = t * TQ;
  constexpr bool kF32 = sizeof(Acc) == 4;
  __shared__ int hs[32];
  if (a.srcexp_slab || kF32) {
    // the block's column exponents on this slab: for a tensor-core assembly
    // that follows, and for the scaling of the float32 pass
    slab_col_exponents(hs, S, si.rows, [&](int r, int l) { return a.W[(si.row0 + r) * a.ldw + l]; });
    if (a.srcexp_slab && tid < S) a.srcexp_slab[(int64_t)slab * 32 + tid] = hs[tid];
  }
  int sh[S];
#pragma unroll
  for (int l = 0; l < S; ++l) sh[l] = kF32 ? col_shift(hs[l]) : 0;
  Acc acc[TQ][S];
#pragma unroll
  for (int i = 0; i < TQ; ++i)
#pragma unroll
    for (int l = 0; l < S; ++l) acc[i][l] = Acc(0);
  if (active) {
    for (int r = g; r < si.rows; r += G) {
      const int64_t row = si.row0 + r;
      const double* wr = a.W + row * a.ldw;
      Acc b[S];
      if (a.op_nx) {  // the operator's block (float64 form), kept in U by one thread per row
#pragma unroll
        for (int l = 0; l < S; ++l) b[l] = (Acc)op_value(a, row, l);
        if (t == 0)
#pragma unroll
          for (int l = 0; l < S; ++l) a.U[row * a.ldu + l] = (double)b[l];
      } else {
#pragma unroll
        for (int l = 0; l < S; ++l) b[l] = load_scaled<Acc>(wr + l, sh[l]);
      }
      Acc av[TQ];
#pragma unroll
      for (int i = 0; i < TQ; ++i) {
        const int q = q0 + i;
        if (q < k)
          av[i] = load_as<Acc>(a.V + (int64_t)(q / S) * a.n * S + row * S + (q % S));
        else if (q < Kt)
          av[i] = a.op_nx ? (Acc)op_value(a, row, q - k) : load_scaled<Acc>(wr + (q - k), kF32 ? col_shift(hs[q - k]) : 0);
        else
          av[i] = Acc(0);
      }
#pragma unroll
      for (int i = 0; i < TQ; ++i)
#pragma unroll
        for (int l = 0; l < S; ++l) acc[i][l] += av[i] * b[l];
    }
#pragma unroll
    for (int i = 0; i < TQ; ++i)
#pragma unroll
      for (int l = 0; l < S; ++l) red[(g * T + t) * (TQ * S) + i * S + l] = (double)acc[i][l];
  }
  __syncthreads();
  double* out = a.part + (int64_t)slab * a.Kmax * S;
  for (int e = tid; e < Kt * S; e += kThreads) {
    const int q = e / S, l = e - q * S, tt = q / TQ, i = q - tt * TQ;
    double v = 0.0;
    for (int gg = 0; gg < G; ++gg) v += red[(gg * T + tt) * (TQ * S) + i * S + l];
    if (kF32) v = scale2(v, -col_shift(hs[l]) - (q >= k ? col_shift(hs[q - k]) : 0));
    out[e] = v;
  }
  __syncthreads();
}

template <int S, typename Acc>
__global__ void __launch_bounds__(kThreads) k_gram1(StepArgs a) {
  extern __shared__ __align__(16) double red[];
  gram1_slab<S, Acc>(a, blockIdx.x, red);
}

// Stage-1 Gram of a step without prior blocks (k = 0) for narrow blocks
// (S <= 4), every pass: the partial A_i^T A_i of each 256-row slab, with A_i
// = W_i in pass 1 and, from pass 2 on, the iterate Y = A_prev N_last^{-1}
// (Alg. 8, U_1; no projection at k = 0) formed on the fly and written into
// the new local panel.  Four lanes share a slab, 64 rows each, with the S x S
// products in registers; the four partials are added by two shuffle levels
// in a fixed order.  Per row that is S^2 float64 multiply-adds (plus S(S+1)/2
// for the iterate) and no row-group reduction: the float64 pipe, not a
// serial sum, bounds the narrow widths.
template <int S>
__global__ void __launch_bounds__(128) k_gram_narrow(StepArgs a, int pass) {
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = gid >> 2, q = gid & 3;  // slab, quarter
  const bool valid = w < a.nslab;
  SlabInfo si{};
  if (valid) si = a.slabs[w];
  double acc[S][S];
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int l = 0; l < S; ++l) acc[i][l] = 0.0;
  const int r0 = 64 * q, r1 = valid ? min(si.rows, r0 + 64) : 0;
  if (pass == 1) {
    const double* src = a.W + (si.row0 + r0) * a.ldw;
#pragma unroll 4
    for (int r = r0; r < r1; ++r, src += a.ldw) {
      double x[S];
#pragma unroll
      for (int l = 0; l < S; ++l) x[l] = __ldg(src + l);
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int l = i; l < S; ++l) acc[i][l] = fma(x[i], x[l], acc[i][l]);
    }
  } else {
    const double* src = (pass == 2) ? a.W : a.V;
    const int64_t lds = (pass == 2) ? a.ldw : S;
    double* slot = a.V;  // nb = 0
    double ninv[S][S];
    if (valid) {
      const double* Ninv = chunk_small(a, si.chunk) + SmallLayout::make(a.Kmax, S).Ninv_last;
#pragma unroll
      for (int j = 0; j < S; ++j)
#pragma unroll
        for (int l = 0; l < S; ++l) ninv[j][l] = Ninv[j * S + l];
    }
    for (int r = r0; r < r1; ++r) {
      const int64_t row = si.row0 + r;
      double x[S], y[S];
#pragma unroll
      for (int l = 0; l < S; ++l) x[l] = src[row * lds + l];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j <= l; ++j) v = fma(x[j], ninv[j][l], v);
        y[l] = v;
      }
#pragma unroll
      for (int l = 0; l < S; ++l) slot[row * S + l] = y[l];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int l = i; l < S; ++l) acc[i][l] = fma(y[i], y[l], acc[i][l]);
    }
  }
  // the four quarters of a slab: (q0 + q1) + (q2 + q3)
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int l = i; l < S; ++l) {
      acc[i][l] += __shfl_xor_sync(0xffffffffu, acc[i][l], 1);
      acc[i][l] += __shfl_xor_sync(0xffffffffu, acc[i][l], 2);
    }
  if (valid && q == 0) {
    double* out = a.part + (int64_t)w * a.Kmax * S;
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int l = 0; l < S; ++l) out[i * S + l] = (l >= i) ? acc[i][l] : acc[l][i];
  }
}

cudaError_t launch_gram_narrow(const StepArgs& a, int pass, cudaStream_t st) {
  if (a.slab_rows > 256) return cudaErrorInvalidValue;  // four lanes x 64 rows per slab
  const int blocks = (int)(((int64_t)a.nslab * 4 + 127) / 128);
  switch (a.s) {
    case 1: k_gram_narrow<1><<<blocks, 128, 0, st>>>(a, pass); break;
    case 2: k_gram_narrow<2><<<blocks, 128, 0, st>>>(a, pass); break;
    case 3: k_gram_narrow<3><<<blocks, 128, 0, st>>>(a, pass); break;
    case 4: k_gram_narrow<4><<<blocks, 128, 0, st>>>(a, pass); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Acc>
cudaError_t launch_gram1(const StepArgs& a, cudaStream_t st) {
  const size_t sm = sizeof(double) * kThreads * 32;
  switch (a.s) {
    case 1: k_gram1<1, Acc><<<a.nslab, kThreads, sm, st>>>(a); break;
    case 2: k_gram1<2, Acc><<<a.nslab, kThreads, sm, st>>>(a); break;
    case 4: k_gram1<4, Acc><<<a.nslab, kThreads, sm, st>>>(a); break;
    case 8: k_gram1<8, Acc><<<a.nslab, kThreads, sm, st>>>(a); break;
    case 16: k_gram1<16, Acc><<<a.nslab, kThreads, sm, st>>>(a); break;
    case 32: k_gram1<32, Acc><<<a.nslab, kThreads, sm, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

bool gram1_supported(int s) { return s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32; }

// ---------------------------------------------------------------------------
// Leaf factorization of pass `pass`, one CTA per chunk: sum the slab partials
// in slab order, then N = chol(G - P^T P) (Alg. 7), N^{-1}, and the
// reiteration bookkeeping of Alg. 8: P_comb <- P_comb + P N_comb,
// N_comb <- N N_comb.  Decides on the next pass from kappa_F(N).  u_gram is
// the unit roundoff of this pass's Gram (float64: DBL_EPSILON; the mixed
// form's digit Gram: 2^-31): the breakdown test and the shift of the retry
// scale with it.
__device__ void leaf_chunk(const StepArgs& a, int pass, double shift_rel, int allow_shift, double u_gram, int c,
                           double* sm) {
  const int s = a.s, k = a.nb * s, Kt = k + s, E = Kt * s, ss = s * s;
  double* C = sm;             // Kt x s
  double* M = C + E;          // s x s
  double* Ni = M + ss;        // s x s
  double* Nc = Ni + ss;       // s x s (old N_comb)
  double* tmp = Nc + ss;      // s x s
  double* red = tmp + ss;     // 4
  const int sl0 = a.chunk_slab0[c], sl1 = a.chunk_slab0[c + 1];
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double v = 0.0;
    for (int sl = sl0; sl < sl1; ++sl) v += a.part[(int64_t)sl * a.Kmax * s + e];
    C[e] = v;
  }
  if (a.srcexp) {  // tensor-core form: the pass block's column exponents per chunk
    for (int l = threadIdx.x; l < s; l += blockDim.x) {
      int m = 0;
      for (int sl = sl0; sl < sl1; ++sl) m = max(m, a.srcexp_slab[(int64_t)sl * 32 + l]);
      a.srcexp[(int64_t)c * 32 + l] = m;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    const int i = e / s, j = e - i * s;
    double m = C[(k + i) * s + j];
    for (int q = 0; q < k; ++q) m -= C[q * s + i] * C[q * s + j];
    M[e] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < s; ++i) tr += C[(k + i) * s + i];
    red[1] = tr;
  }
  __syncthreads();
  const double trG = red[1];
  if (shift_rel > 0.0) {  // shifted Cholesky (first pass of the mixed form)
    for (int i = threadIdx.x; i < s; i += blockDim.x) M[i * s + i] += shift_rel * trG;
    __syncthreads();
  }
  const double tol = (double)s * u_gram * trG;
  const int64_t rows = a.chunk_row0[c + 1] - a.chunk_row0[c];
  const double sigma = 11.0 * ((double)rows * s + (double)s * (s + 1)) * u_gram * trG;
  // deflation (first pass only; later passes see the dropped columns as exact
  // zeros): pivots against the whole block's squared norm, floored at the
  // Gram's rounding level
  double defl = 0.0;
  if (a.deflation_tol > 0.0 && pass == 1) {
    const GlobLayout GLd = GlobLayout::make(a.Kmax, s);
    defl = fmax(a.deflation_tol * a.deflation_tol, 64.0 * s * DBL_EPSILON) * a.glob[GLd.scal + 1];
  }
  const bool shifted = cta_cholesky_shifted(M, tmp, s, tol, sigma, allow_shift != 0 && a.deflation_tol <= 0.0,
                                            a.flags, reinterpret_cast<int*>(red + 2), defl);
  if (shifted && threadIdx.x == 0)
    for (int t = pass + 1; t <= pass + 2 && t <= kMaxPass; ++t) atomicOr(&a.flags[kFlagPass + t - 1], 1);
  cta_upper_inverse(M, Ni, s);
  const double kap = cta_pip_kappa(trG, Ni, s, red);

  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  double* Plast = smallc + SL.P_last;
  double* Pcomb = smallc + SL.P_comb;
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) Plast[e] = C[e];
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    smallc[SL.N_last + e] = M[e];
    smallc[SL.Ninv_last + e] = Ni[e];
    Nc[e] = (pass == 1) ? 0.0 : smallc[SL.N_comb + e];
  }
  __syncthreads();
  if (pass == 1) {
    for (int e = threadIdx.x; e < k * s; e += blockDim.x) Pcomb[e] = C[e];
    for (int e = threadIdx.x; e < ss; e += blockDim.x) smallc[SL.N_comb + e] = M[e];
  } else {
    // P_comb += P Nc_old ; N_comb = N Nc_old
    for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
      const int q = e / s, l = e - q * s;
      double v = Pcomb[e];
      for (int j = 0; j <= l; ++j) v += C[q * s + j] * Nc[j * s + l];
      Pcomb[e] = v;
    }
    cta_matmul_ss(M, Nc, tmp, s);
    for (int e = threadIdx.x; e < ss; e += blockDim.x) smallc[SL.N_comb + e] = tmp[e];
  }
  if (threadIdx.x == 0 && pass < kMaxPass) {
    const bool auto_mode = (a.leaf != LO_LEAF_PIP) || (a.precision == LO_PREC_MIXED_FP32) ||
                           (a.precision == LO_PREC_MIXED_TC);
    if (auto_mode && !(DBL_EPSILON * kap * kap <= a.refine_tol))
      atomicOr(&a.flags[kFlagPass + pass], 1);
  }
}

__global__ void __launch_bounds__(kThreads) k_leaf(StepArgs a, int pass, double shift_rel, int allow_shift,
                                                   double u_gram) {
  if (pass >= 2 && !a.flags[kFlagPass + pass - 1]) return;
  extern __shared__ __align__(16) double sm[];
  leaf_chunk(a, pass, shift_rel, allow_shift, u_gram, blockIdx.x, sm);
}

// ||W||_F^2 of the step from the pass-1 Gram partials (the diagonal of each
// slab's W^T W block, slabs in order), for the deflation thresholds of the
// local leaves.  One CTA.
__global__ void __launch_bounds__(kThreads) k_defl_trace(StepArgs a) {
  __shared__ double red[kThreads];
  const int s = a.s, k = a.nb * s;
  double v = 0.0;
  for (int e = threadIdx.x; e < a.nslab * s; e += kThreads) {
    const int sl = e / s, i = e - sl * s;
    v += a.part[(int64_t)sl * a.Kmax * s + (int64_t)(k + i) * s + i];
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.glob[GlobLayout::make(a.Kmax, s).scal + 1] = red[0];
}

// ---------------------------------------------------------------------------
// Reduction step (Sec. 4.1), solved with BCGS-PIP on the stacked factors
// [[T_i, X_i], [0, Nx_i]], reiterated as in Alg. 8 when needed.
// Iteration `it` input: (P_comb, N_comb) for it = 1, else (P_hat, N_hat).

// z_i = [T_i^T X_i ; X_i^T X_i + Nx_i^T Nx_i]  ((k + s) x s)
__device__ void tree_contrib_chunk(const StepArgs& a, int it, int c, double* sm) {
  const int s = a.s, k = a.nb * s, ss = s * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  const double* Xg = smallc + (it == 1 ? SL.P_comb : SL.P_hat);
  const double* Nxg = smallc + (it == 1 ? SL.N_comb : SL.N_hat);
  double* X = sm;            // k x s
  double* Nx = X + k * s;    // s x s
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) X[e] = Xg[e];
  for (int e = threadIdx.x; e < ss; e += blockDim.x) Nx[e] = Nxg[e];
  __syncthreads();
  const double* Tc = a.T + (int64_t)c * a.tstride;
  double* Z = smallc + SL.Z;
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
    const int q = e / s, l = e - q * s, cb = q / s, qq = q - cb * s;
    const double* Tb = Tc + tblock_offset(cb, s);   // ((cb+1) s) x s
    double v = 0.0;
    for (int r = 0; r < (cb + 1) * s; ++r) v += Tb[r * s + qq] * X[r * s + l];
    Z[e] = v;
  }
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    const int i = e / s, j = e - i * s;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += X[r * s + i] * X[r * s + j];
    for (int r = 0; r < s; ++r) v += Nx[r * s + i] * Nx[r * s + j];
    Z[k * s + e] = v;
  }
}

__global__ void __launch_bounds__(kThreads) k_tree_contrib(StepArgs a, int it) {
  if (!a.flags[kFlagTree + it - 1]) return;
  extern __shared__ __align__(16) double sm[];
  tree_contrib_chunk(a, it, blockIdx.x, sm);
}

// First level of the fixed-order sum over chunks: group g sums chunks
// [g * kTreeGroup, (g + 1) * kTreeGroup) in index order.
__global__ void __launch_bounds__(kThreads) k_tree_sum1(StepArgs a, int it) {
  if (!a.flags[kFlagTree + it - 1]) return;
  const int s = a.s, E = (a.nb * s + s) * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  // blockIdx.y splits the entries so that many CTAs share the work
  const int c0 = blockIdx.x * kTreeGroup, c1 = min(a.p, c0 + kTreeGroup);
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < E; e += gridDim.y * blockDim.x) {
    double v = 0.0;
    for (int c = c0; c < c1; ++c) v += a.small[(int64_t)c * SL.stride + SL.Z + e];
    a.tsum[(int64_t)blockIdx.x * a.Kmax * s + e] = v;
  }
}

// Second level + the small factorization of the reduction PQR:
// P = sum T_i^T X_i, G = sum (X_i^T X_i + Nx_i^T Nx_i), N = chol(G - P^T P);
// accumulates P_acc <- P_acc + P N_acc, N_acc <- N N_acc (Alg. 8 combine).
// The small factorization of iteration `it` once Z (the summed contributions,
// global Zsum) is complete.  Whole CTA.
__device__ void tree_sum2_core(const StepArgs& a, int it, double* sm) {
  const int s = a.s, k = a.nb * s, ss = s * s;
  const GlobLayout GL = GlobLayout::make(a.Kmax, s);
  double* Z = a.glob + GL.Zsum;
  double* M = sm;
  double* Ni = M + ss;
  double* Na = Ni + ss;
  double* tmp = Na + ss;
  double* red = tmp + ss;
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    const int i = e / s, j = e - i * s;
    double m = Z[(k + i) * s + j];
    for (int q = 0; q < k; ++q) m -= Z[q * s + i] * Z[q * s + j];
    M[e] = m;
  }
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < s; ++i) tr += Z[(k + i) * s + i];
    red[1] = tr;
  }
  __syncthreads();
  const double trG = red[1];
  const double sigma = 11.0 * ((double)a.p * (k + s) * s + (double)s * (s + 1)) * DBL_EPSILON * trG;
  const bool deflate = a.deflation_tol > 0.0;
  const double defl =
      (deflate && it == 1) ? fmax(a.deflation_tol * a.deflation_tol, 64.0 * s * DBL_EPSILON) * trG : 0.0;
  const bool shifted = cta_cholesky_shifted(M, tmp, s, (double)s * DBL_EPSILON * trG, sigma,
                                            it == 1 && a.reduction != 1 && !deflate, a.flags,
                                            reinterpret_cast<int*>(red + 2), defl);
  if (shifted && threadIdx.x == 0)
    for (int t = it + 1; t <= it + 2 && t <= kMaxTreeIter; ++t) atomicOr(&a.flags[kFlagTree + t - 1], 1);
  if (it == 1 && threadIdx.x == 0) a.glob[GL.scal] = trG;  // |W|_F^2 of the step
  cta_upper_inverse(M, Ni, s);
  const double kap = cta_pip_kappa(trG, Ni, s, red);
  double* P_it = a.glob + GL.P_it;
  double* P_acc = a.glob + GL.P_acc;
  double* N_acc = a.glob + GL.N_acc;
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) P_it[e] = Z[e];
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    a.glob[GL.N_it + e] = M[e];
    a.glob[GL.Ninv_it + e] = Ni[e];
    Na[e] = (it == 1) ? 0.0 : N_acc[e];
  }
  __syncthreads();
  if (it == 1) {
    for (int e = threadIdx.x; e < k * s; e += blockDim.x) P_acc[e] = Z[e];
    for (int e = threadIdx.x; e < ss; e += blockDim.x) N_acc[e] = M[e];
  } else {
    for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
      const int q = e / s, l = e - q * s;
      double v = P_acc[e];
      for (int j = 0; j <= l; ++j) v += Z[q * s + j] * Na[j * s + l];
      P_acc[e] = v;
    }
    cta_matmul_ss(M, Na, tmp, s);
    for (int e = threadIdx.x; e < ss; e += blockDim.x) N_acc[e] = tmp[e];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // numerical rank: a normalizer diagonal at the rounding level of the block
    // (the deflation case of Sec. 3, not supported) is a breakdown
    const double floor_ = 64.0 * s * DBL_EPSILON * sqrt(a.glob[GL.scal]);
    for (int i = 0; i < s; ++i)
      if (!(fabs(N_acc[i * s + i]) > floor_) && !(deflate && N_acc[i * s + i] == 0.0))
        set_status(a.flags, LO_ERR_BREAKDOWN);
  }
  if (threadIdx.x == 0 && it < kMaxTreeIter) {
    if (a.reduction == 0 && !(DBL_EPSILON * kap * kap <= a.refine_tol))
      atomicOr(&a.flags[kFlagTree + it], 1);
  }
}

__global__ void __launch_bounds__(kThreads) k_tree_sum2(StepArgs a, int it, int ngroups) {
  if (!a.flags[kFlagTree + it - 1]) return;
  extern __shared__ __align__(16) double sm[];
  const int s = a.s, k = a.nb * s, E = (k + s) * s;
  double* Z = a.glob + GlobLayout::make(a.Kmax, s).Zsum;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double v = 0.0;
    for (int g = 0; g < ngroups; ++g) v += a.tsum[(int64_t)g * a.Kmax * s + e];
    Z[e] = v;
  }
  __syncthreads();
  tree_sum2_core(a, it, sm);
}

// Per chunk: X_hat = (X - T_i P) N^{-1}, Nx_hat = Nx N^{-1}; the result is
// also written as column block nb of T_i: [Pt_i; Nt_i] (Alg. 9 output).
__device__ void tree_update_chunk(const StepArgs& a, int it, int c, double* sm) {
  const int s = a.s, k = a.nb * s, ss = s * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  const GlobLayout GL = GlobLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  const double* Xg = smallc + (it == 1 ? SL.P_comb : SL.P_hat);
  const double* Nxg = smallc + (it == 1 ? SL.N_comb : SL.N_hat);
  const double* Pg = a.glob + GL.P_it;
  const double* Ninv = a.glob + GL.Ninv_it;
  const double* Tc = a.T + (int64_t)c * a.tstride;
  double* t = sm;           // k x s
  double* Nx = t + k * s;   // s x s
  double* Nin = Nx + ss;    // s x s
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    Nx[e] = Nxg[e];
    Nin[e] = Ninv[e];
  }
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
    const int r = e / s, l = e - r * s;
    double v = Xg[e];
    for (int cb = r / s; cb < a.nb; ++cb) {
      const double* Tb = Tc + tblock_offset(cb, s);
      for (int qq = 0; qq < s; ++qq) v -= Tb[r * s + qq] * Pg[(cb * s + qq) * s + l];
    }
    t[e] = v;
  }
  __syncthreads();
  double* Ph = smallc + SL.P_hat;
  double* Tnew = a.T + (int64_t)c * a.tstride + tblock_offset(a.nb, s);  // (k + s) x s
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
    const int r = e / s, l = e - r * s;
    double v = 0.0;
    for (int j = 0; j <= l; ++j) v += t[r * s + j] * Nin[j * s + l];
    Ph[e] = v;
    Tnew[e] = v;
  }
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    const int i = e / s, l = e - i * s;
    double v = 0.0;
    if (i <= l)
      for (int j = i; j <= l; ++j) v += Nx[i * s + j] * Nin[j * s + l];
    smallc[SL.N_hat + e] = v;
    Tnew[k * s + e] = v;
  }
}

// The same two products with T_i read through shared memory, kTreeRows rows
// at a time across all its column blocks: every thread's sums read T_i from
// global memory one dependent term after another, which left both latency-
// bound (80 us per round at k = 120).  Each output keeps the order of its
// terms, so the results are those of the functions above, bit for bit.
constexpr int kTreeRows = 32;

// Bytes of shared memory of the staged reduction kernels (0: does not fit).
size_t tree_staged_smem(int k, int s) {
  const int nb = k / s;
  const size_t b = 8 * (3 * (size_t)k * s + 2 * (size_t)s * s + (size_t)nb * kTreeRows * s);
  return b <= 200 * 1024 ? b : 0;
}

// Rows r0 .. r1 - 1 of every column block cb of T_i that has them (block cb
// holds rows 0 .. (cb + 1) s - 1) into Tst[(cb kTreeRows + r - r0) s + qq].
__device__ __forceinline__ void tree_stage_rows(const double* Tc, int nb, int s, int r0, int r1, double* Tst) {
  const int cb0 = r0 / s, per = kTreeRows * s;
  for (int e = threadIdx.x; e < (nb - cb0) * per; e += blockDim.x) {
    const int cb = cb0 + e / per, w = e - (cb - cb0) * per, rr = w / s, qq = w - rr * s, r = r0 + rr;
    if (r < r1 && r < (cb + 1) * s) Tst[(cb * kTreeRows + rr) * s + qq] = Tc[tblock_offset(cb, s) + (int64_t)r * s + qq];
  }
}

// tree_update_chunk with T_i and P staged; smem: t, P (k x s), Nx, Nin (s x s), the row window.
__device__ void tree_update_chunk_st(const StepArgs& a, int it, int c, double* sm) {
  const int s = a.s, nb = a.nb, k = nb * s, ss = s * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  const GlobLayout GL = GlobLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  const double* Xg = smallc + (it == 1 ? SL.P_comb : SL.P_hat);
  const double* Nxg = smallc + (it == 1 ? SL.N_comb : SL.N_hat);
  const double* Pg = a.glob + GL.P_it;
  const double* Ninv = a.glob + GL.Ninv_it;
  const double* Tc = a.T + (int64_t)c * a.tstride;
  double* t = sm;            // k x s
  double* P = t + k * s;     // k x s
  double* Nx = P + k * s;    // s x s
  double* Nin = Nx + ss;     // s x s
  double* Tst = Nin + ss;    // nb x kTreeRows x s
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    Nx[e] = Nxg[e];
    Nin[e] = Ninv[e];
  }
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) P[e] = Pg[e];
  for (int r0 = 0; r0 < k; r0 += kTreeRows) {
    const int r1 = min(k, r0 + kTreeRows);
    __syncthreads();
    tree_stage_rows(Tc, nb, s, r0, r1, Tst);
    __syncthreads();
    for (int e = r0 * s + threadIdx.x; e < r1 * s; e += blockDim.x) {
      const int r = e / s, l = e - r * s;
      double v = Xg[e];
      for (int cb = r / s; cb < nb; ++cb) {
        const double* Tb = Tst + (cb * kTreeRows + (r - r0)) * s;
        for (int qq = 0; qq < s; ++qq) v -= Tb[qq] * P[(cb * s + qq) * s + l];
      }
      t[e] = v;
    }
  }
  __syncthreads();
  double* Ph = smallc + SL.P_hat;
  double* Tnew = a.T + (int64_t)c * a.tstride + tblock_offset(nb, s);  // (k + s) x s
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
    const int r = e / s, l = e - r * s;
    double v = 0.0;
    for (int j = 0; j <= l; ++j) v += t[r * s + j] * Nin[j * s + l];
    Ph[e] = v;
    Tnew[e] = v;
  }
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    const int i = e / s, l = e - i * s;
    double v = 0.0;
    if (i <= l)
      for (int j = i; j <= l; ++j) v += Nx[i * s + j] * Nin[j * s + l];
    smallc[SL.N_hat + e] = v;
    Tnew[k * s + e] = v;
  }
}

// tree_contrib_chunk with T_i staged; smem: X, the partial sums (k x s), Nx (s x s), the row window.
__device__ void tree_contrib_chunk_st(const StepArgs& a, int it, int c, double* sm) {
  const int s = a.s, nb = a.nb, k = nb * s, ss = s * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  const double* Xg = smallc + (it == 1 ? SL.P_comb : SL.P_hat);
  const double* Nxg = smallc + (it == 1 ? SL.N_comb : SL.N_hat);
  const double* Tc = a.T + (int64_t)c * a.tstride;
  double* X = sm;             // k x s
  double* Zp = X + k * s;     // k x s
  double* Nx = Zp + k * s;    // s x s
  double* Tst = Nx + 2 * ss;  // nb x kTreeRows x s (after the update's layout size)
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
    X[e] = Xg[e];
    Zp[e] = 0.0;
  }
  for (int e = threadIdx.x; e < ss; e += blockDim.x) Nx[e] = Nxg[e];
  for (int r0 = 0; r0 < k; r0 += kTreeRows) {
    const int r1 = min(k, r0 + kTreeRows);
    __syncthreads();
    tree_stage_rows(Tc, nb, s, r0, r1, Tst);
    __syncthreads();
    for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
      const int q = e / s, l = e - q * s, cb = q / s, qq = q - cb * s;
      const int rend = min(r1, (cb + 1) * s);
      if (r0 >= rend) continue;
      double v = Zp[e];
      for (int r = r0; r < rend; ++r) v += Tst[(cb * kTreeRows + (r - r0)) * s + qq] * X[r * s + l];
      Zp[e] = v;
    }
  }
  __syncthreads();
  double* Z = smallc + SL.Z;
  for (int e = threadIdx.x; e < k * s; e += blockDim.x) Z[e] = Zp[e];
  for (int e = threadIdx.x; e < ss; e += blockDim.x) {
    const int i = e / s, j = e - i * s;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += X[r * s + i] * X[r * s + j];
    for (int r = 0; r < s; ++r) v += Nx[r * s + i] * Nx[r * s + j];
    Z[k * s + e] = v;
  }
}

__global__ void __launch_bounds__(kThreads) k_tree_update(StepArgs a, int it) {
  if (!a.flags[kFlagTree + it - 1]) return;
  extern __shared__ __align__(16) double sm[];
  tree_update_chunk(a, it, blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// Stage 2 (assembly, Sec. 4.1): per row of chunk i,
//   u = (A_last - q P_last) N_last^{-1}   -> new local panel (U_i)
//   out = q Pt_i + u Nt_i                 -> caller's U
// where A_last is W (one pass) or the stored previous iterate.
__device__ void update_slab(const StepArgs& a, int tile_rows, int slab, double* sm) {
  const SlabInfo si = a.slabs[slab];
  const int s = a.s, k = a.nb * s;
  const int L = passes_run(a);
  double* slot = a.V + (int64_t)a.nb * a.n * s;
  const double* src = (L == 1) ? a.W : slot;
  const int64_t lds = (L == 1) ? a.ldw : s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  const double* smallc = a.small + (int64_t)si.chunk * SL.stride;
  const double* Plast = smallc + SL.P_last;
  const double* Ninv = smallc + SL.Ninv_last;
  const double* Tb = a.T + (int64_t)si.chunk * a.tstride + tblock_offset(a.nb, s);
  const double* Pt = Tb;            // k x s
  const double* Nt = Tb + k * s;    // s x s
  double* Aq = sm;                          // tile_rows x k
  double* Tm = Aq + tile_rows * k;          // tile_rows x s
  double* Us = Tm + tile_rows * s;          // tile_rows x s
  const int tid = threadIdx.x;
  for (int r0 = 0; r0 < si.rows; r0 += tile_rows) {
    const int rows = min(tile_rows, si.rows - r0);
    const int64_t grow0 = si.row0 + r0;
    for (int idx = tid; idx < rows * k; idx += kThreads) {
      const int b = idx / (rows * s), rem = idx - b * rows * s, r = rem / s, j = rem - r * s;
      Aq[r * k + b * s + j] = a.V[(int64_t)b * a.n * s + (grow0 + r) * s + j];
    }
    __syncthreads();
    for (int idx = tid; idx < rows * s; idx += kThreads) {
      const int r = idx / s, l = idx - r * s;
      double t = src[(grow0 + r) * lds + l];
      for (int q = 0; q < k; ++q) t -= Aq[r * k + q] * Plast[q * s + l];
      Tm[idx] = t;
    }
    __syncthreads();
    for (int idx = tid; idx < rows * s; idx += kThreads) {
      const int r = idx / s, l = idx - r * s;
      double u = 0.0;
      for (int j = 0; j <= l; ++j) u += Tm[r * s + j] * Ninv[j * s + l];
      Us[idx] = u;
      slot[(grow0 + r) * s + l] = u;
    }
    __syncthreads();
    for (int idx = tid; idx < rows * s; idx += kThreads) {
      const int r = idx / s, l = idx - r * s;
      double o = 0.0;
      for (int q = 0; q < k; ++q) o += Aq[r * k + q] * Pt[q * s + l];
      for (int j = 0; j <= l; ++j) o += Us[r * s + j] * Nt[j * s + l];
      a.U[(grow0 + r) * a.ldu + l] = o;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_update(StepArgs a, int tile_rows) {
  extern __shared__ __align__(16) double sm[];
  update_slab(a, tile_rows, blockIdx.x, sm);
}

// Stage 2 of a step without prior blocks for narrow blocks (S <= 4): per row
// u = A_last N_last^{-1} (new local panel) and out = u Nt_i (caller's U),
// one thread per row (coalesced rows of S values), the two triangular S x S
// factors of the row's chunk in registers.
template <int S>
__global__ void __launch_bounds__(256) k_update_narrow(StepArgs a) {
  const SlabInfo si = a.slabs[blockIdx.x];
  const int r = threadIdx.x;
  if (r >= si.rows) return;
  const int L = passes_run(a);
  double* slot = a.V;  // nb = 0
  const double* src = (L == 1) ? a.W : slot;
  const int64_t lds = (L == 1) ? a.ldw : S;
  const SmallLayout SL = SmallLayout::make(a.Kmax, S);
  const double* smallc = a.small + (int64_t)si.chunk * SL.stride;
  const double* Ninv = smallc + SL.Ninv_last;
  const double* Nt = a.T + (int64_t)si.chunk * a.tstride + tblock_offset(0, S);
  const int64_t row = si.row0 + r;
  double x[S], u[S];
#pragma unroll
  for (int l = 0; l < S; ++l) x[l] = src[row * lds + l];
#pragma unroll
  for (int l = 0; l < S; ++l) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j <= l; ++j) v = fma(x[j], __ldg(Ninv + j * S + l), v);
    u[l] = v;
  }
#pragma unroll
  for (int l = 0; l < S; ++l) slot[row * S + l] = u[l];
#pragma unroll
  for (int l = 0; l < S; ++l) {
    double o = 0.0;
#pragma unroll
    for (int j = 0; j <= l; ++j) o = fma(u[j], __ldg(Nt + j * S + l), o);
    a.U[row * a.ldu + l] = o;
  }
}

cudaError_t launch_update_narrow(const StepArgs& a, cudaStream_t st) {
  if (a.slab_rows > 256) return cudaErrorInvalidValue;  // one thread per row of a slab
  switch (a.s) {
    case 1: k_update_narrow<1><<<a.nslab, 256, 0, st>>>(a); break;
    case 2: k_update_narrow<2><<<a.nslab, 256, 0, st>>>(a); break;
    case 3: k_update_narrow<3><<<a.nslab, 256, 0, st>>>(a); break;
    case 4: k_update_narrow<4><<<a.nslab, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// apply_Q: Z_i = T_i C (k x m) per chunk, then Y_i = Q_i Z_i.
__global__ void __launch_bounds__(kThreads) k_apply_z(StepArgs a, const double* C, int m,
                                                      int64_t ldc, double* Z) {
  const int c = blockIdx.x, s = a.s, k = a.nb * s;
  const double* Tc = a.T + (int64_t)c * a.tstride;
  double* Zc = Z + (int64_t)c * k * m;
  for (int e = threadIdx.x; e < k * m; e += blockDim.x) {
    const int r = e / m, j = e - r * m;
    double v = 0.0;
    for (int cb = r / s; cb < a.nb; ++cb) {
      const double* Tb = Tc + tblock_offset(cb, s);
      for (int qq = 0; qq < s; ++qq) v += Tb[r * s + qq] * C[(int64_t)(cb * s + qq) * ldc + j];
    }
    Zc[e] = v;
  }
}

__global__ void __launch_bounds__(kThreads) k_apply_y(StepArgs a, int m, const double* Z, double* Y,
                                                      int64_t ldy, int tile_rows) {
  extern __shared__ __align__(16) double sm[];
  const SlabInfo si = a.slabs[blockIdx.x];
  const int s = a.s, k = a.nb * s;
  const double* Zc = Z + (int64_t)si.chunk * k * m;
  double* Aq = sm;
  for (int r0 = 0; r0 < si.rows; r0 += tile_rows) {
    const int rows = min(tile_rows, si.rows - r0);
    const int64_t grow0 = si.row0 + r0;
    for (int idx = threadIdx.x; idx < rows * k; idx += kThreads) {
      const int b = idx / (rows * s), rem = idx - b * rows * s, r = rem / s, j = rem - r * s;
      Aq[r * k + b * s + j] = a.V[(int64_t)b * a.n * s + (grow0 + r) * s + j];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * m; idx += kThreads) {
      const int r = idx / m, j = idx - r * m;
      double v = 0.0;
      for (int q = 0; q < k; ++q) v += Aq[r * k + q] * Zc[q * m + j];
      Y[(grow0 + r) * ldy + j] = v;
    }
    __syncthreads();
  }
}

// 2D 5-point Laplacian with homogeneous Dirichlet boundary, s columns.
__global__ void k_laplace5(int nx, int ny, int s, const double* X, int64_t ldx, double* Y,
                           int64_t ldy) {
  const int64_t total = (int64_t)nx * ny * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pt = e / s;
    const int l = (int)(e - pt * s);
    const int ix = (int)(pt % nx), iy = (int)(pt / nx);
    double v = 4.0 * X[pt * ldx + l];
    if (ix > 0) v -= X[(pt - 1) * ldx + l];
    if (ix < nx - 1) v -= X[(pt + 1) * ldx + l];
    if (iy > 0) v -= X[(pt - nx) * ldx + l];
    if (iy < ny - 1) v -= X[(pt + nx) * ldx + l];
    Y[pt * ldy + l] = v;
  }
}

// ---------------------------------------------------------------------------
// Householder leaf of the step without prior blocks (Alg. 6 with an empty
// basis, k = 0).  One CTA per chunk holds the chunk tile W_i (rows x s,
// column-major in shared memory), reduces it to R_i by s reflections
// H_j = I - tau_j v_j v_j^T (v_j[j] = 1, supported on rows j ..), with the
// sign rule of Alg. 6: R_jj = sigma ||x||, sigma = -sgn(x_j), sgn(0) = +1, so
// that x_j - R_jj never cancels.  It then forms the explicit
// Q_i = H_0 ... H_{s-1} [I; 0] in place (the reflectors applied backwards to
// the unit vectors) and normalizes the signs so that diag(R_i) >= 0.
// Outputs: Q_i into the new local panel, R_i as the chunk's normalizer
// (N_last = N_comb), N_last^{-1} recorded as the identity (the panel already
// is the chunk's orthonormal factor), and for the tensor-core forms the
// panel's column exponents.  A column that vanishes on and below the diagonal
// gets no reflection (tau = 0): R_jj = 0 and Q_i keeps the unit direction e_j.

// Sum over the CTA of v[0 .. cnt) of every thread, in a fixed order (lanes by
// a butterfly, then warps in index order), into out[0 .. cnt).
template <int SMAX>
__device__ __forceinline__ void hh_block_sum(double (&v)[SMAX], int cnt, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < SMAX; ++c) {
    if (c < cnt) {
      double x = v[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[c] = x;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < SMAX; ++c)
      if (c < cnt) red[warp * 32 + c] = v[c];
  }
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    double x = 0.0;
    for (int w = 0; w < kHHThreads / 32; ++w) x += red[w * 32 + threadIdx.x];
    out[threadIdx.x] = x;
  }
  __syncthreads();
}

// Apply H_j = I - t v v^T (v = column j of A below the diagonal, v_j = 1) to
// columns j + 1 .. s - 1 of A (rows j ..): w_c = A[j][c] + sum_{r > j} v_r A[r][c],
// A[., c] -= t v w_c.  Whole CTA; returns after a barrier.
template <int SMAX>
__device__ __forceinline__ void hh_apply_lda(double* A, int lda, int rows, int s, int j, double t, double* red,
                                             double* vsum, double* wsh) {
  const int nc = s - j - 1, tid = threadIdx.x;
  if (nc <= 0 || t == 0.0) return;
  const double* x = A + (int64_t)j * lda;
  double w[SMAX];
#pragma unroll
  for (int cc = 0; cc < SMAX; ++cc) w[cc] = 0.0;
  for (int r = j + 1 + tid; r < rows; r += kHHThreads) {
    const double vr = x[r];
#pragma unroll
    for (int cc = 0; cc < SMAX; ++cc)
      if (cc < nc) w[cc] = fma(vr, A[(int64_t)(j + 1 + cc) * lda + r], w[cc]);
  }
  hh_block_sum<SMAX>(w, nc, red, vsum);
  if (tid < nc) wsh[tid] = A[(int64_t)(j + 1 + tid) * lda + j] + vsum[tid];
  __syncthreads();
  if (tid < nc) A[(int64_t)(j + 1 + tid) * lda + j] -= t * wsh[tid];
  for (int r = j + 1 + tid; r < rows; r += kHHThreads) {
    const double tv = t * x[r];
#pragma unroll
    for (int cc = 0; cc < SMAX; ++cc)
      if (cc < nc) A[(int64_t)(j + 1 + cc) * lda + r] -= tv * wsh[cc];
  }
  __syncthreads();
}

template <int SMAX>
__device__ __forceinline__ void hh_apply(double* A, int rows, int s, int j, double t, double* red, double* vsum,
                                         double* wsh) {
  hh_apply_lda<SMAX>(A, rows, rows, s, j, t, red, vsum, wsh);
}

template <int SMAX>
__global__ void __launch_bounds__(kHHThreads) k_hh_leaf(StepArgs a) {
  extern __shared__ __align__(16) double A[];  // rows x s, column-major
  __shared__ double red[(kHHThreads / 32) * 32];
  __shared__ double vsum[32], wsh[32], tau[32], dsg[32];
  __shared__ double Rs[32 * 32];
  __shared__ int hs[32];
  __shared__ int bad;
  const int c = blockIdx.x, s = a.s, tid = threadIdx.x;
  const int64_t r0 = a.chunk_row0[c];
  const int rows = (int)(a.chunk_row0[c + 1] - r0);
  if (tid == 0) bad = 0;
  if (tid < 32) hs[tid] = 0;
  __syncthreads();
  for (int idx = tid; idx < rows * s; idx += kHHThreads) {
    const int r = idx / s, l = idx - r * s;
    const double x = a.W[(r0 + r) * a.ldw + l];
    if (!isfinite(x)) bad = 1;
    A[(int64_t)l * rows + r] = x;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) set_status(a.flags, LO_ERR_NONFINITE);
    return;
  }
  // R_i: one reflection per column
  for (int j = 0; j < s; ++j) {
    double* x = A + (int64_t)j * rows;
    double v[SMAX];
#pragma unroll
    for (int cc = 0; cc < SMAX; ++cc) v[cc] = 0.0;
    for (int r = j + tid; r < rows; r += kHHThreads) v[0] = fma(x[r], x[r], v[0]);
    hh_block_sum<SMAX>(v, 1, red, vsum);
    const double alpha = sqrt(vsum[0]);
    const double x0 = x[j];
    const double beta = (x0 >= 0.0) ? -alpha : alpha;
    const double t = (alpha == 0.0) ? 0.0 : (beta - x0) / beta;
    if (!isfinite(alpha)) {
      if (tid == 0) set_status(a.flags, LO_ERR_NONFINITE);
      return;
    }
    __syncthreads();  // every thread has read x_j
    if (alpha != 0.0) {
      const double scal = 1.0 / (x0 - beta);
      for (int r = j + 1 + tid; r < rows; r += kHHThreads) x[r] *= scal;
    }
    if (tid == 0) {
      x[j] = beta;
      tau[j] = t;
    }
    __syncthreads();
    hh_apply<SMAX>(A, rows, s, j, t, red, vsum, wsh);
  }
  for (int e = tid; e < s * s; e += kHHThreads) {
    const int i = e / s, l = e - i * s;
    Rs[e] = (i <= l) ? A[(int64_t)l * rows + i] : 0.0;
  }
  __syncthreads();
  // Q_i = H_0 .. H_{s-1} [I; 0], formed in place from the last reflection back
  for (int j = s - 1; j >= 0; --j) {
    const double t = tau[j];
    hh_apply<SMAX>(A, rows, s, j, t, red, vsum, wsh);
    double* x = A + (int64_t)j * rows;
    for (int r = tid; r < rows; r += kHHThreads) x[r] = (r < j) ? 0.0 : (r == j ? 1.0 - t : -t * x[r]);
    __syncthreads();
  }
  // signs: D = diag(sgn(R_jj)), Q_i D and D R_i
  if (tid < s) dsg[tid] = (Rs[tid * s + tid] >= 0.0) ? 1.0 : -1.0;
  __syncthreads();
  double* slot = a.V;  // the new local panel (k = 0)
  for (int idx = tid; idx < rows * s; idx += kHHThreads) {
    const int r = idx / s, l = idx - r * s;
    slot[(r0 + r) * s + l] = A[(int64_t)l * rows + r] * dsg[l];
  }
  if (a.colexp) {  // largest biased exponent of each panel column on this chunk
    for (int l = 0; l < s; ++l) {
      int m = 0;
      for (int r = tid; r < rows; r += kHHThreads)
        m = max(m, (int)((((unsigned long long)__double_as_longlong(A[(int64_t)l * rows + r])) >> 52) & 0x7FF));
      m = __reduce_max_sync(0xffffffffu, m);
      if ((tid & 31) == 0) atomicMax(&hs[l], m);
    }
    __syncthreads();
    if (tid < s) a.colexp[(int64_t)tid * a.p + c] = hs[tid];
  }
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  for (int e = tid; e < s * s; e += kHHThreads) {
    const int i = e / s, l = e - i * s;
    const double nv = Rs[e] * dsg[i];
    smallc[SL.N_last + e] = nv;
    smallc[SL.N_comb + e] = nv;
    smallc[SL.Ninv_last + e] = (i == l) ? 1.0 : 0.0;
  }
}

// FlatTSPQR (Alg. 10) inside a chunk too large for one tile, with Householder
// sub-solvers: one CTA walks the chunk's sub-tiles X_1 .. X_m of up to T rows
// in order.  Stage 1 is the Householder QR of X_1; stage i > 1 factors the
// previous R stacked on the next sub-tile, [R_{i-1}; X_i] = Qh_i R_i
// ((s + rows_i) x s, the carried rows first).  The reflectors stay behind:
// their parts on the sub-tile's rows in the chunk's rows of the new panel,
// their parts on the carried rows and the tau in hh_scratch.  The chunk's R
// is R_m (signs normalized, D = diag(sgn R_jj)).  The explicit local factor
// then comes from a backward pass: with M_m = D and M_{i-1} = Qh_i^top M_i,
// the rows of sub-tile i are Qh_i^bot M_i (Qh_1 M_1 for the first), where
// Qh_i is formed in place from its reflectors as in k_hh_leaf.  Three levels
// of the method's recursion: sub-tiles (flat) -> chunk -> reduction tree.

// Householder QR of the nrows x s column-major tile A (leading dimension
// lda): reflectors below the diagonal (v_j[j] = 1 implicit), tau_j in tau[j],
// R on and above it.  Whole CTA.  Returns false (after latching
// LO_ERR_NONFINITE) on a non-finite norm.
template <int SMAX>
__device__ bool hh_factor_tile(double* A, int lda, int nrows, int s, double* tau, double* red, double* vsum,
                               double* wsh, int* flags) {
  const int tid = threadIdx.x;
  for (int j = 0; j < s; ++j) {
    double* x = A + (int64_t)j * lda;
    double v[SMAX];
#pragma unroll
    for (int cc = 0; cc < SMAX; ++cc) v[cc] = 0.0;
    for (int r = j + tid; r < nrows; r += kHHThreads) v[0] = fma(x[r], x[r], v[0]);
    hh_block_sum<SMAX>(v, 1, red, vsum);
    const double alpha = sqrt(vsum[0]);
    const double x0 = x[j];
    const double beta = (x0 >= 0.0) ? -alpha : alpha;
    const double t = (alpha == 0.0) ? 0.0 : (beta - x0) / beta;
    if (!isfinite(alpha)) {
      if (tid == 0) set_status(flags, LO_ERR_NONFINITE);
      return false;
    }
    __syncthreads();
    if (alpha != 0.0) {
      const double scal = 1.0 / (x0 - beta);
      for (int r = j + 1 + tid; r < nrows; r += kHHThreads) x[r] *= scal;
    }
    if (tid == 0) {
      x[j] = beta;
      tau[j] = t;
    }
    __syncthreads();
    hh_apply_lda<SMAX>(A, lda, nrows, s, j, t, red, vsum, wsh);
  }
  return true;
}

// Qh = H_0 .. H_{s-1} [I; 0] in place over the reflectors of the tile.
template <int SMAX>
__device__ void hh_form_q(double* A, int lda, int nrows, int s, const double* tau, double* red, double* vsum,
                          double* wsh) {
  for (int j = s - 1; j >= 0; --j) {
    const double t = tau[j];
    hh_apply_lda<SMAX>(A, lda, nrows, s, j, t, red, vsum, wsh);
    double* x = A + (int64_t)j * lda;
    for (int r = threadIdx.x; r < nrows; r += kHHThreads) x[r] = (r < j) ? 0.0 : (r == j ? 1.0 - t : -t * x[r]);
    __syncthreads();
  }
}

template <int SMAX>
__global__ void __launch_bounds__(kHHThreads) k_hh_flat(StepArgs a, int T) {
  extern __shared__ __align__(16) double A[];  // (s + T) x s, column-major, leading dimension s + T
  __shared__ double red[(kHHThreads / 32) * 32];
  __shared__ double vsum[32], wsh[32], tau[32], dsg[32];
  __shared__ double Rs[32 * 32], Mn[32 * 32];
  __shared__ int hs[32];
  const int c = blockIdx.x, s = a.s, tid = threadIdx.x, lda = s + T;
  const int64_t r0 = a.chunk_row0[c];
  const int rows = (int)(a.chunk_row0[c + 1] - r0);
  const int m = (rows + T - 1) / T;
  const int stage = s * s + s;
  double* scr = a.hh_scratch + (int64_t)c * a.hh_stages * stage;  // per stage: carried parts s x s, then tau
  double* slot = a.V;
  if (tid < 32) hs[tid] = 0;
  // ---- forward: stage i factors [R_{i-1}; X_i]
  for (int i = 0; i < m; ++i) {
    const int off = (i > 0) ? s : 0, ri = min(T, rows - i * T), nr = off + ri;
    const int64_t g0 = r0 + (int64_t)i * T;
    if (i > 0)  // the carried rows: R_{i-1}, zeros below its diagonal
      for (int e = tid; e < s * s; e += kHHThreads) {
        const int rr = e / s, l = e - rr * s;
        A[(int64_t)l * lda + rr] = (rr <= l) ? Rs[rr * s + l] : 0.0;
      }
    int bad = 0;
    for (int idx = tid; idx < ri * s; idx += kHHThreads) {
      const int r = idx / s, l = idx - r * s;
      const double x = a.W[(g0 + r) * a.ldw + l];
      bad |= isfinite(x) ? 0 : 1;
      A[(int64_t)l * lda + off + r] = x;
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) set_status(a.flags, LO_ERR_NONFINITE);
      return;
    }
    if (!hh_factor_tile<SMAX>(A, lda, nr, s, tau, red, vsum, wsh, a.flags)) return;
    // keep R_i; store the reflectors (carried rows: scratch; sub-tile rows: the panel)
    for (int e = tid; e < s * s; e += kHHThreads) {
      const int rr = e / s, l = e - rr * s;
      Rs[e] = (rr <= l) ? A[(int64_t)l * lda + rr] : 0.0;
      if (i > 0) scr[(int64_t)i * stage + e] = A[(int64_t)l * lda + rr];
    }
    if (tid < s) scr[(int64_t)i * stage + s * s + tid] = tau[tid];
    for (int idx = tid; idx < ri * s; idx += kHHThreads) {
      const int r = idx / s, l = idx - r * s;
      slot[(g0 + r) * s + l] = A[(int64_t)l * lda + off + r];
    }
    __syncthreads();
  }
  if (tid < s) dsg[tid] = (Rs[tid * s + tid] >= 0.0) ? 1.0 : -1.0;
  __syncthreads();
  // ---- the chunk's normalizer D R_m, N_last^{-1} = I
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  double* smallc = a.small + (int64_t)c * SL.stride;
  for (int e = tid; e < s * s; e += kHHThreads) {
    const int ii = e / s, l = e - ii * s;
    const double nv = Rs[e] * dsg[ii];
    smallc[SL.N_last + e] = nv;
    smallc[SL.N_comb + e] = nv;
    smallc[SL.Ninv_last + e] = (ii == l) ? 1.0 : 0.0;
  }
  // ---- backward: M_m = D; stage i: Qh_i from its reflectors, rows times M_i
  for (int e = tid; e < s * s; e += kHHThreads) Rs[e] = ((e / s) == (e % s)) ? dsg[e / s] : 0.0;
  __syncthreads();
  int hmax[SMAX];  // this thread's largest biased exponent per panel column
#pragma unroll
  for (int l = 0; l < SMAX; ++l) hmax[l] = 0;
  for (int i = m - 1; i >= 0; --i) {
    const int off = (i > 0) ? s : 0, ri = min(T, rows - i * T), nr = off + ri;
    const int64_t g0 = r0 + (int64_t)i * T;
    if (i > 0)
      for (int e = tid; e < s * s; e += kHHThreads) {
        const int rr = e / s, l = e - rr * s;
        A[(int64_t)l * lda + rr] = scr[(int64_t)i * stage + e];
      }
    for (int idx = tid; idx < ri * s; idx += kHHThreads) {
      const int r = idx / s, l = idx - r * s;
      A[(int64_t)l * lda + off + r] = slot[(g0 + r) * s + l];
    }
    if (tid < s) tau[tid] = scr[(int64_t)i * stage + s * s + tid];
    __syncthreads();
    hh_form_q<SMAX>(A, lda, nr, s, tau, red, vsum, wsh);
    // rows of Qh_i times M_i: the sub-tile's rows into the panel, the carried rows the next M
    for (int r = tid; r < nr; r += kHHThreads) {
      double q[SMAX];
#pragma unroll
      for (int l = 0; l < SMAX; ++l) q[l] = (l < s) ? A[(int64_t)l * lda + r] : 0.0;
#pragma unroll
      for (int l = 0; l < SMAX; ++l) {
        if (l < s) {
          double o = 0.0;
#pragma unroll
          for (int j = 0; j < SMAX; ++j)
            if (j < s) o = fma(q[j], Rs[j * s + l], o);
          if (r >= off) {
            slot[(g0 + r - off) * s + l] = o;
            hmax[l] = max(hmax[l], (int)((((unsigned long long)__double_as_longlong(o)) >> 52) & 0x7FF));
          } else {
            Mn[r * s + l] = o;
          }
        }
      }
    }
    __syncthreads();
    if (i > 0) {
      for (int e = tid; e < s * s; e += kHHThreads) Rs[e] = Mn[e];
      __syncthreads();
    }
  }
  if (a.colexp) {
#pragma unroll
    for (int l = 0; l < SMAX; ++l)
      if (l < s) {
        const int mx = __reduce_max_sync(0xffffffffu, hmax[l]);
        if ((tid & 31) == 0) atomicMax(&hs[l], mx);
      }
    __syncthreads();
    if (tid < s) a.colexp[(int64_t)tid * a.p + c] = hs[tid];
  }
}

// Stage 2 after the Householder leaf: the local panel is Q_i already, so the
// assembly is U = Q_i Nt_i (Sec. 4.1, with P empty at k = 0); one thread per
// row, the row's s values in registers, Nt_i upper triangular.
template <int SMAX>
__global__ void __launch_bounds__(256) k_hh_assemble(StepArgs a) {
  const SlabInfo si = a.slabs[blockIdx.x];
  const int s = a.s;
  const double* slot = a.V;
  const double* Nt = a.T + (int64_t)si.chunk * a.tstride + tblock_offset(0, s);
  for (int r = threadIdx.x; r < si.rows; r += 256) {
    const int64_t row = si.row0 + r;
    double q[SMAX];
#pragma unroll
    for (int l = 0; l < SMAX; ++l) q[l] = (l < s) ? slot[row * s + l] : 0.0;
#pragma unroll
    for (int l = 0; l < SMAX; ++l) {
      if (l < s) {
        double o = 0.0;
#pragma unroll
        for (int j = 0; j <= l; ++j) o = fma(q[j], __ldg(Nt + j * s + l), o);
        a.U[row * a.ldu + l] = o;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Many independent PQR steps in one persistent launch.
//
// The work of every instance is cut into items -- (instance, slab) for the two
// Gram passes and the assembly, (instance, chunk) for the reduction's per-chunk
// products -- and all items form one list in phase order: pass-1 Grams of all
// instances, pass-2 iterates and Grams, first reduction updates, second
// reduction updates, assemblies, digit planes.  Each CTA takes the next item
// from a global counter.  Tickets hand the small factorizations to the CTA
// that finishes last: the last Gram slab of a chunk runs the chunk's leaf
// (Alg. 7 / Alg. 8), the last chunk of an instance the reduction's small
// factorization (the tree's two summation levels in the same fixed order as
// k_tree_sum1 / k_tree_sum2, so results are bit for bit those of the
// sequential launches).  An item waits only for work handed out before it
// (items are taken in list order and every dependency points backwards), so
// the CTAs that hold it are running and the wait ends; each wait is bounded
// all the same (about 1 s), after which the batch is aborted with
// LO_ERR_TIMEOUT.  The instances run BCGS-PIP+ with exactly two local passes
// and two reduction iterations; one whose estimate asks for more (or whose
// Cholesky needed the shifted retry) is marked in its flags and redone by the
// caller on the regular path.

// Per-instance ticket area (ints), p = chunks.
struct TickLayout {
  static __host__ __device__ int cntA(int p) { return 0; }      // [p] pass-1 slabs done per chunk
  static __host__ __device__ int cntB(int p) { return p; }      // [p] pass-2 slabs done per chunk
  static __host__ __device__ int cntE(int p) { return 2 * p; }  // [p] assembly slabs done per chunk
  static __host__ __device__ int stage(int p) { return 3 * p; } // [p] chunk stage (1 leaf 1, 2 leaf 2, 4 tree, 5 panel)
  static __host__ __device__ int inst(int p) { return 4 * p; }  // [4]: chunks done (it 1), (it 2), instance stage
  static __host__ __device__ int ints(int p) { return 4 * p + 4; }
};

constexpr int kBatchPhases = 6;
constexpr long long kBatchWaitCycles = 2000000000ll;  // ~1 s

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait of the whole CTA until *p >= v; false if the batch was aborted
// (here or elsewhere).
__device__ bool batch_wait(const int* p, int v, int* abort_word, int* flags) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int good = 1;
    if (ld_acquire(p) < v) {
      const long long t0 = clock64();
      while (ld_acquire(p) < v) {
        if (ld_acquire(abort_word) != 0) {
          good = 0;
          break;
        }
        if (clock64() - t0 > kBatchWaitCycles) {
          atomicExch(abort_word, 1);
          set_status(flags, LO_ERR_TIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  const bool r = ok != 0;
  __syncthreads();
  return r;
}

// Returns true in every thread of the CTA that took the last of `total`
// tickets on *cnt (after its own work: the release of what it wrote, and the
// acquire of what the others wrote).
__device__ bool batch_ticket(int* cnt, int total) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = (atomicAdd(cnt, 1) == total - 1) ? 1 : 0;
    if (last) __threadfence();
  }
  __syncthreads();
  const bool r = last != 0;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void batch_release(int* p, int v) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(p, v);
}

// The reduction's summed contributions Z = sum_i z_i in the two fixed levels
// of k_tree_sum1 / k_tree_sum2 (groups of kTreeGroup chunks, then the groups).
__device__ void batch_tree_sum(const StepArgs& a) {
  const int s = a.s, E = (a.nb * s + s) * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  double* Z = a.glob + GlobLayout::make(a.Kmax, s).Zsum;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double tot = 0.0;
    for (int c0 = 0; c0 < a.p; c0 += kTreeGroup) {
      double v = 0.0;
      for (int c = c0; c < min(a.p, c0 + kTreeGroup); ++c) v += a.small[(int64_t)c * SL.stride + SL.Z + e];
      tot += v;
    }
    Z[e] = tot;
  }
  __syncthreads();
}

// Stage 2 of one slab and, for a tensor-core basis, the new panel's column
// exponents on it (maxima into colexp, zeroed by the chunk's last tree item).
__device__ void batch_update_slab(const BatchInst& I, int slab, double* sm) {
  const StepArgs& a = I.a;
  update_slab(a, I.tile_u, slab, sm);
  __syncthreads();
  if (a.colexp) {
    const SlabInfo si = a.slabs[slab];
    const int s = a.s, k = a.nb * s;
    const double* slot = a.V + (int64_t)a.nb * a.n * s;
    for (int l = 0; l < s; ++l) {
      int m = 0;
      for (int r = threadIdx.x; r < si.rows; r += blockDim.x) m = max(m, bexp(slot[(si.row0 + r) * s + l]));
      m = __reduce_max_sync(0xffffffffu, m);
      if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&a.colexp[(int64_t)(k + l) * a.p + si.chunk], m);
    }
  }
}

__device__ void batch_gram1(const BatchInst& I, int slab, unsigned char* smem) {
  const StepArgs& a = I.a;
  double* red = reinterpret_cast<double*>(smem);
  if (I.gram1) {
    switch (a.s) {
      case 1: gram1_slab<1, double>(a, slab, red); return;
      case 2: gram1_slab<2, double>(a, slab, red); return;
      case 4: gram1_slab<4, double>(a, slab, red); return;
      case 8: gram1_slab<8, double>(a, slab, red); return;
      case 16: gram1_slab<16, double>(a, slab, red); return;
      case 32: gram1_slab<32, double>(a, slab, red); return;
    }
  }
  gram_slab<double, double>(a, 1, I.tile_g, slab, smem);
}

__device__ void batch_digitize(const StepArgs& a, int slab) {
  switch (a.s) {
    case 8: digitize_slab<8>(a, slab); break;
    case 16: digitize_slab<16>(a, slab); break;
    case 32: digitize_slab<32>(a, slab); break;
  }
}

// Flags of every instance as k_step_begin sets them (PIP+: pass 2 and tree
// iteration 2 forced), zeroed tickets, the item counter and the abort word.
__global__ void k_batch_init(BatchInst* insts, int ninst, int* counters) {
  if (blockIdx.x == 0 && threadIdx.x < 2) counters[threadIdx.x] = 0;
  for (int j = blockIdx.x; j < ninst; j += gridDim.x) {
    const BatchInst& I = insts[j];
    if (threadIdx.x == 0) {
      for (int t = 1; t <= kMaxPass; ++t) I.a.flags[kFlagPass + t - 1] = (t <= 2) ? 1 : 0;
      for (int t = 1; t <= kMaxTreeIter; ++t) I.a.flags[kFlagTree + t - 1] = (t <= 2) ? 1 : 0;
    }
    for (int e = threadIdx.x; e < TickLayout::ints(I.a.p); e += blockDim.x) I.tick[e] = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_batch_step(const BatchInst* __restrict__ insts, int ninst,
                                                         const int* __restrict__ pref, int* counters) {
  extern __shared__ __align__(16) unsigned char bsm[];
  double* sm = reinterpret_cast<double*>(bsm);
  __shared__ int item, aborted;
  int* next = counters;
  int* abort_word = counters + 1;
  const int total = pref[kBatchPhases * (ninst + 1) - 1];
  // every pass takes a new, larger item index, so a CTA makes at most total + 1 passes
  for (int pass_no = 0; pass_no <= total; ++pass_no) {
    if (threadIdx.x == 0) {
      item = atomicAdd(next, 1);
      aborted = ld_acquire(abort_word);
    }
    __syncthreads();
    const int g = item;
    const bool skip = aborted != 0;
    __syncthreads();
    if (g >= total) break;
    if (skip) continue;
    // phase and instance: pref[ph * (ninst + 1) + j] is the first item of instance j in phase ph
    int ph = 0;
    while (g >= pref[ph * (ninst + 1) + ninst]) ++ph;  // ph < kBatchPhases: g < total = end of the last phase
    int j = 0;
    while (g >= pref[ph * (ninst + 1) + j + 1]) ++j;   // j < ninst: g < the phase's end
    const int idx = g - pref[ph * (ninst + 1) + j];
    const BatchInst& I = insts[j];
    const StepArgs& a = I.a;
    const int p = a.p;
    int* tick = I.tick;
    int* inst = tick + TickLayout::inst(p);
    if (ph == 0) {  // pass-1 Gram of slab idx
      batch_gram1(I, idx, bsm);
      const int c = a.slabs[idx].chunk;
      if (batch_ticket(tick + TickLayout::cntA(p) + c, a.chunk_slab0[c + 1] - a.chunk_slab0[c])) {
        leaf_chunk(a, 1, 0.0, a.leaf != LO_LEAF_PIP ? 1 : 0, DBL_EPSILON, c, sm);
        batch_release(tick + TickLayout::stage(p) + c, 1);
      }
    } else if (ph == 1) {  // pass-2 iterate and Gram of slab idx
      const int c = a.slabs[idx].chunk;
      if (!batch_wait(tick + TickLayout::stage(p) + c, 1, abort_word, a.flags)) continue;
      gram_slab<double, double>(a, 2, I.tile_g, idx, bsm);
      if (batch_ticket(tick + TickLayout::cntB(p) + c, a.chunk_slab0[c + 1] - a.chunk_slab0[c])) {
        leaf_chunk(a, 2, 0.0, 0, DBL_EPSILON, c, sm);
        __syncthreads();
        tree_contrib_chunk(a, 1, c, sm);
        batch_release(tick + TickLayout::stage(p) + c, 2);
        if (batch_ticket(inst + 0, p)) {
          batch_tree_sum(a);
          tree_sum2_core(a, 1, sm);
          batch_release(inst + 2, 1);
        }
      }
    } else if (ph == 2) {  // first reduction update and second contribution of chunk idx
      if (!batch_wait(inst + 2, 1, abort_word, a.flags)) continue;
      tree_update_chunk(a, 1, idx, sm);
      __syncthreads();
      tree_contrib_chunk(a, 2, idx, sm);
      if (batch_ticket(inst + 1, p)) {
        batch_tree_sum(a);
        tree_sum2_core(a, 2, sm);
        __syncthreads();
        const GlobLayout GL = GlobLayout::make(a.Kmax, a.s);
        const int ks = a.nb * a.s * a.s, ss = a.s * a.s;
        if (I.H)
          for (int e = threadIdx.x; e < ks; e += blockDim.x) I.H[e] = a.glob[GL.P_acc + e];
        if (I.R)
          for (int e = threadIdx.x; e < ss; e += blockDim.x) I.R[e] = a.glob[GL.N_acc + e];
        batch_release(inst + 2, 2);
      }
    } else if (ph == 3) {  // second reduction update of chunk idx: the new column block of T_i
      if (!batch_wait(inst + 2, 2, abort_word, a.flags)) continue;
      tree_update_chunk(a, 2, idx, sm);
      if (a.colexp)
        for (int l = threadIdx.x; l < a.s; l += blockDim.x) a.colexp[(int64_t)(a.nb * a.s + l) * p + idx] = 0;
      batch_release(tick + TickLayout::stage(p) + idx, 4);
    } else if (ph == 4) {  // assembly of slab idx
      const int c = a.slabs[idx].chunk;
      if (!batch_wait(tick + TickLayout::stage(p) + c, 4, abort_word, a.flags)) continue;
      batch_update_slab(I, idx, sm);
      if (I.digitize && batch_ticket(tick + TickLayout::cntE(p) + c, a.chunk_slab0[c + 1] - a.chunk_slab0[c]))
        batch_release(tick + TickLayout::stage(p) + c, 5);
    } else {  // digit planes of the new panel on slab idx (the chunk's exponents are final)
      const int c = a.slabs[idx].chunk;
      if (!batch_wait(tick + TickLayout::stage(p) + c, 5, abort_word, a.flags)) continue;
      batch_digitize(a, idx);
    }
  }
}

// The reduction (Sec. 4.1, BCGS-PIP reiterated as in Alg. 8) in two launches
// per iteration.  k_tree_round: every chunk's CTA first applies the update of
// the previous iteration (with_update: X_hat, Nx_hat and the column block of
// T_i), then forms its contribution z_i of iteration `it`.  k_tree_sum:
// the first summation level of k_tree_sum1 (groups of kTreeGroup chunks, the
// entries split over blockIdx.y), and the CTA that finishes last (ticket on
// a.tree_ticket, reset after use) sums the groups and runs the small
// factorization of k_tree_sum2.  Nothing waits; the same arithmetic in the
// same order as the four kernels per iteration, bit for bit.
__global__ void __launch_bounds__(kThreads) k_tree_round(StepArgs a, int it, int with_update) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x;
  if (with_update && a.flags[kFlagTree + it - 2]) {
    tree_update_chunk(a, it - 1, c, sm);
    __syncthreads();
  }
  if (!a.flags[kFlagTree + it - 1]) return;
  tree_contrib_chunk(a, it, c, sm);
}

// k_tree_round and k_tree_update with T_i staged in shared memory (when
// tree_staged_smem fits).
__global__ void __launch_bounds__(kThreads) k_tree_round_st(StepArgs a, int it, int with_update) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x;
  if (with_update && a.flags[kFlagTree + it - 2]) {
    tree_update_chunk_st(a, it - 1, c, sm);
    __syncthreads();
  }
  if (!a.flags[kFlagTree + it - 1]) return;
  tree_contrib_chunk_st(a, it, c, sm);
}

__global__ void __launch_bounds__(kThreads) k_tree_update_st(StepArgs a, int it) {
  if (!a.flags[kFlagTree + it - 1]) return;
  extern __shared__ __align__(16) double sm[];
  tree_update_chunk_st(a, it, blockIdx.x, sm);
}

__global__ void __launch_bounds__(kThreads) k_tree_sum(StepArgs a, int it, int ngroups) {
  extern __shared__ __align__(16) double sm[];
  if (!a.flags[kFlagTree + it - 1]) return;
  const int s = a.s, E = (a.nb * s + s) * s;
  const SmallLayout SL = SmallLayout::make(a.Kmax, s);
  const int c0 = blockIdx.x * kTreeGroup, c1 = min(a.p, c0 + kTreeGroup);
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < E; e += gridDim.y * blockDim.x) {
    double v = 0.0;
    for (int c = c0; c < c1; ++c) v += a.small[(int64_t)c * SL.stride + SL.Z + e];
    a.tsum[(int64_t)blockIdx.x * a.Kmax * s + e] = v;
  }
  if (batch_ticket(a.tree_ticket, (int)(gridDim.x * gridDim.y))) {
    double* Z = a.glob + GlobLayout::make(a.Kmax, s).Zsum;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      double v = 0.0;
      for (int g = 0; g < ngroups; ++g) v += a.tsum[(int64_t)g * a.Kmax * s + e];
      Z[e] = v;
    }
    __syncthreads();
    tree_sum2_core(a, it, sm);
    if (threadIdx.x == 0) *a.tree_ticket = 0;
  }
}

// Shared-memory budget of the streaming kernels (bytes).
constexpr int kTileSmem = 96 * 1024;

int gram_tile_rows(int Kt, int s, int elem) {
  int r = (kTileSmem - 8 * 32 * s) / (elem * Kt);
  return r < 1 ? 1 : (r > 32 ? 32 : r);
}

int update_tile_rows(int k, int s) {
  int per_row = 8 * (k + 2 * s);
  int r = kTileSmem / per_row;
  return r < 1 ? 1 : (r > 32 ? 32 : r);
}

bool g_attr_done = false;

cudaError_t set_attrs() {
  if (g_attr_done) return cudaSuccess;
  const int big = 200 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_gram<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_gram<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
#define LO_GRAM1_ATTR(S)                                                                            if ((e = cudaFuncSetAttribute(k_gram1<S, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))     return e;                                                                                       if ((e = cudaFuncSetAttribute(k_gram1<S, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  LO_GRAM1_ATTR(1)
  LO_GRAM1_ATTR(2)
  LO_GRAM1_ATTR(4)
  LO_GRAM1_ATTR(8)
  LO_GRAM1_ATTR(16)
  LO_GRAM1_ATTR(32)
#undef LO_GRAM1_ATTR
  if ((e = cudaFuncSetAttribute(k_tree_contrib, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_tree_sum2, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_tree_update, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_apply_y, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_tree_round, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_tree_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_tree_round_st, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_tree_update_st, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_leaf<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_flat<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_flat<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_flat<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_flat<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_leaf<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_leaf<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  if ((e = cudaFuncSetAttribute(k_hh_leaf<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kHHTileBytes))) return e;
  g_attr_done = true;
  return cudaSuccess;
}

std::atomic<long long> g_launches{0};

inline void mark(ProfHook* h, int kind, bool begin, cudaStream_t st) {
  if (h) h->mark(kind, begin, st);
}

}  // namespace

long long launches() { return g_launches.load(); }

cudaError_t launch_prepare() {
  cudaError_t e = set_attrs();
  if (e == cudaSuccess) e = oz_set_attrs();
  if (e == cudaSuccess) e = umma_set_attrs();
  return e;
}

namespace {
// Deterministic, well-conditioned synthetic block for timing (a sum of sines of
// incommensurate frequencies per column); used only by the chunk-size tuner.
__global__ void k_fill_pattern(double* X, int64_t count, unsigned salt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)(i + 1) * 0.6180339887498949 + (double)salt * 0.7548776662466927;
    X[i] = sin(x * 12.9898) + 0.5 * cos(x * 78.233);
  }
}
unsigned g_fill_salt = 0;
}  // namespace

cudaError_t launch_fill_pattern(double* X, int64_t count, cudaStream_t st) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_fill_pattern<<<(int)blocks, 256, 0, st>>>(X, count, ++g_fill_salt);
  count_launches(1);
  return cudaGetLastError();
}
void count_launches(int k) { g_launches += k; }

// Reduction step (Sec. 4.1): BCGS-PIP on the stacked factors, reiterated.
void launch_reduction(const StepArgs& a, cudaStream_t st, ProfHook* hook) {
  const int s = a.s, k = a.nb * s, Kt = k + s, ss = s * s;
  const int ngroups = (a.p + kTreeGroup - 1) / kTreeGroup;
  const int iters = a.reduction == 1 ? 1 : kMaxTreeIter;
  mark(hook, kKindTree, true, st);
  if (a.tree_ticket) {
    // per iteration: (update of it - 1 +) contribution, then the ticketed sums
    // and factorization; the last update at the end
    const size_t smr = 8 * ((size_t)k * s + 2 * ss), sst = tree_staged_smem(k, s);
    const dim3 gsum(ngroups, (unsigned)((Kt * s + kThreads - 1) / kThreads));
    for (int it = 1; it <= iters; ++it) {
      if (sst)
        k_tree_round_st<<<a.p, kThreads, sst, st>>>(a, it, it > 1 ? 1 : 0);
      else
        k_tree_round<<<a.p, kThreads, smr, st>>>(a, it, it > 1 ? 1 : 0);
      k_tree_sum<<<gsum, kThreads, 8 * (4 * (size_t)ss + 4), st>>>(a, it, ngroups);
    }
    if (sst)
      k_tree_update_st<<<a.p, kThreads, sst, st>>>(a, iters);
    else
      k_tree_update<<<a.p, kThreads, 8 * ((size_t)k * s + 2 * ss), st>>>(a, iters);
    count_launches(2 * iters + 1);
  } else {
    for (int it = 1; it <= iters; ++it) {
      k_tree_contrib<<<a.p, kThreads, 8 * ((size_t)k * s + ss), st>>>(a, it);
      k_tree_sum1<<<dim3(ngroups, (unsigned)((Kt * s + kThreads - 1) / kThreads)), kThreads, 0, st>>>(a, it);
      k_tree_sum2<<<1, kThreads, 8 * (4 * (size_t)ss + 4), st>>>(a, it, ngroups);
      k_tree_update<<<a.p, kThreads, 8 * ((size_t)k * s + 2 * ss), st>>>(a, it);
      count_launches(4);
    }
  }
  mark(hook, kKindTree, false, st);
}

// The step without prior blocks with the Householder leaf: k_hh_leaf per
// chunk, the reduction, and the assembly U = Q_i Nt_i (plus the digit planes of
// the new panel for a tensor-core basis that keeps them).
cudaError_t launch_step_hh(const StepArgs& a, cudaStream_t st, ProfHook* hook) {
  const int s = a.s;
  const size_t tile = sizeof(double) * (size_t)a.max_chunk_rows * s;
  const bool flat = tile > (size_t)kHHTileBytes;  // chunks walked as sub-tiles (FlatTSPQR)
  if (a.nb != 0 || (flat && !a.hh_scratch)) return cudaErrorInvalidValue;
  const size_t ftile = sizeof(double) * (size_t)(a.hh_T + s) * s;
  const bool tc = (a.precision == LO_PREC_FP64_TC || a.precision == LO_PREC_MIXED_TC);
  cudaError_t e;
  if (tc && (e = umma_set_attrs())) return e;
  k_step_begin<<<1, 32, 0, st>>>(a.flags, 0, a.reduction != 1);
  count_launches(1);
  mark(hook, kKindLeaf, true, st);
  if (flat) {
    if (s <= 4)
      k_hh_flat<4><<<a.p, kHHThreads, ftile, st>>>(a, a.hh_T);
    else if (s <= 8)
      k_hh_flat<8><<<a.p, kHHThreads, ftile, st>>>(a, a.hh_T);
    else if (s <= 16)
      k_hh_flat<16><<<a.p, kHHThreads, ftile, st>>>(a, a.hh_T);
    else
      k_hh_flat<32><<<a.p, kHHThreads, ftile, st>>>(a, a.hh_T);
  } else if (s <= 4) {
    k_hh_leaf<4><<<a.p, kHHThreads, tile, st>>>(a);
  } else if (s <= 8) {
    k_hh_leaf<8><<<a.p, kHHThreads, tile, st>>>(a);
  } else if (s <= 16) {
    k_hh_leaf<16><<<a.p, kHHThreads, tile, st>>>(a);
  } else {
    k_hh_leaf<32><<<a.p, kHHThreads, tile, st>>>(a);
  }
  count_launches(1);
  mark(hook, kKindLeaf, false, st);
  launch_reduction(a, st, hook);
  mark(hook, kKindUpdate, true, st);
  if (s <= 4)
    k_hh_assemble<4><<<a.nslab, 256, 0, st>>>(a);
  else if (s <= 8)
    k_hh_assemble<8><<<a.nslab, 256, 0, st>>>(a);
  else if (s <= 16)
    k_hh_assemble<16><<<a.nslab, 256, 0, st>>>(a);
  else
    k_hh_assemble<32><<<a.nslab, 256, 0, st>>>(a);
  count_launches(1);
  if (tc && a.dig && a.nb + 1 < a.M) {
    if ((e = launch_umma_digitize(a, st))) return e;
    count_launches(1);
  }
  mark(hook, kKindUpdate, false, st);
  return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs& a_in, cudaStream_t st, ProfHook* hook) {
  cudaError_t e = set_attrs();
  if (e) return e;
  StepArgs a = a_in;
  if (a.op_nx) {
    // The operator is formed inside the first Gram pass where that pass can
    // (the float64 Grams; on the tensor cores the digit-plane Gram of the
    // float64 form); otherwise the operator kernel writes the block into U
    // first.  Either way the rest of the step reads the block from U.
    const bool mixed_form = (a.precision == LO_PREC_MIXED_FP32 || a.precision == LO_PREC_MIXED_TC);
    const bool tc_form = (a.precision == LO_PREC_FP64_TC || a.precision == LO_PREC_MIXED_TC);
    const bool fused = a.nb > 0 && !mixed_form && a.leaf != LO_LEAF_HH && (!tc_form || umma_op_supported(a));
    if (!fused) {
      if ((e = launch_laplace5(a.op_nx, a.op_ny, a.s, a.op_V, a.op_ldv, a.U, a.ldu, st))) return e;
      a.op_nx = 0;
      a.W = a.U;
      a.ldw = a.ldu;
    }
  }
  if (a.leaf == LO_LEAF_HH && a.nb == 0) return launch_step_hh(a, st, hook);
  const int s = a.s, k = a.nb * s, Kt = k + s, ss = s * s;
  const bool mixed = (a.precision == LO_PREC_MIXED_FP32 || a.precision == LO_PREC_MIXED_TC);
  // The reduction always reiterates (BCGS-PIP+) unless plain PIP is asked for: its
  // projection uses the stacked tree factors of all earlier steps, whose rounding
  // errors a single pass amplifies step after step.
  k_step_begin<<<1, 32, 0, st>>>(a.flags, (a.leaf == LO_LEAF_PIP2) || (a.leaf == LO_LEAF_HH) || mixed,
                                 a.reduction != 1);
  count_launches(1);
  // stage 1
  const int maxpass = (a.leaf == LO_LEAF_PIP && !mixed) ? 1 : kMaxPass;
  const bool tc = (a.precision == LO_PREC_FP64_TC || a.precision == LO_PREC_MIXED_TC);
  if (tc && (e = oz_set_attrs())) return e;
  if (tc && (e = umma_set_attrs())) return e;
  for (int pass = 1; pass <= maxpass; ++pass) {
    mark(hook, pass == 1 ? kKindGram : kKindRefine, true, st);
    if (tc && !(pass == 1 && mixed)) {
      if (pass >= 2 && (e = launch_oz_ypass(a, pass, st))) return e;
      if ((e = launch_oz_gram(a, pass, st))) return e;
      count_launches(pass >= 2 ? 3 : (umma_enabled(a) ? 2 : 1));
    } else if (tc && pass == 1 && mixed && umma_enabled(a)) {
      // the mixed form's first pass on the tensor cores: the leading digits
      // of both factors, only their planes read
      if ((e = launch_umma_gram_mixed(a, st))) return e;
      count_launches(2);
    } else if (a.nb == 0 && s <= 4 && !(pass == 1 && mixed)) {
      if ((e = launch_gram_narrow(a, pass, st))) return e;
      count_launches(1);
    } else if (pass == 1 && gram1_supported(s)) {
      if ((e = mixed ? launch_gram1<float>(a, st) : launch_gram1<double>(a, st))) return e;
      count_launches(1);
    } else if (pass == 1 && mixed) {
      const int tr = gram_tile_rows(Kt, s, 4);
      const size_t sm = (((size_t)4 * tr * Kt + 15) & ~(size_t)15) + 8 * (size_t)tr * s + 8 * kThreads;
      k_gram<float, float><<<a.nslab, kThreads, sm, st>>>(a, pass, tr);
      count_launches(1);
    } else {
      const int tr = gram_tile_rows(Kt, s, 8);
      const size_t sm = (size_t)8 * tr * Kt + 8 * (size_t)tr * s + 8 * kThreads;
      k_gram<double, double><<<a.nslab, kThreads, sm, st>>>(a, pass, tr);
      count_launches(1);
    }
    mark(hook, pass == 1 ? kKindGram : kKindRefine, false, st);
    if (pass == 1 && a.op_nx) {  // the operator's block is in U from here on
      a.op_nx = 0;
      a.W = a.U;
      a.ldw = a.ldu;
    }
    // the reduced-precision first pass of the mixed form: above a float32
    // Gram a fixed shift of 1e-5 of the trace; above the 32-bit digit Gram on
    // the tensor cores the plain Cholesky, with the shifted retry (and two
    // more passes) only on breakdown, both scaled to its unit roundoff, so a
    // moderately conditioned block needs no third pass
    const bool digit_first = pass == 1 && mixed && tc && umma_enabled(a) && a.leaf != LO_LEAF_PIP;
    const double shift = (pass == 1 && mixed && !digit_first) ? 1e-5 : 0.0;
    const double u_gram = digit_first ? 0x1p-31 : DBL_EPSILON;
    const size_t smleaf = 8 * ((size_t)Kt * s + 4 * ss + 4);
    if (pass == 1 && a.deflation_tol > 0.0) {
      k_defl_trace<<<1, kThreads, 0, st>>>(a);
      count_launches(1);
    }
    mark(hook, kKindLeaf, true, st);
    const int allow_shift = (pass == 1 && (!mixed || digit_first) && a.leaf != LO_LEAF_PIP) ? 1 : 0;
    k_leaf<<<a.p, kThreads, smleaf, st>>>(a, pass, shift, allow_shift, u_gram);
    mark(hook, kKindLeaf, false, st);
    count_launches(1);
  }
  launch_reduction(a, st, hook);
  // stage 2
  mark(hook, kKindUpdate, true, st);
  if (tc) {
    if ((e = cudaMemsetAsync(a.colexp + (int64_t)k * a.p, 0, sizeof(int) * (size_t)s * a.p, st))) return e;
    if ((e = launch_oz_stage2(a, st))) return e;
    count_launches(2);
    if (a.dig && a.nb + 1 < a.M) {  // the last panel is never read as a prior block
      if ((e = launch_umma_digitize(a, st))) return e;
      count_launches(1);
    }
  } else if (a.nb == 0 && s <= 4) {
    if ((e = launch_update_narrow(a, st))) return e;
    count_launches(1);
  } else {
    const int tu = update_tile_rows(k, s);
    k_update<<<a.nslab, kThreads, (size_t)8 * tu * (k + 2 * s), st>>>(a, tu);
    count_launches(1);
  }
  mark(hook, kKindUpdate, false, st);
  return cudaGetLastError();
}

cudaError_t launch_apply_q(const StepArgs& a, const double* C, int m, int64_t ldc, double* Z,
                           double* Y, int64_t ldy, cudaStream_t st, ProfHook* hook) {
  cudaError_t e = set_attrs();
  if (e) return e;
  const int k = a.nb * a.s;
  if (umma_apply_supported(a)) {  // digit planes of the panels: the tensor-core assembly
    if ((e = umma_set_attrs())) return e;
    mark(hook, kKindApply, true, st);
    e = launch_umma_apply(a, C, ldc, m, Y, ldy, st);
    mark(hook, kKindApply, false, st);
    count_launches(2 * ((m + a.s - 1) / a.s));
    return e;
  }
  mark(hook, kKindApply, true, st);
  k_apply_z<<<a.p, kThreads, 0, st>>>(a, C, m, ldc, Z);
  int tr = kTileSmem / (8 * (k > 0 ? k : 1));
  tr = tr < 1 ? 1 : (tr > 32 ? 32 : tr);
  k_apply_y<<<a.nslab, kThreads, (size_t)8 * tr * k, st>>>(a, m, Z, Y, ldy, tr);
  mark(hook, kKindApply, false, st);
  count_launches(2);
  return cudaGetLastError();
}

int batch_tick_ints(int p) { return TickLayout::ints(p); }

bool batch_fill(BatchInst* bi) {
  StepArgs& a = bi->a;
  const int s = a.s, k = a.nb * s, Kt = k + s;
  const bool tc = (a.precision == LO_PREC_FP64_TC);
  if (!(a.precision == LO_PREC_FP64 || tc)) return false;
  if (!(a.leaf == LO_LEAF_PIP2 || (a.leaf == LO_LEAF_HH && a.nb > 0))) return false;
  if (a.reduction == 1 || a.deflation_tol > 0.0 || a.test_stall) return false;
  bi->tile_g = gram_tile_rows(Kt, s, 8);
  bi->tile_u = update_tile_rows(k, s);
  bi->gram1 = gram1_supported(s) ? 1 : 0;
  bi->digitize = (tc && a.dig && a.nb + 1 < a.M && (s == 8 || s == 16 || s == 32)) ? 1 : 0;
  // float64 arithmetic throughout: no per-pass exponents of the digit forms
  a.srcexp = nullptr;
  a.srcexp_slab = nullptr;
  if (!tc) a.colexp = nullptr;
  return true;
}

size_t batch_smem(const BatchInst* insts, int ninst) {
  size_t m = sizeof(double) * kThreads * 32;  // the register-tiled Gram's reduction buffer
  for (int j = 0; j < ninst; ++j) {
    const StepArgs& a = insts[j].a;
    const size_t s = a.s, k = (size_t)a.nb * a.s, Kt = k + s, ss = s * s, tg = insts[j].tile_g;
    const size_t need[] = {8 * tg * Kt + 8 * tg * s + 8 * kThreads, 8 * (Kt * s + 4 * ss + 4), 8 * (k * s + 2 * ss),
                           8 * (4 * ss + 4), 8 * (size_t)insts[j].tile_u * (k + 2 * s)};
    for (size_t v : need) m = v > m ? v : m;
  }
  return m;
}

cudaError_t launch_batch(BatchInst* d_insts, int ninst, const int* d_pref, int* d_counters, size_t smem,
                         cudaStream_t st) {
  cudaError_t e = set_attrs();
  if (e) return e;
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_step, kThreads, smem) != cudaSuccess || per < 1)
    per = 1;
  k_batch_init<<<ninst < 152 ? ninst : 152, 256, 0, st>>>(d_insts, ninst, d_counters);
  k_batch_step<<<sms * per, kThreads, smem, st>>>(d_insts, ninst, d_pref, d_counters);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_laplace5(int nx, int ny, int s, const double* X, int64_t ldx, double* Y,
                            int64_t ldy, cudaStream_t st) {
  const int64_t total = (int64_t)nx * ny * s;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  k_laplace5<<<(int)blocks, 256, 0, st>>>(nx, ny, s, X, ldx, Y, ldy);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace lo

// ---------------------------------------------------------------------------
// Allocation-free variant of the first step (k = 0, a tall-skinny QR W = U R)
// for callers that may not allocate device memory.  All scratch of the step
// (flags, slab tables, Gram partials, per-chunk and global small matrices,
// tree factors) lives in one fixed file-scope device array; the caller's U is
// the working panel.  The kernels are the ones of the basis path, unchanged.
namespace lo {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

__global__ void k_noalloc_tables(int64_t n, int cr, int p, int slab_rows, int spc, int spl,
                                 SlabInfo* slabs, int32_t* chunk_slab0, int64_t* chunk_row0) {
  const int nslab = (p - 1) * spc + spl;
  const int64_t rows_last = n - (int64_t)(p - 1) * cr;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslab; i += gridDim.x * blockDim.x) {
    int c, j;
    int64_t crows;
    if (i < (p - 1) * spc) {
      c = i / spc;
      j = i - c * spc;
      crows = cr;
    } else {
      c = p - 1;
      j = i - (p - 1) * spc;
      crows = rows_last;
    }
    SlabInfo si;
    si.row0 = (int64_t)c * cr + (int64_t)j * slab_rows;
    const int64_t left = crows - (int64_t)j * slab_rows;
    si.rows = (int32_t)(left < slab_rows ? left : slab_rows);
    si.chunk = c;
    si.tile0 = 0;
    si.pad_ = 0;
    slabs[i] = si;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= p; c += gridDim.x * blockDim.x) {
    chunk_slab0[c] = (c < p) ? c * spc : nslab;
    chunk_row0[c] = (c < p) ? (int64_t)c * cr : n;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lo

namespace lo {
namespace {

// Scratch layout of one lo_tsqr_noalloc call (byte offsets into the array),
// validated and computed on the host before any device work.
struct NoAllocLayout {
  int p, nslab, slab_rows, spc, spl, ngroups;
  size_t o_flags, o_slabs, o_cs0, o_cr0, o_part, o_small, o_glob, o_tsum, o_T, bytes;
};

lo_status noalloc_layout(int64_t n, int32_t s, int32_t chunk_rows, NoAllocLayout* L) {
  if (n < 1 || s < 1 || s > kMaxS || chunk_rows < 1) return LO_ERR_INVALID_ARG;
  const int64_t p64 = n / chunk_rows > 0 ? n / chunk_rows : 1;
  if (p64 > (1 << 30)) return LO_ERR_INVALID_ARG;
  const int p = (int)p64;
  const int64_t min_rows = (p == 1) ? n : chunk_rows;
  if (min_rows < s) return LO_ERR_CHUNK_TOO_SMALL;
  const int slab_rows = 16 * s > 256 ? 16 * s : 256;
  const int64_t rows_last = n - (int64_t)(p - 1) * chunk_rows;
  const int64_t spc = (chunk_rows + slab_rows - 1) / slab_rows;
  const int64_t spl = (rows_last + slab_rows - 1) / slab_rows;
  const int64_t nslab64 = (int64_t)(p - 1) * spc + spl;
  if (nslab64 > (1 << 30) || spl > (1 << 30)) return LO_ERR_INVALID_ARG;
  const int nslab = (int)nslab64;
  const int ngroups = (p + kTreeGroup - 1) / kTreeGroup;
  const SmallLayout SL = SmallLayout::make(s, s);
  const GlobLayout GL = GlobLayout::make(s, s);
  const size_t ss = (size_t)s * s;
  size_t off = 0;
  L->o_flags = off;   off = align256(off + sizeof(int) * kFlagCount);
  L->o_slabs = off;   off = align256(off + sizeof(SlabInfo) * (size_t)nslab);
  L->o_cs0 = off;     off = align256(off + sizeof(int32_t) * (size_t)(p + 1));
  L->o_cr0 = off;     off = align256(off + sizeof(int64_t) * (size_t)(p + 1));
  L->o_part = off;    off = align256(off + sizeof(double) * (size_t)nslab * ss);
  L->o_small = off;   off = align256(off + sizeof(double) * (size_t)p * SL.stride);
  L->o_glob = off;    off = align256(off + sizeof(double) * (size_t)GL.stride);
  L->o_tsum = off;    off = align256(off + sizeof(double) * (size_t)ngroups * ss);
  L->o_T = off;       off = align256(off + sizeof(double) * (size_t)p * ss);
  L->bytes = off;
  L->p = p;
  L->nslab = nslab;
  L->slab_rows = slab_rows;
  L->spc = (int)spc;
  L->spl = (int)spl;
  L->ngroups = ngroups;
  return LO_OK;
}

}  // namespace
}  // namespace lo

extern "C" lo_status lo_tsqr_noalloc_scratch(int64_t n, int32_t s, int32_t chunk_rows, uint64_t* need_bytes,
                                             uint64_t* capacity_bytes) {
  using namespace lo;
  if (capacity_bytes) *capacity_bytes = kNoAllocScratchBytes;
  NoAllocLayout L;
  const lo_status st = noalloc_layout(n, s, chunk_rows, &L);
  if (st != LO_OK) return st;
  if (need_bytes) *need_bytes = L.bytes;
  return L.bytes > kNoAllocScratchBytes ? LO_ERR_CAPACITY : LO_OK;
}

extern "C" lo_status lo_tsqr_noalloc(int64_t n, int32_t s, int32_t chunk_rows, const double* W,
                                     int64_t ldw, double* U, double* R, void* cuda_stream) {
  using namespace lo;
  if (n < 1 || s < 1 || s > kMaxS || chunk_rows < 1 || !W || !U || !R || ldw < s) return LO_ERR_INVALID_ARG;
  if (U == W) {
    if (ldw != s) return LO_ERR_INVALID_ARG;  // in place only with a contiguous block
  } else {
    const double* wend = W + (n - 1) * ldw + s;  // distinct buffers must not overlap
    const double* uend = U + n * s;
    if (!(uend <= W || wend <= U)) return LO_ERR_INVALID_ARG;
  }
  // sizes first: a problem that does not fit is rejected before any CUDA call
  NoAllocLayout lay;
  lo_status st = noalloc_layout(n, s, chunk_rows, &lay);
  if (st != LO_OK) return st;
  if (lay.bytes > kNoAllocScratchBytes) return LO_ERR_CAPACITY;
  const int p = lay.p, nslab = lay.nslab;
  const GlobLayout GL = GlobLayout::make(s, s);
  const size_t ss = (size_t)s * s;

  // The device address of the scratch array in the current context, looked up
  // on every call (cheap next to the synchronization below): after a device
  // reset the module is loaded again, possibly at another address.
  void* base = nullptr;
  if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) {
    cudaGetLastError();
    return LO_ERR_CUDA;
  }
  unsigned char* sc = static_cast<unsigned char*>(base);
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  StepArgs a{};
  a.n = n;
  a.s = s;
  a.M = 1;
  a.p = p;
  a.nb = 0;
  a.Kmax = s;
  a.V = U;                    // the local panel of block 0 is the caller's U
  a.T = reinterpret_cast<double*>(sc + lay.o_T);
  a.tstride = (int64_t)ss;
  a.part = reinterpret_cast<double*>(sc + lay.o_part);
  a.small = reinterpret_cast<double*>(sc + lay.o_small);
  a.glob = reinterpret_cast<double*>(sc + lay.o_glob);
  a.tsum = reinterpret_cast<double*>(sc + lay.o_tsum);
  a.flags = reinterpret_cast<int*>(sc + lay.o_flags);
  a.slabs = reinterpret_cast<const SlabInfo*>(sc + lay.o_slabs);
  a.chunk_slab0 = reinterpret_cast<const int32_t*>(sc + lay.o_cs0);
  a.chunk_row0 = reinterpret_cast<const int64_t*>(sc + lay.o_cr0);
  a.nslab = nslab;
  a.slab_rows = lay.slab_rows;
  a.max_chunk_rows = (int)std::max<int64_t>(p > 1 ? chunk_rows : 0, n - (int64_t)(p - 1) * chunk_rows);
  a.precision = LO_PREC_FP64;
  a.leaf = LO_LEAF_PIP2;      // the library default (BCGS-PIP+, Alg. 8)
  a.reduction = 0;
  a.refine_tol = 1e-13;
  a.W = W;
  a.ldw = ldw;
  a.U = U;
  a.ldu = s;

  // the status word must start at zero; everything else is written before it is read
  cudaError_t e = cudaMemsetAsync(a.flags, 0, sizeof(int) * kFlagCount, stream);
  if (e == cudaSuccess) {
    int blocks = (nslab + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    k_noalloc_tables<<<blocks, 256, 0, stream>>>(n, chunk_rows, p, lay.slab_rows, lay.spc, lay.spl,
                                                  reinterpret_cast<SlabInfo*>(sc + lay.o_slabs),
                                                  reinterpret_cast<int32_t*>(sc + lay.o_cs0),
                                                  reinterpret_cast<int64_t*>(sc + lay.o_cr0));
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_step(a, stream, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(R, a.glob + GL.N_acc, sizeof(double) * ss, cudaMemcpyDeviceToDevice, stream);
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, a.flags, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LO_ERR_CUDA;
  }
  if (bits & (1 << LO_ERR_NONFINITE)) return LO_ERR_NONFINITE;
  if (bits & (1 << LO_ERR_BREAKDOWN)) return LO_ERR_BREAKDOWN;
  if (bits) return LO_ERR_CUDA;
  return LO_OK;
}

// Host side of the C ABI (include/lo.h): basis object, argument validation,
// staging of host buffers, kernel sequencing and status reporting.
#include <atomic>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "lo_internal.h"

using lo::GlobLayout;
using lo::SlabInfo;
using lo::SmallLayout;
using lo::StepArgs;

// Event-pair profiler for the kernel groups of one basis.
struct Profiler : lo::ProfHook {
  struct Pair {
    int kind;
    cudaEvent_t b, e;
  };
  bool enabled = false;
  std::vector<Pair> done;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open[lo::kKindCount] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t ev = pool.back();
      pool.pop_back();
      return ev;
    }
    cudaEvent_t ev = nullptr;
    cudaEventCreate(&ev);
    return ev;
  }
  void mark(int kind, bool begin, cudaStream_t st) override {
    if (!enabled) return;
    cudaEvent_t ev = get();
    cudaEventRecord(ev, st);
    if (begin) {
      open[kind] = ev;
    } else {
      done.push_back(Pair{kind, open[kind], ev});
      open[kind] = nullptr;
    }
  }
  // Sum of elapsed times (ms) and number of intervals per kind; recycles the events.
  cudaError_t collect(double* ms, long long* cnt) {
    for (int k = 0; k < lo::kKindCount; ++k) {
      ms[k] = 0.0;
      cnt[k] = 0;
    }
    cudaError_t err = cudaSuccess;
    for (auto& pr : done) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(pr.e);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pr.b, pr.e);
      if (e != cudaSuccess) err = e;
      ms[pr.kind] += t;
      cnt[pr.kind] += 1;
      pool.push_back(pr.b);
      pool.push_back(pr.e);
    }
    done.clear();
    return err;
  }
  ~Profiler() override {
    for (auto& pr : done) {
      cudaEventDestroy(pr.b);
      cudaEventDestroy(pr.e);
    }
    for (auto ev : pool) cudaEventDestroy(ev);
  }
};

struct lo_basis {
  uint64_t id = 0;  // process-unique, never reused (keys of the batched graph cache)
  int64_t n = 0;
  int s = 0, M = 0, cr = 0, p = 0, nb = 0, Kmax = 0;
  lo_options opt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  double* V = nullptr;
  double* T = nullptr;
  double* part = nullptr;
  double* small = nullptr;
  double* glob = nullptr;
  double* tsum = nullptr;
  int* flags = nullptr;
  int* tick = nullptr;     // ticket area of the persistent batched launch
  int* h_flags = nullptr;  // pinned
  SlabInfo* d_slabs = nullptr;
  int32_t* d_chunk_slab0 = nullptr;
  int64_t* d_chunk_row0 = nullptr;
  int nslab = 0, slab_rows = 0, ngroups = 0;
  int64_t tstride = 0;
  std::vector<int64_t> chunk_row0;
  // lazily allocated
  double* stage_in = nullptr;
  size_t stage_in_cap = 0;
  double* stage_out = nullptr;
  size_t stage_out_cap = 0;
  double* zq = nullptr;
  size_t zq_cap = 0;
  double* cdev = nullptr;
  size_t cdev_cap = 0;
  // tensor-core form
  double* hh_scratch = nullptr;  // Householder leaf over chunks larger than one tile
  int hh_T = 0, hh_stages = 0;
  int* colexp = nullptr;
  int* srcexp_slab = nullptr;
  int* srcexp = nullptr;
  int* coefexp = nullptr;
  uint32_t* coefdig = nullptr;
  int64_t coefdig_stride = 0;
  uint8_t* dig = nullptr;  // digit planes of the panels (null when off)
  int64_t dtiles = 0;
  lo::UmmaMaps maps{};
  Profiler prof;
};

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

lo_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LO_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LO_ERR_OOM : LO_ERR_CUDA;
}

lo_status status_from_bits(int bits) {
  // a wait that gave up leaves the step's later factors meaningless: report it first
  if (bits & (1 << LO_ERR_TIMEOUT)) return LO_ERR_TIMEOUT;
  if (bits & (1 << LO_ERR_NONFINITE)) return LO_ERR_NONFINITE;
  if (bits & (1 << LO_ERR_BREAKDOWN)) return LO_ERR_BREAKDOWN;
  if (bits) return LO_ERR_CUDA;
  return LO_OK;
}

void evict_basis_graphs(uint64_t id);

lo_status ensure(double** buf, size_t* cap, size_t need) {
  if (*cap >= need) return LO_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, need * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return LO_ERR_OOM;
  }
  *cap = need;
  return LO_OK;
}

StepArgs make_args(const lo_basis* b) {
  StepArgs a{};
  a.n = b->n;
  a.s = b->s;
  a.M = b->M;
  a.p = b->p;
  a.nb = b->nb;
  a.Kmax = b->Kmax;
  a.V = b->V;
  a.T = b->T;
  a.tstride = b->tstride;
  a.part = b->part;
  a.small = b->small;
  a.glob = b->glob;
  a.tsum = b->tsum;
  a.flags = b->flags;
  a.tree_ticket = b->tick + 4 * b->p + 3;  // the ticket area's last int (TickLayout)
  a.slabs = b->d_slabs;
  a.chunk_slab0 = b->d_chunk_slab0;
  a.chunk_row0 = b->d_chunk_row0;
  a.nslab = b->nslab;
  a.slab_rows = b->slab_rows;
  a.hh_T = b->hh_T;
  a.hh_stages = b->hh_stages;
  a.hh_scratch = b->hh_scratch;
  for (int c = 0; c < b->p; ++c)
    a.max_chunk_rows = std::max<int>(a.max_chunk_rows, (int)(b->chunk_row0[c + 1] - b->chunk_row0[c]));
  a.test_stall = b->opt.test_stall;
  a.precision = b->opt.precision;
  a.leaf = b->opt.leaf;
  a.reduction = b->opt.reduction;
  a.refine_tol = b->opt.refine_tol > 0 ? b->opt.refine_tol : 1e-13;
  a.deflation_tol = b->opt.deflation_tol;
  a.colexp = b->colexp;
  a.srcexp_slab = b->srcexp_slab;
  a.srcexp = b->srcexp;
  a.coefdig = b->coefdig;
  a.coefexp = b->coefexp;
  a.coefdig_stride = b->coefdig_stride;
  a.dig = b->dig;
  a.dtiles = b->dtiles;
  a.maps = &b->maps;
  return a;
}

// Read and clear the latched device status (synchronizes the stream).
lo_status read_status(lo_basis* b, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(b->h_flags, b->flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  const int bits = b->h_flags[0];
  if (bits) {
    cudaMemsetAsync(b->flags, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
  }
  return status_from_bits(bits);
}

// Enqueue one PQR step on `st` for device-resident W/U.  Does not touch nb.
lo_status enqueue_step(lo_basis* b, const double* W, int64_t ldw, double* U, int64_t ldu,
                       cudaStream_t st) {
  StepArgs a = make_args(b);
  a.W = W;
  a.ldw = ldw;
  a.U = U;
  a.ldu = ldu;
  return from_cuda(lo::launch_step(a, st, &b->prof));
}

lo_status copy_small_outputs(lo_basis* b, double* H, double* R, cudaStream_t st) {
  const GlobLayout GL = GlobLayout::make(b->Kmax, b->s);
  const size_t ks = (size_t)b->nb * b->s * b->s, ss = (size_t)b->s * b->s;
  cudaError_t e = cudaSuccess;
  if (H && ks) e = cudaMemcpyAsync(H, b->glob + GL.P_acc, ks * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess && R)
    e = cudaMemcpyAsync(R, b->glob + GL.N_acc, ss * sizeof(double), cudaMemcpyDefault, st);
  return from_cuda(e);
}

// Stream pool and graph cache of lo_orthogonalize_batched (one per process).
// A cached graph bakes in the device buffers of the bases it was captured
// for; its key names each basis by its process-unique id (never by address:
// a new basis may be created at a destroyed one's address), and
// lo_basis_destroy, or a reallocation of a staging buffer a graph may name,
// evicts every entry that names the basis.
constexpr int kPool = 8;
constexpr size_t kGraphCache = 8;
constexpr size_t kKeyHead = 3;    // count, stream, route mode
constexpr size_t kKeyPer = 9;     // words per instance; the basis id comes first
struct GraphEntry {
  std::vector<uintptr_t> key;
  cudaGraphExec_t exec;
  unsigned long long stamp;
  // the persistent launch's instance table, item prefix and counters (device)
  lo::BatchInst* d_insts;
  int* d_pref;
  int* d_counters;
  std::vector<char> persistent;  // per instance: run by the persistent launch
};
void free_entry(GraphEntry& ent) {
  cudaGraphExecDestroy(ent.exec);
  cudaFree(ent.d_insts);
  cudaFree(ent.d_pref);
  cudaFree(ent.d_counters);
}
struct BatchGraphs {
  std::mutex mu;
  int device = -1;
  cudaStream_t st[kPool] = {};
  cudaStream_t cap = nullptr;     // capture origin (the caller's stream may be the legacy one)
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kPool] = {};
  std::vector<GraphEntry> cache;
  unsigned long long clock = 0;
};
BatchGraphs& batch_graphs() {
  static BatchGraphs* g = new BatchGraphs();  // lives until process exit
  return *g;
}
bool key_names(const std::vector<uintptr_t>& key, uint64_t id) {
  for (size_t i = kKeyHead; i < key.size(); i += kKeyPer)
    if ((uint64_t)key[i] == id) return true;
  return false;
}
// Caller holds bg.mu.
void evict_locked(BatchGraphs& bg, uint64_t id) {
  for (size_t i = 0; i < bg.cache.size();) {
    if (key_names(bg.cache[i].key, id)) {
      free_entry(bg.cache[i]);
      bg.cache.erase(bg.cache.begin() + i);
    } else {
      ++i;
    }
  }
}
void evict_basis_graphs(uint64_t id) {
  BatchGraphs& bg = batch_graphs();
  std::lock_guard<std::mutex> lock(bg.mu);
  evict_locked(bg, id);
}
// The pool lives on one device; a switch tears down the old pool (on its own
// device) before creating the new one.
cudaError_t ensure_pool(BatchGraphs& bg, int device) {
  if (bg.device == device) return cudaSuccess;
  if (bg.device >= 0) {
    int cur = device;
    cudaSetDevice(bg.device);
    for (auto& ent : bg.cache) free_entry(ent);
    bg.cache.clear();
    for (int i = 0; i < kPool; ++i) {
      if (bg.st[i]) cudaStreamDestroy(bg.st[i]);
      if (bg.join[i]) cudaEventDestroy(bg.join[i]);
      bg.st[i] = nullptr;
      bg.join[i] = nullptr;
    }
    if (bg.fork) cudaEventDestroy(bg.fork);
    if (bg.cap) cudaStreamDestroy(bg.cap);
    bg.fork = nullptr;
    bg.cap = nullptr;
    bg.device = -1;
    cudaGetLastError();
    cudaSetDevice(cur);
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kPool && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&bg.st[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bg.join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bg.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bg.cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) bg.device = device;
  return e;
}

// Grow one of the basis's lazily allocated buffers; a move evicts the
// batched graphs of the basis (they may name the old buffer).
lo_status ensure_owned(lo_basis* b, double** buf, size_t* cap, size_t need) {
  if (*cap >= need) return LO_OK;
  evict_basis_graphs(b->id);
  return ensure(buf, cap, need);
}

std::atomic<uint64_t> g_next_basis_id{1};

// Route of the batched call's instances: 0 auto (the persistent launch for
// native float64 instances of at most kPersistentWork n (k + s), graph
// branches for the rest), 1 the persistent launch wherever it can run,
// 2 graph branches only.  Measured on GB300, 64 small steps (n = 4096, s = 4,
// k = 32): float64 bases 2.86 ms persistent against 4.19 ms in graph
// branches; tensor-core bases 2.88 ms persistent against 2.14 ms.
std::atomic<int> g_batch_route{0};
// Crossover of the auto route, in n (k + s): below it one persistent float64
// launch beats an instance's own kernel sequence (measured on GB300).
constexpr double kPersistentWork = 4.0e6;

}  // namespace

extern "C" {

void lo_options_default(lo_options* opt) {
  if (!opt) return;
  opt->precision = LO_PREC_FP64;
  opt->leaf = LO_LEAF_PIP2;
  opt->reduction = 0;
  opt->sync = 1;
  opt->refine_tol = 1e-13;
  opt->digit_planes = LO_PLANES_AUTO;
  opt->test_stall = 0;
  opt->deflation_tol = 0.0;
}

const char* lo_status_string(lo_status st) {
  switch (st) {
    case LO_OK: return "ok";
    case LO_ERR_INVALID_ARG: return "invalid argument";
    case LO_ERR_CAPACITY: return "basis is full (max_blocks reached)";
    case LO_ERR_CHUNK_TOO_SMALL: return "chunk has fewer rows than max_blocks*s";
    case LO_ERR_BREAKDOWN: return "Cholesky breakdown: block is numerically rank deficient";
    case LO_ERR_NONFINITE: return "non-finite value in a small factor";
    case LO_ERR_TIMEOUT: return "bounded device wait timed out";
    case LO_ERR_CUDA: return "CUDA runtime error";
    case LO_ERR_OOM: return "out of memory";
    case LO_ERR_UNSUPPORTED: return "unsupported option combination";
  }
  return "unknown status";
}

lo_status lo_basis_create(int64_t n, int32_t s, int32_t max_blocks, int32_t chunk_rows,
                          const lo_options* opt, void* cuda_stream, lo_basis** out) {
  if (!out) return LO_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || s < 1 || s > lo::kMaxS || max_blocks < 1 || chunk_rows < 1) return LO_ERR_INVALID_ARG;
  const int64_t Kmax = (int64_t)max_blocks * s;
  if (Kmax > lo::kMaxK || Kmax * s > lo::kMaxKS) return LO_ERR_INVALID_ARG;
  lo_options o;
  lo_options_default(&o);
  if (opt) o = *opt;
  if (o.precision < 0 || o.precision > 3 || o.leaf < 0 || o.leaf > 3 || o.reduction < 0 ||
      o.reduction > 2 || o.digit_planes < 0 || o.digit_planes > 1 || o.test_stall < 0 || o.test_stall > 2)
    return LO_ERR_INVALID_ARG;
  // A one-block basis (tall-skinny QR) of at most kNativeMaxS columns runs
  // the native float64 kernels in the tensor-core forms too: with no prior
  // columns its products (s / 4 flop per streamed byte) are too narrow for a
  // 128-row MMA tile to pay (measured at s = 1, 2, 4, n = 2^12 .. 2^22: native
  // float64 1.0 - 2.2x faster).  With prior blocks the tensor-core form wins
  // (n = 4096, s = 4, k = 32: 2.2x) and is kept.
  if (s <= lo::kNativeMaxS && max_blocks == 1) {
    if (o.precision == LO_PREC_FP64_TC) o.precision = LO_PREC_FP64;
    if (o.precision == LO_PREC_MIXED_TC) o.precision = LO_PREC_MIXED_FP32;
  }
  const bool tc = (o.precision == LO_PREC_FP64_TC || o.precision == LO_PREC_MIXED_TC);
  if (tc && !lo::oz_supported(s)) return LO_ERR_UNSUPPORTED;
  if (!(o.deflation_tol >= 0.0) || !std::isfinite(o.deflation_tol)) return LO_ERR_INVALID_ARG;
  if (o.deflation_tol > 0.0 && (o.precision == LO_PREC_MIXED_FP32 || o.precision == LO_PREC_MIXED_TC))
    return LO_ERR_UNSUPPORTED;
  if (o.refine_tol <= 0) o.refine_tol = 1e-13;
  const int64_t p64 = n / chunk_rows > 0 ? n / chunk_rows : 1;
  if (p64 > (1 << 30)) return LO_ERR_INVALID_ARG;
  const int p = (int)p64;
  const int64_t min_rows = (p == 1) ? n : chunk_rows;
  if (min_rows < Kmax) return LO_ERR_CHUNK_TOO_SMALL;

  lo_basis* b = new (std::nothrow) lo_basis();
  if (!b) return LO_ERR_OOM;
  b->id = g_next_basis_id.fetch_add(1);
  b->n = n;
  b->s = s;
  b->M = max_blocks;
  b->cr = chunk_rows;
  b->p = p;
  b->Kmax = (int)Kmax;
  b->opt = o;
  b->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&b->device);
  b->tstride = (int64_t)s * s * max_blocks * (max_blocks + 1) / 2;
  b->slab_rows = 16 * s > 256 ? 16 * s : 256;

  // chunks and slabs
  std::vector<SlabInfo> slabs;
  std::vector<int32_t> cs0;
  int64_t tiles = 0;
  b->chunk_row0.resize(p + 1);
  for (int c = 0; c < p; ++c) {
    const int64_t r0 = (int64_t)c * chunk_rows;
    const int64_t r1 = (c == p - 1) ? n : r0 + chunk_rows;
    b->chunk_row0[c] = r0;
    cs0.push_back((int32_t)slabs.size());
    for (int64_t r = r0; r < r1; r += b->slab_rows) {
      SlabInfo si;
      si.row0 = r;
      si.rows = (int32_t)((r1 - r) < b->slab_rows ? (r1 - r) : b->slab_rows);
      si.chunk = c;
      si.tile0 = (int32_t)tiles;
      si.pad_ = 0;
      tiles += (si.rows + 15) / 16;
      slabs.push_back(si);
    }
  }
  b->chunk_row0[p] = n;
  cs0.push_back((int32_t)slabs.size());
  b->nslab = (int)slabs.size();
  b->ngroups = (p + lo::kTreeGroup - 1) / lo::kTreeGroup;

  const SmallLayout SL = SmallLayout::make(b->Kmax, s);
  const GlobLayout GL = GlobLayout::make(b->Kmax, s);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
  };
  alloc((void**)&b->V, sizeof(double) * (size_t)n * Kmax);
  alloc((void**)&b->T, sizeof(double) * (size_t)p * b->tstride);
  alloc((void**)&b->part, sizeof(double) * (size_t)b->nslab * Kmax * s);
  alloc((void**)&b->small, sizeof(double) * (size_t)p * SL.stride);
  alloc((void**)&b->glob, sizeof(double) * (size_t)GL.stride);
  alloc((void**)&b->tsum, sizeof(double) * (size_t)b->ngroups * Kmax * s);
  alloc((void**)&b->flags, sizeof(int) * lo::kFlagCount);
  alloc((void**)&b->tick, sizeof(int) * lo::batch_tick_ints(p));
  if (o.leaf == LO_LEAF_HH) {
    // chunks larger than one tile are walked as sub-tiles (FlatTSPQR inside the chunk)
    int64_t maxrows = 0;
    for (int c = 0; c < p; ++c) maxrows = std::max<int64_t>(maxrows, b->chunk_row0[c + 1] - b->chunk_row0[c]);
    if (maxrows * s * (int64_t)sizeof(double) > lo::kHHTileBytes) {
      b->hh_T = lo::hh_subtile_rows(s);
      b->hh_stages = (int)((maxrows + b->hh_T - 1) / b->hh_T);
      alloc((void**)&b->hh_scratch, sizeof(double) * (size_t)p * b->hh_stages * (s * s + s));
    }
  }
  alloc((void**)&b->d_slabs, sizeof(SlabInfo) * slabs.size());
  alloc((void**)&b->d_chunk_slab0, sizeof(int32_t) * cs0.size());
  alloc((void**)&b->d_chunk_row0, sizeof(int64_t) * b->chunk_row0.size());
  if (tc) {
    b->coefdig_stride = lo::oz_coef_words(b->Kmax, 2 * s);
    if (lo::umma_coef_words(b->Kmax, s) > b->coefdig_stride) b->coefdig_stride = lo::umma_coef_words(b->Kmax, s);
    alloc((void**)&b->colexp, sizeof(int) * (size_t)Kmax * p);
    alloc((void**)&b->srcexp_slab, sizeof(int) * (size_t)b->nslab * 32);
    alloc((void**)&b->srcexp, sizeof(int) * (size_t)p * 32);
    alloc((void**)&b->coefexp, sizeof(int) * (size_t)p * 64);
    alloc((void**)&b->coefdig, sizeof(uint32_t) * (size_t)p * b->coefdig_stride);
    if (e == cudaSuccess) e = cudaMemset(b->colexp, 0, sizeof(int) * (size_t)Kmax * p);
    if (o.digit_planes == LO_PLANES_AUTO && lo::oz_planes_supported(s) && max_blocks > 1) {
      b->dtiles = tiles;
      const size_t dbytes = (size_t)max_blocks * (s / 8) * lo::kOzDigits * (size_t)tiles * 256;
      alloc((void**)&b->dig, dbytes);
      // planes not yet written must hold finite digits (they meet zero coefficients)
      if (e == cudaSuccess) e = cudaMemset(b->dig, 0, dbytes);
      if (e == cudaSuccess) e = lo::umma_make_maps(b->dig, s, max_blocks, tiles, &b->maps);
    }
  }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_flags, sizeof(int) * lo::kFlagCount);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_slabs, slabs.data(), sizeof(SlabInfo) * slabs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_chunk_slab0, cs0.data(), sizeof(int32_t) * cs0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_chunk_row0, b->chunk_row0.data(), sizeof(int64_t) * b->chunk_row0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->T, 0, sizeof(double) * (size_t)p * b->tstride);
  if (e == cudaSuccess) e = cudaMemset(b->flags, 0, sizeof(int) * lo::kFlagCount);
  if (e == cudaSuccess) e = cudaMemset(b->tick, 0, sizeof(int) * lo::batch_tick_ints(p));
  if (e == cudaSuccess) e = cudaMemset(b->glob, 0, sizeof(double) * (size_t)GL.stride);
  if (e != cudaSuccess) {
    lo_status st = from_cuda(e);
    lo_basis_destroy(b);
    return st;
  }
  *out = b;
  return LO_OK;
}

void lo_basis_destroy(lo_basis* b) {
  if (!b) return;
  // no cached batched graph may outlive the buffers it names
  evict_basis_graphs(b->id);
  cudaFree(b->V);
  cudaFree(b->T);
  cudaFree(b->part);
  cudaFree(b->small);
  cudaFree(b->glob);
  cudaFree(b->tsum);
  cudaFree(b->flags);
  cudaFree(b->tick);
  cudaFree(b->hh_scratch);
  cudaFree(b->d_slabs);
  cudaFree(b->d_chunk_slab0);
  cudaFree(b->d_chunk_row0);
  cudaFree(b->stage_in);
  cudaFree(b->stage_out);
  cudaFree(b->zq);
  cudaFree(b->cdev);
  cudaFree(b->colexp);
  cudaFree(b->srcexp_slab);
  cudaFree(b->srcexp);
  cudaFree(b->coefexp);
  cudaFree(b->coefdig);
  cudaFree(b->dig);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  cudaGetLastError();
  delete b;
}

lo_status lo_basis_reset(lo_basis* b) {
  if (!b) return LO_ERR_INVALID_ARG;
  b->nb = 0;
  return LO_OK;
}

int32_t lo_basis_num_blocks(const lo_basis* b) { return b ? b->nb : -1; }

int32_t lo_basis_num_chunks(const lo_basis* b) { return b ? b->p : -1; }

lo_status lo_basis_sync(lo_basis* b) {
  if (!b) return LO_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  return read_status(b, b->stream);
}

lo_status lo_orthogonalize(lo_basis* b, const double* W, int64_t ldw, double* U, int64_t ldu,
                           double* H, double* R) {
  if (!b || !W || !U || ldw < b->s || ldu < b->s) return LO_ERR_INVALID_ARG;
  if (b->nb >= b->M) return LO_ERR_CAPACITY;
  cudaSetDevice(b->device);
  cudaStream_t st = b->stream;
  const int s = b->s;
  const int64_t n = b->n;
  const bool w_dev = is_device_ptr(W), u_dev = is_device_ptr(U);
  const double* Wd = W;
  int64_t ldwd = ldw;
  double* Ud = U;
  int64_t ldud = ldu;
  lo_status rs;
  if (!w_dev) {
    if ((rs = ensure_owned(b, &b->stage_in, &b->stage_in_cap, (size_t)n * s)) != LO_OK) return rs;
    cudaError_t e = cudaMemcpy2DAsync(b->stage_in, s * sizeof(double), W, ldw * sizeof(double),
                                      s * sizeof(double), n, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return from_cuda(e);
    Wd = b->stage_in;
    ldwd = s;
  }
  if (!u_dev) {
    if ((rs = ensure_owned(b, &b->stage_out, &b->stage_out_cap, (size_t)n * s)) != LO_OK) return rs;
    Ud = b->stage_out;
    ldud = s;
  }
  if ((rs = enqueue_step(b, Wd, ldwd, Ud, ldud, st)) != LO_OK) return rs;
  if ((rs = copy_small_outputs(b, H, R, st)) != LO_OK) return rs;
  if (!u_dev) {
    cudaError_t e = cudaMemcpy2DAsync(U, ldu * sizeof(double), Ud, s * sizeof(double), s * sizeof(double), n,
                                      cudaMemcpyDefault, st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (b->opt.sync || !w_dev || !u_dev) {
    lo_status d = read_status(b, st);
    if (d != LO_OK) return d;
  }
  b->nb += 1;
  return LO_OK;
}

lo_status lo_orthogonalize_laplace5(lo_basis* b, int32_t nx, int32_t ny, const double* V, int64_t ldv, double* U,
                                    int64_t ldu, double* H, double* R) {
  if (!b || !V || !U || nx < 1 || ny < 1 || ldv < b->s || ldu < b->s) return LO_ERR_INVALID_ARG;
  if ((int64_t)nx * ny != b->n) return LO_ERR_INVALID_ARG;
  if (b->nb >= b->M) return LO_ERR_CAPACITY;
  cudaSetDevice(b->device);
  if (!is_device_ptr(V) || !is_device_ptr(U)) return LO_ERR_INVALID_ARG;
  {  // U is written while the stencil still reads neighbouring rows of V
    const double* vend = V + (b->n - 1) * ldv + b->s;
    const double* uend = U + (b->n - 1) * ldu + b->s;
    if (!(uend <= V || vend <= U)) return LO_ERR_INVALID_ARG;
  }
  cudaStream_t st = b->stream;
  StepArgs a = make_args(b);
  a.W = U;  // the block is formed into U; the step then reads it there
  a.ldw = ldu;
  a.U = U;
  a.ldu = ldu;
  a.op_nx = nx;
  a.op_ny = ny;
  a.op_V = V;
  a.op_ldv = ldv;
  lo_status rs = from_cuda(lo::launch_step(a, st, &b->prof));
  if (rs != LO_OK) return rs;
  if ((rs = copy_small_outputs(b, H, R, st)) != LO_OK) return rs;
  const bool host_small = (H && !is_device_ptr(H)) || (R && !is_device_ptr(R));
  if (b->opt.sync || host_small) {
    lo_status d = read_status(b, st);
    if (d != LO_OK) return d;
  }
  b->nb += 1;
  return LO_OK;
}

lo_status lo_orthogonalize_batched(lo_basis* const* bases, int32_t count, const double* const* W,
                                   const int64_t* ldw, double* const* U, const int64_t* ldu,
                                   double* const* H, double* const* R) {
  if (count < 0 || (count > 0 && (!bases || !W || !ldw || !U || !ldu))) return LO_ERR_INVALID_ARG;
  if (count == 0) return LO_OK;
  for (int j = 0; j < count; ++j) {
    lo_basis* b = bases[j];
    if (!b || !W[j] || !U[j] || ldw[j] < b->s || ldu[j] < b->s) return LO_ERR_INVALID_ARG;
    if (b->nb >= b->M) return LO_ERR_CAPACITY;
    if (b->device != bases[0]->device) return LO_ERR_INVALID_ARG;
    for (int i = 0; i < j; ++i)
      if (bases[i] == b) return LO_ERR_INVALID_ARG;  // one step per basis and call
  }
  cudaSetDevice(bases[0]->device);
  cudaStream_t cs = bases[0]->stream;
  // Host buffers (as in lo_orthogonalize): W is staged into the basis's device
  // buffer before the graph runs, U is written to a device buffer and copied
  // out after it, and host H, R are copied from the basis's small outputs
  // after it.  The graph itself only ever names device memory.
  std::vector<const double*> Wd(count);
  std::vector<int64_t> ldwd(count), ldud(count);
  std::vector<double*> Ud(count), Hd(count), Rd(count);
  std::vector<char> w_host(count), u_host(count), h_host(count), r_host(count);
  for (int j = 0; j < count; ++j) {
    lo_basis* b = bases[j];
    w_host[j] = !is_device_ptr(W[j]);
    u_host[j] = !is_device_ptr(U[j]);
    double* hj = H ? H[j] : nullptr;
    double* rj = R ? R[j] : nullptr;
    h_host[j] = hj && !is_device_ptr(hj);
    r_host[j] = rj && !is_device_ptr(rj);
    Hd[j] = h_host[j] ? nullptr : hj;
    Rd[j] = r_host[j] ? nullptr : rj;
    Wd[j] = W[j];
    ldwd[j] = ldw[j];
    Ud[j] = U[j];
    ldud[j] = ldu[j];
    lo_status rs;
    if (w_host[j]) {
      if ((rs = ensure_owned(b, &b->stage_in, &b->stage_in_cap, (size_t)b->n * b->s)) != LO_OK) return rs;
      Wd[j] = b->stage_in;
      ldwd[j] = b->s;
    }
    if (u_host[j]) {
      if ((rs = ensure_owned(b, &b->stage_out, &b->stage_out_cap, (size_t)b->n * b->s)) != LO_OK) return rs;
      Ud[j] = b->stage_out;
      ldud[j] = b->s;
    }
  }
  // the staging copies of host W run on the caller's stream before the graph
  for (int j = 0; j < count; ++j) {
    if (!w_host[j]) continue;
    lo_basis* b = bases[j];
    cudaError_t e = cudaMemcpy2DAsync(b->stage_in, b->s * sizeof(double), W[j], ldw[j] * sizeof(double),
                                      b->s * sizeof(double), b->n, cudaMemcpyDefault, cs);
    if (e != cudaSuccess) return from_cuda(e);
  }
  BatchGraphs& bg = batch_graphs();
  std::unique_lock<std::mutex> lock(bg.mu);
  cudaError_t e = ensure_pool(bg, bases[0]->device);
  if (e != cudaSuccess) return from_cuda(e);
  const int route = g_batch_route.load();
  // key: everything the captured work depends on; a basis by its id
  std::vector<uintptr_t> key;
  key.reserve(kKeyPer * (size_t)count + kKeyHead);
  key.push_back((uintptr_t)count);
  key.push_back((uintptr_t)cs);
  key.push_back((uintptr_t)route);
  for (int j = 0; j < count; ++j) {
    key.push_back((uintptr_t)bases[j]->id);
    key.push_back((uintptr_t)bases[j]->nb);
    key.push_back((uintptr_t)Wd[j]);
    key.push_back((uintptr_t)ldwd[j]);
    key.push_back((uintptr_t)Ud[j]);
    key.push_back((uintptr_t)ldud[j]);
    key.push_back((uintptr_t)Hd[j]);
    key.push_back((uintptr_t)Rd[j]);
    key.push_back((uintptr_t)bases[j]->h_flags);
  }
  GraphEntry* ent = nullptr;
  for (auto& en : bg.cache)
    if (en.key == key) {
      ent = &en;
      en.stamp = ++bg.clock;
    }
  if (!ent) {
    // the route of every instance: the persistent launch (device buffers only) or its own branch
    GraphEntry ne{key, nullptr, 0, nullptr, nullptr, nullptr, std::vector<char>(count, 0)};
    std::vector<lo::BatchInst> insts;
    std::vector<int> which;
    for (int j = 0; j < count && route != 2; ++j) {
      lo_basis* b = bases[j];
      if (w_host[j] || u_host[j] || h_host[j] || r_host[j]) continue;
      lo::BatchInst bi{};
      bi.a = make_args(b);
      bi.a.W = Wd[j];
      bi.a.ldw = ldwd[j];
      bi.a.U = Ud[j];
      bi.a.ldu = ldud[j];
      bi.tick = b->tick;
      bi.H = (b->nb > 0) ? Hd[j] : nullptr;
      bi.R = Rd[j];
      if (!lo::batch_fill(&bi)) continue;
      // auto: float64-form instances up to the crossover; a tensor-core
      // instance keeps its own branch (its tcgen05 kernels beat the float64
      // pipe the persistent launch runs on)
      if (route == 0 && (b->opt.precision != LO_PREC_FP64 ||
                         (double)b->n * (double)(b->nb * b->s + b->s) > kPersistentWork))
        continue;
      ne.persistent[j] = 1;
      insts.push_back(bi);
      which.push_back(j);
    }
    const int ni = (int)insts.size();
    size_t smem = 0;
    if (ni > 0) {
      // item prefix, phase-major: pass 1, pass 2, tree 1, tree 2, assembly, digit planes
      std::vector<int> pref(6 * (size_t)(ni + 1));
      int off = 0;
      for (int ph = 0; ph < 6; ++ph) {
        for (int q = 0; q < ni; ++q) {
          pref[ph * (ni + 1) + q] = off;
          const lo::StepArgs& a = insts[q].a;
          const int cnt = (ph == 2 || ph == 3) ? a.p : (ph == 5 ? (insts[q].digitize ? a.nslab : 0) : a.nslab);
          off += cnt;
        }
        pref[ph * (ni + 1) + ni] = off;
      }
      smem = lo::batch_smem(insts.data(), ni);
      if (cudaMalloc(&ne.d_insts, sizeof(lo::BatchInst) * ni) != cudaSuccess ||
          cudaMalloc(&ne.d_pref, sizeof(int) * pref.size()) != cudaSuccess ||
          cudaMalloc(&ne.d_counters, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ne.d_insts);
        cudaFree(ne.d_pref);
        cudaFree(ne.d_counters);
        return LO_ERR_OOM;
      }
      e = cudaMemcpy(ne.d_insts, insts.data(), sizeof(lo::BatchInst) * ni, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(ne.d_pref, pref.data(), sizeof(int) * pref.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(ne.d_insts);
        cudaFree(ne.d_pref);
        cudaFree(ne.d_counters);
        return from_cuda(e);
      }
    }
    // capture: fork onto the pool streams (the persistent launch on the first,
    // the other instances round-robin on the rest), join
    if ((e = lo::launch_prepare()) != cudaSuccess) {
      cudaFree(ne.d_insts);
      cudaFree(ne.d_pref);
      cudaFree(ne.d_counters);
      return from_cuda(e);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(bg.cap, cudaStreamCaptureModeThreadLocal);
    lo_status rs = from_cuda(e);
    if (rs == LO_OK) {
      cudaEventRecord(bg.fork, bg.cap);
      for (int i = 0; i < kPool; ++i) cudaStreamWaitEvent(bg.st[i], bg.fork, 0);
      if (ni > 0) {
        rs = from_cuda(lo::launch_batch(ne.d_insts, ni, ne.d_pref, ne.d_counters, smem, bg.st[0]));
        for (int q = 0; q < ni && rs == LO_OK; ++q) {
          lo_basis* b = bases[which[q]];
          rs = from_cuda(cudaMemcpyAsync(b->h_flags, b->flags, sizeof(int) * lo::kFlagCount,
                                         cudaMemcpyDeviceToHost, bg.st[0]));
        }
      }
      int rr = 0;
      for (int j = 0; j < count && rs == LO_OK; ++j) {
        if (ne.persistent[j]) continue;
        lo_basis* b = bases[j];
        cudaStream_t st = bg.st[ni > 0 ? 1 + (rr++ % (kPool - 1)) : (rr++ % kPool)];
        StepArgs a = make_args(b);
        a.W = Wd[j];
        a.ldw = ldwd[j];
        a.U = Ud[j];
        a.ldu = ldud[j];
        rs = from_cuda(lo::launch_step(a, st, nullptr));
        if (rs == LO_OK) rs = copy_small_outputs(b, Hd[j], Rd[j], st);
        if (rs == LO_OK)
          rs = from_cuda(cudaMemcpyAsync(b->h_flags, b->flags, sizeof(int) * lo::kFlagCount,
                                         cudaMemcpyDeviceToHost, st));
      }
      for (int i = 0; i < kPool; ++i) {
        cudaEventRecord(bg.join[i], bg.st[i]);
        cudaStreamWaitEvent(bg.cap, bg.join[i], 0);
      }
      e = cudaStreamEndCapture(bg.cap, &graph);
      if (rs == LO_OK) rs = from_cuda(e);
    }
    if (rs == LO_OK) {
      e = cudaGraphInstantiate(&ne.exec, graph, 0);
      rs = from_cuda(e);
    }
    if (graph) cudaGraphDestroy(graph);
    if (rs != LO_OK) {
      cudaFree(ne.d_insts);
      cudaFree(ne.d_pref);
      cudaFree(ne.d_counters);
      return rs;
    }
    if (bg.cache.size() >= kGraphCache) {
      size_t old = 0;
      for (size_t i = 1; i < bg.cache.size(); ++i)
        if (bg.cache[i].stamp < bg.cache[old].stamp) old = i;
      free_entry(bg.cache[old]);
      bg.cache.erase(bg.cache.begin() + old);
    }
    ne.stamp = ++bg.clock;
    bg.cache.push_back(std::move(ne));
    ent = &bg.cache.back();
  }
  const std::vector<char> persistent = ent->persistent;
  for (int j = 0; j < count; ++j)
    for (int f = 0; f < lo::kFlagCount; ++f) bases[j]->h_flags[f] = 0;
  e = cudaGraphLaunch(ent->exec, cs);
  lock.unlock();
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return from_cuda(e);
  // Instances of the persistent launch that asked for a third local pass or
  // reduction iteration (or the shifted retry) are redone on the regular
  // path; the launch left their block count alone.
  for (int j = 0; j < count; ++j) {
    if (!persistent[j]) continue;
    lo_basis* b = bases[j];
    const int* f = b->h_flags;
    const bool timeout = (f[0] & (1 << LO_ERR_TIMEOUT)) != 0;
    if (!timeout && (f[lo::kFlagPass + 2] || f[lo::kFlagTree + 2])) {
      cudaMemsetAsync(b->flags, 0, sizeof(int), cs);
      lo_status rs = enqueue_step(b, Wd[j], ldwd[j], Ud[j], ldud[j], cs);
      if (rs == LO_OK) rs = copy_small_outputs(b, Hd[j], Rd[j], cs);
      if (rs == LO_OK)
        rs = from_cuda(cudaMemcpyAsync(b->h_flags, b->flags, sizeof(int), cudaMemcpyDeviceToHost, cs));
      if (rs != LO_OK) return rs;
    }
  }
  // host outputs: after the graph, on the same stream
  for (int j = 0; j < count && e == cudaSuccess; ++j) {
    lo_basis* b = bases[j];
    if (u_host[j])
      e = cudaMemcpy2DAsync(U[j], ldu[j] * sizeof(double), b->stage_out, b->s * sizeof(double),
                            b->s * sizeof(double), b->n, cudaMemcpyDefault, cs);
    if (e == cudaSuccess && (h_host[j] || r_host[j])) {
      lo_status rs = copy_small_outputs(b, h_host[j] ? H[j] : nullptr, r_host[j] ? R[j] : nullptr, cs);
      if (rs != LO_OK) return rs;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return from_cuda(e);
  lo_status first = LO_OK;
  for (int j = 0; j < count; ++j) {
    lo_basis* b = bases[j];
    const int bits = b->h_flags[0];
    if (bits == 0) {
      b->nb += 1;
    } else {
      cudaMemset(b->flags, 0, sizeof(int));
      if (first == LO_OK) first = status_from_bits(bits);
    }
  }
  return first;
}

lo_status lo_set_batched_route(int32_t mode) {
  if (mode < 0 || mode > 2) return LO_ERR_INVALID_ARG;
  g_batch_route.store(mode);
  return LO_OK;
}

int32_t lo_batched_persistent_count(void) {
  BatchGraphs& bg = batch_graphs();
  std::lock_guard<std::mutex> lock(bg.mu);
  if (bg.cache.empty()) return 0;
  size_t last = 0;
  for (size_t i = 1; i < bg.cache.size(); ++i)
    if (bg.cache[i].stamp > bg.cache[last].stamp) last = i;
  int32_t c = 0;
  for (char v : bg.cache[last].persistent) c += v ? 1 : 0;
  return c;
}

uint64_t lo_basis_id(const lo_basis* b) { return b ? b->id : 0; }

int32_t lo_batched_cache_entries(uint64_t basis_id) {
  BatchGraphs& bg = batch_graphs();
  std::lock_guard<std::mutex> lock(bg.mu);
  if (basis_id == 0) return (int32_t)bg.cache.size();
  int32_t c = 0;
  for (auto& ent : bg.cache) c += key_names(ent.key, basis_id) ? 1 : 0;
  return c;
}

lo_status lo_basis_truncate(lo_basis* b, int32_t num_blocks) {
  if (!b || num_blocks < 0 || num_blocks > b->nb) return LO_ERR_INVALID_ARG;
  b->nb = num_blocks;
  return LO_OK;
}

lo_status lo_tune_chunk_rows(int64_t n, int32_t s, int32_t max_blocks, const lo_options* opt,
                             void* cuda_stream, int32_t* chunk_rows) {
  if (!chunk_rows || n < 1 || s < 1 || s > lo::kMaxS || max_blocks < 1) return LO_ERR_INVALID_ARG;
  *chunk_rows = 0;
  const int64_t Kmax = (int64_t)max_blocks * s;
  if (Kmax > lo::kMaxK || Kmax * s > lo::kMaxKS || n < Kmax) return LO_ERR_CHUNK_TOO_SMALL;
  lo_options o;
  lo_options_default(&o);
  if (opt) o = *opt;
  o.sync = 1;
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, int32_t> memo;
  const int nbucket = (int)std::floor(std::log2((double)n) * 4.0);
  const auto mkey = std::make_tuple(nbucket, (int)s, (int)max_blocks, (int)o.precision, (int)o.leaf);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find(mkey);
    if (it != memo.end()) {
      *chunk_rows = it->second;
      return LO_OK;
    }
  }
  // candidates: powers of two from max(Kmax, 256) up to n (and n itself for one chunk)
  std::vector<int64_t> cand;
  int64_t c0 = 256;
  while (c0 < Kmax) c0 *= 2;
  for (int64_t c = c0; c <= n && cand.size() < 9; c *= 2) cand.push_back(c);
  if (cand.empty()) cand.push_back(n);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* Wd = nullptr;
  double* Ud = nullptr;
  if (cudaMalloc(&Wd, sizeof(double) * (size_t)n * s) != cudaSuccess ||
      cudaMalloc(&Ud, sizeof(double) * (size_t)n * s) != cudaSuccess) {
    cudaFree(Wd);
    cudaGetLastError();
    return LO_ERR_OOM;
  }
  cudaError_t e = lo::launch_fill_pattern(Wd, n * s, st);
  const int kb = max_blocks > 1 ? max_blocks / 2 : 0;  // time the step at half capacity
  double best_t = 1e300;
  int64_t best = cand[0];
  for (int64_t c : cand) {
    if (e != cudaSuccess) break;
    lo_basis* b = nullptr;
    if (lo_basis_create(n, s, max_blocks, (int32_t)std::min<int64_t>(c, (int64_t)1 << 30), &o, cuda_stream, &b) != LO_OK)
      continue;
    bool ok = true;
    for (int j = 0; j < kb && ok; ++j) ok = lo_orthogonalize(b, Wd, s, Ud, s, nullptr, nullptr) == LO_OK &&
                                          lo::launch_fill_pattern(Wd, n * s, st) == cudaSuccess;
    double t = 1e300;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      b->nb = kb;
      cudaStreamSynchronize(st);
      const auto t0 = std::chrono::steady_clock::now();
      ok = lo_orthogonalize(b, Wd, s, Ud, s, nullptr, nullptr) == LO_OK;
      const auto t1 = std::chrono::steady_clock::now();
      t = std::min(t, std::chrono::duration<double>(t1 - t0).count());
    }
    lo_basis_destroy(b);
    if (ok && t < best_t) {
      best_t = t;
      best = c;
    }
  }
  cudaFree(Wd);
  cudaFree(Ud);
  if (e != cudaSuccess) return from_cuda(e);
  if (!(best_t < 1e300)) return LO_ERR_UNSUPPORTED;  // no candidate could run (e.g. Householder tiles too large)
  *chunk_rows = (int32_t)best;
  std::lock_guard<std::mutex> lock(mu);
  memo[mkey] = *chunk_rows;
  return LO_OK;
}

lo_status lo_tune_leaf(int64_t n, int32_t s, int32_t max_blocks, const lo_options* opt, void* cuda_stream,
                       int32_t* leaf, int32_t* chunk_rows) {
  if (!leaf || !chunk_rows) return LO_ERR_INVALID_ARG;
  *leaf = LO_LEAF_PIP2;
  *chunk_rows = 0;
  lo_options o;
  lo_options_default(&o);
  if (opt) o = *opt;
  o.sync = 1;
  // chunk rows per leaf (memoized by the chunk-size tuner)
  lo_options op = o, oh = o;
  op.leaf = LO_LEAF_PIP2;
  oh.leaf = LO_LEAF_HH;
  int32_t crp = 0, crh = 0;
  lo_status st = lo_tune_chunk_rows(n, s, max_blocks, &op, cuda_stream, &crp);
  if (st != LO_OK) return st;
  // a basis of several blocks keeps the chunk size its later steps want; the
  // leaf only changes its first step
  if (max_blocks > 1)
    crh = crp;
  else if (lo_tune_chunk_rows(n, s, max_blocks, &oh, cuda_stream, &crh) != LO_OK)
    crh = 0;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  double* Wd = nullptr;
  double* Ud = nullptr;
  if (cudaMalloc(&Wd, sizeof(double) * (size_t)n * s) != cudaSuccess ||
      cudaMalloc(&Ud, sizeof(double) * (size_t)n * s) != cudaSuccess) {
    cudaFree(Wd);
    cudaGetLastError();
    return LO_ERR_OOM;
  }
  cudaError_t e = lo::launch_fill_pattern(Wd, n * s, stream);
  // the first step (k = 0) with each leaf, best of three
  double best[2] = {1e300, 1e300};
  const lo_options* ops[2] = {&op, &oh};
  const int32_t crs[2] = {crp, crh};
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    if (crs[q] <= 0) continue;
    lo_basis* b = nullptr;
    if (lo_basis_create(n, s, max_blocks, crs[q], ops[q], cuda_stream, &b) != LO_OK) continue;
    for (int rep = 0; rep < 4; ++rep) {
      b->nb = 0;
      cudaStreamSynchronize(stream);
      const auto t0 = std::chrono::steady_clock::now();
      const bool ok = lo_orthogonalize(b, Wd, s, Ud, s, nullptr, nullptr) == LO_OK;
      const auto t1 = std::chrono::steady_clock::now();
      if (!ok) break;
      if (rep > 0) best[q] = std::min(best[q], std::chrono::duration<double>(t1 - t0).count());
    }
    lo_basis_destroy(b);
  }
  cudaFree(Wd);
  cudaFree(Ud);
  if (e != cudaSuccess) return from_cuda(e);
  const int q = (best[1] < best[0]) ? 1 : 0;
  *leaf = q ? LO_LEAF_HH : LO_LEAF_PIP2;
  *chunk_rows = crs[q];
  return LO_OK;
}

lo_status lo_apply_Q(lo_basis* b, const double* C, int32_t m, int64_t ldc, double* Y, int64_t ldy) {
  if (!b || !Y || m < 1 || m > lo::kMaxK || ldy < m) return LO_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  cudaStream_t st = b->stream;
  const int64_t n = b->n;
  const int k = b->nb * b->s;
  const bool y_dev = is_device_ptr(Y);
  lo_status rs;
  if (k == 0) {
    cudaError_t e = y_dev ? cudaMemset2DAsync(Y, ldy * sizeof(double), 0, m * sizeof(double), n, st)
                          : cudaSuccess;
    if (!y_dev)
      for (int64_t r = 0; r < n; ++r) memset(Y + r * ldy, 0, m * sizeof(double));
    return from_cuda(e);
  }
  if (!C || ldc < m) return LO_ERR_INVALID_ARG;
  const double* Cd = C;
  int64_t ldcd = ldc;
  if (!is_device_ptr(C)) {
    if ((rs = ensure_owned(b, &b->cdev, &b->cdev_cap, (size_t)k * m)) != LO_OK) return rs;
    cudaError_t e = cudaMemcpy2DAsync(b->cdev, m * sizeof(double), C, ldc * sizeof(double), m * sizeof(double), k,
                                      cudaMemcpyDefault, st);
    if (e != cudaSuccess) return from_cuda(e);
    Cd = b->cdev;
    ldcd = m;
  }
  if ((rs = ensure_owned(b, &b->zq, &b->zq_cap, (size_t)b->p * k * m)) != LO_OK) return rs;
  double* Yd = Y;
  int64_t ldyd = ldy;
  if (!y_dev) {
    if ((rs = ensure_owned(b, &b->stage_out, &b->stage_out_cap, (size_t)n * m)) != LO_OK) return rs;
    Yd = b->stage_out;
    ldyd = m;
  }
  StepArgs a = make_args(b);
  cudaError_t e = lo::launch_apply_q(a, Cd, m, ldcd, b->zq, Yd, ldyd, st, &b->prof);
  if (e != cudaSuccess) return from_cuda(e);
  if (!y_dev) {
    e = cudaMemcpy2DAsync(Y, ldy * sizeof(double), Yd, m * sizeof(double), m * sizeof(double), n, cudaMemcpyDefault,
                          st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (b->opt.sync || !y_dev) return read_status(b, st);  // the tensor-core form can latch a status
  return LO_OK;
}

lo_status lo_basis_export_chunk(lo_basis* b, int32_t chunk, double* Qi_host, double* Ti_host, int64_t* rows) {
  if (!b || chunk < 0 || chunk >= b->p) return LO_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  const int s = b->s, k = b->nb * s;
  const int64_t r0 = b->chunk_row0[chunk], r1 = b->chunk_row0[chunk + 1];
  if (rows) *rows = r1 - r0;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return from_cuda(e);
  if (Qi_host && k > 0) {
    for (int blk = 0; blk < b->nb && e == cudaSuccess; ++blk)
      e = cudaMemcpy2D(Qi_host + blk * s, k * sizeof(double), b->V + (size_t)blk * b->n * s + r0 * s,
                       s * sizeof(double), s * sizeof(double), r1 - r0, cudaMemcpyDeviceToHost);
  }
  if (Ti_host && k > 0 && e == cudaSuccess) {
    std::vector<double> tb((size_t)b->tstride);
    e = cudaMemcpy(tb.data(), b->T + (size_t)chunk * b->tstride, sizeof(double) * b->tstride, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      memset(Ti_host, 0, sizeof(double) * (size_t)k * k);
      for (int cb = 0; cb < b->nb; ++cb) {
        const double* blk = tb.data() + lo::tblock_offset(cb, s);
        for (int r = 0; r < (cb + 1) * s; ++r)
          for (int j = 0; j < s; ++j) Ti_host[(size_t)r * k + cb * s + j] = blk[r * s + j];
      }
    }
  }
  return from_cuda(e);
}

long long lo_launch_count(void) { return lo::launches(); }

lo_status lo_basis_last_rank(lo_basis* b, int32_t* rank) {
  if (!b || !rank) return LO_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  const GlobLayout GL = GlobLayout::make(b->Kmax, b->s);
  std::vector<double> N((size_t)b->s * b->s);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(N.data(), b->glob + GL.N_acc, sizeof(double) * N.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  int t = 0;
  for (int i = 0; i < b->s; ++i) t += N[(size_t)i * b->s + i] != 0.0 ? 1 : 0;
  *rank = t;
  return LO_OK;
}

lo_status lo_basis_last_step_info(lo_basis* b, int32_t* passes, int32_t* tree_iterations) {
  if (!b) return LO_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  int f[lo::kFlagCount];
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaMemcpy(f, b->flags, sizeof(f), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  int L = 0, Tn = 0;
  for (int t = 1; t <= lo::kMaxPass; ++t)
    if (f[lo::kFlagPass + t - 1]) L = t;
  for (int t = 1; t <= lo::kMaxTreeIter; ++t)
    if (f[lo::kFlagTree + t - 1]) Tn = t;
  if (passes) *passes = L;
  if (tree_iterations) *tree_iterations = Tn;
  return LO_OK;
}

lo_status lo_basis_set_profiling(lo_basis* b, int32_t enable) {
  if (!b) return LO_ERR_INVALID_ARG;
  b->prof.enabled = enable != 0;
  return LO_OK;
}

lo_status lo_basis_profile_read(lo_basis* b, double* ms, int64_t* intervals, int32_t nkinds) {
  if (!b || !ms || !intervals || nkinds < lo::kKindCount) return LO_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  long long cnt[lo::kKindCount];
  cudaError_t e = b->prof.collect(ms, cnt);
  for (int k = 0; k < lo::kKindCount; ++k) intervals[k] = cnt[k];
  return from_cuda(e);
}

lo_status lo_laplace5_apply(int32_t nx, int32_t ny, int32_t s, const double* X, int64_t ldx, double* Y,
                            int64_t ldy, void* cuda_stream) {
  if (nx < 1 || ny < 1 || s < 1 || !X || !Y || ldx < s || ldy < s) return LO_ERR_INVALID_ARG;
  return from_cuda(lo::launch_laplace5(nx, ny, s, X, ldx, Y, ldy, (cudaStream_t)cuda_stream));
}

}  // extern "C"

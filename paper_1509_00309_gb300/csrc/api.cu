// Host side of the C ABI declared in include/clr.h: contexts, matrices, the orchestration of
// one CLR product (plan -> dense x dense products -> low-rank products -> recompression) and
// the Newton–Schulz driver.  Every device step runs in this library's kernels; there is no
// CPU fallback.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "clr_internal.h"

using namespace clr;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t want) {
    if (want <= bytes && p) return cudaSuccess;
    if (p) {
      cudaFree(p);
      p = nullptr;
      bytes = 0;
    }
    size_t sz = std::max<size_t>(want, 256);
    cudaError_t e = cudaMalloc(&p, sz);
    if (e == cudaSuccess) bytes = sz;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

// Process-wide caching allocator for matrix storage.  Freed buffers are kept per (device, size)
// and handed to later allocations of the same size, so creating and freeing matrices in a loop
// (products, uploads, temporaries of the NS driver) costs no cudaMalloc / cudaFree after the
// first round.  At most kPoolCap bytes stay cached; clr_mem_trim releases a device's cache.
class DevicePool {
 public:
  cudaError_t alloc(int dev, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    {
      std::lock_guard<std::mutex> lock(mu_);
      auto it = free_.find({dev, bytes});
      if (it != free_.end() && !it->second.empty()) {
        *p = it->second.back();
        it->second.pop_back();
        cached_ -= bytes;
        return cudaSuccess;
      }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {  // give the cache back and retry once
      cudaGetLastError();
      trim(dev);
      e = cudaMalloc(p, bytes);
    }
    return e;
  }
  void release(int dev, void* p, size_t bytes) {
    if (!p) return;
    bytes = std::max<size_t>(bytes, 16);
    {
      std::lock_guard<std::mutex> lock(mu_);
      if (cached_ + bytes <= kPoolCap) {
        free_[{dev, bytes}].push_back(p);
        cached_ += bytes;
        return;
      }
    }
    cudaFree(p);
  }
  void trim(int dev) {
    std::vector<void*> drop;
    {
      std::lock_guard<std::mutex> lock(mu_);
      for (auto it = free_.begin(); it != free_.end();) {
        if (it->first.first == dev) {
          for (void* p : it->second) {
            drop.push_back(p);
            cached_ -= it->first.second;
          }
          it = free_.erase(it);
        } else {
          ++it;
        }
      }
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    for (void* p : drop) cudaFree(p);
    if (prev != dev) cudaSetDevice(prev);
  }
  size_t cached() {
    std::lock_guard<std::mutex> lock(mu_);
    return cached_;
  }

 private:
  static constexpr size_t kPoolCap = 64ull << 30;
  std::mutex mu_;
  std::map<std::pair<int, size_t>, std::vector<void*>> free_;
  size_t cached_ = 0;
};

DevicePool& pool() {
  static DevicePool* p = new DevicePool;  // never destroyed: matrices may outlive contexts
  return *p;
}

}  // namespace

// Device workspaces of one product in flight (grow-only).  Batched products captured into a
// graph run on several branches, each with its own set.
struct WorkSet {
  DevBuf plan_ints, triples, counters, ws, scratch, panels_a, panels_b, tile_flags, order;
  DevBuf oz_exps;  // row exponents of the exact-slice products (A rows, then B panel rows)
  DevBuf oz_recon; // the exact-slice staging's reconstructions of low-rank operand blocks
  // A's bf16 panels as staged for (matrix, terms, padded sizes): reused only while a caller
  // that guarantees A does not change (clr_multiply_host_stream) sets ctx->reuse_a
  DevBuf host_b, host_c, host_err;  // staging of the streamed host product (per pipeline slot)
  const void* staged_a = nullptr;
  const void* staged_buf = nullptr;  // panels_a's allocation the staging went to
  int staged_terms = 0;
  int64_t staged_m = 0, staged_k = 0;
  void release() {
    for (DevBuf* b : {&plan_ints, &triples, &counters, &ws, &scratch, &panels_a, &panels_b,
                      &tile_flags, &order, &oz_exps, &oz_recon, &host_b, &host_c, &host_err})
      b->release();
  }
};

// Tunable launch parameters of one product, chosen by the autotuner.
struct Tuning {
  int prec = CLR_PREC_FP64;
  int lr_mult = 2;     // CTAs per SM of the low-rank product and recompression kernels
  double eps = -1.0;   // truncation threshold of this product (< 0: the context's eps_lr)
  int recompress = -1; // dense-accumulated C tiles re-tested for low rank (< 0: the context's
                       // recompress_dense)
};

struct clr_ctx_s {
  int device = 0;
  clr_opts opts;
  int n_sm = 0;
  int cc_major = 0, cc_minor = 0;
  std::string err;
  void* encode_fn = nullptr;  // cuTensorMapEncodeTiled
  // workspaces (grow-only)
  std::vector<std::unique_ptr<WorkSet>> wsets;
  WorkSet* cur = nullptr;  // workspace set used by the next product
  DevBuf small, upload, jstats;  // jstats: SVD counters accumulated while profiling
  bool capturing = false;
  // autotuner cache: shape key -> tuning and measured ms
  std::map<std::string, std::pair<Tuning, double>> tune_cache;
  PlanCounters last_counters;
  // profiling: per-product phase events
  bool prof_on = false;
  struct ProfEvent {
    cudaEvent_t e;
    int phase;       // the phase that ENDS here
    cudaStream_t s;  // phases are timed between consecutive events of the same stream
  };
  std::vector<ProfEvent> prof_events;
  // NS runs its two independent products of an iteration concurrently on a side stream
  cudaStream_t side = nullptr;
  cudaStream_t up = nullptr;  // host-to-device uploads of the streamed host product
  cudaStream_t lay = nullptr;      // its layout of uploaded chunks into matrices
  cudaStream_t dn[2] = {nullptr, nullptr};   // its layouts and copies of C tiles to the host
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool reuse_a = false;  // split products may reuse A's staged panels (see WorkSet::staged_a)
  std::vector<cudaEvent_t> event_pool;
  clr_profile prof;
  // NS snapshot of one iteration: X, T, Y, Z (opts.ns_snapshot_iter)
  clr_mat_t snap[4] = {nullptr, nullptr, nullptr, nullptr};
};

struct clr_mat_s {
  int device = 0;
  int nr = 0, nc = 0;
  int64_t n_rows = 0, n_cols = 0;
  std::vector<int> row_sizes, col_sizes, row_off, col_off;
  int* d_row_off = nullptr;
  int* d_col_off = nullptr;
  int* d_row_idx = nullptr;  // cluster of every row
  int* d_col_idx = nullptr;  // cluster of every column
  int* d_kind = nullptr;
  int* d_rank = nullptr;
  double* d_norm = nullptr;
  double* d_pool = nullptr;
  unsigned int* d_cost = nullptr;
  MatView view() const {
    MatView v;
    v.nr = nr;
    v.nc = nc;
    v.n_rows = n_rows;
    v.n_cols = n_cols;
    v.row_off = d_row_off;
    v.col_off = d_col_off;
    v.kind = d_kind;
    v.rank = d_rank;
    v.norm = d_norm;
    v.pool = d_pool;
    v.cost = d_cost;
    return v;
  }
};

struct clr_batch_s;

struct clr_tape_s {
  double alpha = 0.0;
  int iters = 0;
  std::vector<int> sizes;                       // S's clusters (S itself is not kept: the
                                                // caller may free it before the backward)
  int prec = CLR_PREC_FP64;                     // precision of the adjoint products
  std::vector<clr_mat_t> y, z;                  // owned: Y_n, Z_n before update n
};

namespace {

int fail(clr_ctx_t ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(clr_ctx_t ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (ctx) ctx->err = m;
  return e == cudaErrorMemoryAllocation ? CLR_ENOMEM : CLR_ECUDA;
}

#define CLR_CUDA(call)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

#define CLR_CHECK_LAUNCH(where)                                  \
  do {                                                           \
    cudaError_t e_ = cudaGetLastError();                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);     \
  } while (0)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int check_sizes(clr_ctx_t ctx, int n, const int32_t* sizes, const char* what) {
  if (n <= 0 || !sizes) return fail(ctx, CLR_EINVAL, std::string(what) + ": no clusters");
  for (int i = 0; i < n; ++i)
    if (sizes[i] < 1 || sizes[i] > CLR_MAX_CLUSTER)
      return fail(ctx, CLR_EINVAL, std::string(what) + ": cluster size out of [1, 256]");
  return CLR_OK;
}

void free_mat(clr_mat_t m) {
  if (!m) return;
  const size_t nb = (size_t)m->nr * m->nc;
  DevicePool& pl = pool();
  pl.release(m->device, m->d_row_off, (m->nr + 1) * sizeof(int));
  pl.release(m->device, m->d_col_off, (m->nc + 1) * sizeof(int));
  pl.release(m->device, m->d_row_idx, (size_t)m->n_rows * sizeof(int));
  pl.release(m->device, m->d_col_idx, (size_t)m->n_cols * sizeof(int));
  pl.release(m->device, m->d_kind, nb * sizeof(int));
  pl.release(m->device, m->d_rank, nb * sizeof(int));
  pl.release(m->device, m->d_norm, nb * sizeof(double));
  pl.release(m->device, m->d_cost, nb * sizeof(unsigned int));
  pl.release(m->device, m->d_pool, (size_t)m->n_rows * m->n_cols * sizeof(double));
  delete m;
}

int alloc_mat(clr_ctx_t ctx, int nr, const int32_t* rs, int nc, const int32_t* cs,
              clr_mat_t* out) {
  int st = check_sizes(ctx, nr, rs, "row clusters");
  if (st) return st;
  st = check_sizes(ctx, nc, cs, "column clusters");
  if (st) return st;
  clr_mat_t m = new (std::nothrow) clr_mat_s;
  if (!m) return fail(ctx, CLR_ENOMEM, "host allocation");
  m->device = ctx->device;
  m->nr = nr;
  m->nc = nc;
  m->row_sizes.assign(rs, rs + nr);
  m->col_sizes.assign(cs, cs + nc);
  m->row_off.assign(nr + 1, 0);
  m->col_off.assign(nc + 1, 0);
  for (int i = 0; i < nr; ++i) m->row_off[i + 1] = m->row_off[i] + rs[i];
  for (int j = 0; j < nc; ++j) m->col_off[j + 1] = m->col_off[j] + cs[j];
  m->n_rows = m->row_off[nr];
  m->n_cols = m->col_off[nc];
  const size_t nb = (size_t)nr * nc;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = pool().alloc(ctx->device, p, b);
  };
  A((void**)&m->d_row_off, (nr + 1) * sizeof(int));
  A((void**)&m->d_col_off, (nc + 1) * sizeof(int));
  A((void**)&m->d_row_idx, (size_t)m->n_rows * sizeof(int));
  A((void**)&m->d_col_idx, (size_t)m->n_cols * sizeof(int));
  A((void**)&m->d_kind, nb * sizeof(int));
  A((void**)&m->d_rank, nb * sizeof(int));
  A((void**)&m->d_norm, nb * sizeof(double));
  A((void**)&m->d_cost, nb * sizeof(unsigned int));
  A((void**)&m->d_pool, (size_t)m->n_rows * m->n_cols * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_row_off, m->row_off.data(), (nr + 1) * sizeof(int),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_col_off, m->col_off.data(), (nc + 1) * sizeof(int),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    std::vector<int> ri(m->n_rows), ci(m->n_cols);
    for (int i = 0; i < nr; ++i)
      for (int r = m->row_off[i]; r < m->row_off[i + 1]; ++r) ri[r] = i;
    for (int j = 0; j < nc; ++j)
      for (int c = m->col_off[j]; c < m->col_off[j + 1]; ++c) ci[c] = j;
    e = cudaMemcpy(m->d_row_idx, ri.data(), ri.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(m->d_col_idx, ci.data(), ci.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(m->d_kind, 0, nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->d_rank, 0, nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->d_norm, 0, nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(m->d_cost, 0, nb * sizeof(unsigned int));
  if (e != cudaSuccess) {
    free_mat(m);
    return cuda_fail(ctx, e, "matrix allocation");
  }
  *out = m;
  return CLR_OK;
}

bool same_clusters(const std::vector<int>& a, const std::vector<int>& b) { return a == b; }

// Frees the matrices it holds when it goes out of scope, except those handed out by keep().
struct MatGuard {
  std::vector<clr_mat_t> v;
  ~MatGuard() {
    for (clr_mat_t m : v) free_mat(m);
  }
  clr_mat_t keep(clr_mat_t m) {
    v.erase(std::find(v.begin(), v.end(), m));
    return m;
  }
};


// The plan counters of a workspace set, zeroed (the sticky error flag included) when first
// allocated; plans clear only the fields before the flag.
int ensure_counters(clr_ctx_t ctx, WorkSet* w) {
  if (w->counters.p) return CLR_OK;
  CLR_CUDA(w->counters.ensure(sizeof(PlanCounters)));
  CLR_CUDA(cudaMemset(w->counters.p, 0, sizeof(PlanCounters)));
  return CLR_OK;
}

// Reads and clears the sticky device error flags of the context's workspace sets and of
// `extra` (kernels raise them on a bounded-wait timeout or on bad data).  The streams that used
// those sets must have been synchronised.
int take_device_error(clr_ctx_t ctx, const std::vector<std::unique_ptr<WorkSet>>* extra = nullptr) {
  int worst = 0;
  auto visit = [&](WorkSet* w) -> cudaError_t {
    if (!w->counters.p) return cudaSuccess;
    int* pe = &((PlanCounters*)w->counters.p)->err;
    int e = 0;
    cudaError_t ce = cudaMemcpy(&e, pe, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess && e) {
      ce = cudaMemset(pe, 0, sizeof(int));
      if (worst != 1) worst = e;
    }
    return ce;
  };
  for (auto& w : ctx->wsets) CLR_CUDA(visit(w.get()));
  if (extra)
    for (auto& w : *extra) CLR_CUDA(visit(w.get()));
  if (worst == 1) return fail(ctx, CLR_ETIMEOUT, "a device-side wait timed out");
  if (worst == 3) return fail(ctx, CLR_EINVAL, "non-finite data met on the device");
  if (worst) return fail(ctx, CLR_EINVAL, "device reported bad data (flag " + std::to_string(worst) + ")");
  return CLR_OK;
}

// Grow the context workspaces needed by a plan over nI x nJ tiles and nK inner clusters.
int make_plan(clr_ctx_t ctx, int nI, int nJ, int nK, Plan* p) {
  const size_t nt = (size_t)nI * nJ;
  CLR_CUDA(ctx->cur->plan_ints.ensure(11 * nt * sizeof(int)));
  const int64_t max_tr = (int64_t)nt * nK;
  CLR_CUDA(ctx->cur->triples.ensure((size_t)max_tr * sizeof(Triple)));
  int st = ensure_counters(ctx, ctx->cur);
  if (st) return st;
  int* base = (int*)ctx->cur->plan_ints.p;
  p->nI = nI;
  p->nJ = nJ;
  p->nK = nK;
  p->t_count = base;
  p->t_start = base + nt;
  p->t_route = base + 2 * nt;
  p->t_rsum = base + 3 * nt;
  p->l_dense = base + 4 * nt;
  p->l_lr = base + 5 * nt;
  p->l_qr = base + 6 * nt;
  p->l_dcomp = base + 7 * nt;
  p->l_qr_s = base + 8 * nt;
  p->l_dcomp_s = base + 9 * nt;
  p->l_dense_s = base + 10 * nt;
  p->row_off = nullptr;
  p->col_off = nullptr;
  p->c_cost = nullptr;
  p->triples = (Triple*)ctx->cur->triples.p;
  p->max_triples = max_tr;
  p->counters = (PlanCounters*)ctx->cur->counters.p;
  return CLR_OK;
}

int grid_of(clr_ctx_t ctx, int per_sm) { return std::max(1, ctx->n_sm * per_sm); }

// A side stream (and a second workspace set) ordered after `s`: work issued on ctx->side
// between fork_side and join_side runs concurrently with work issued on `s`.
int fork_side(clr_ctx_t ctx, cudaStream_t s) {
  if (ctx->wsets.size() < 2) ctx->wsets.emplace_back(new WorkSet);
  if (!ctx->side && cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess)
    return CLR_ECUDA;
  if (!ctx->ev_fork && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return CLR_ECUDA;
  if (!ctx->ev_join && cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return CLR_ECUDA;
  if (cudaEventRecord(ctx->ev_fork, s) != cudaSuccess ||
      cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0) != cudaSuccess)
    return CLR_ECUDA;
  return CLR_OK;
}

int join_side(clr_ctx_t ctx, cudaStream_t s) {
  if (cudaEventRecord(ctx->ev_join, ctx->side) != cudaSuccess ||
      cudaStreamWaitEvent(s, ctx->ev_join, 0) != cudaSuccess)
    return CLR_ECUDA;
  return CLR_OK;
}

// Device address of page-locked (pinned or registered) host memory, or null for pageable
// memory: kernels may then read or write it directly.
const double* host_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  return (const double*)at.devicePointer;
}


// SVD counters while profiling (not inside a graph capture), else null.  Three blocks of 8:
// [0, 8) for dense truncated SVDs (compress_dense_kernel), [8, 16) for the QR route
// (compress_qr_kernel), [16, 24) SM cycles and counts of compress_dense_kernel's paths.
constexpr int kJstatsBlock = 8;
// counter blocks: 0 compress_dense_kernel, 1 compress_qr_kernel, 2 per-path cycles of
// compress_dense_kernel, 3 its full-SVD stages, 4 its pre-reduced path's stages
constexpr int kJstatsBlocks = 5;
unsigned long long* jst(clr_ctx_t ctx, int block = 0) {
  return (ctx->prof_on && !ctx->capturing && ctx->jstats.p)
             ? (unsigned long long*)ctx->jstats.p + block * kJstatsBlock : nullptr;
}

enum { PH_START = -1, PH_PLAN = 0, PH_STAGE, PH_DENSE, PH_LOWRANK, PH_COMPRESS_QR, PH_COMPRESS,
       PH_FINALIZE };

void prof_mark(clr_ctx_t ctx, cudaStream_t s, int phase) {
  if (!ctx->prof_on || ctx->capturing) return;
  cudaEvent_t e;
  if (!ctx->event_pool.empty()) {
    e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return;
  }
  cudaEventRecord(e, s);
  ctx->prof_events.push_back({e, phase, s});
}

void prof_launches(clr_ctx_t ctx, int n) {
  if (ctx->prof_on && !ctx->capturing) ctx->prof.launches += n;
}

constexpr int64_t kScratchPerCta =
    (int64_t)(CLR_MAX_CLUSTER / 2) * (CLR_MAX_CLUSTER / 2) +
    (int64_t)CLR_MAX_CLUSTER * (CLR_MAX_CLUSTER / 2);
// Per-CTA scratch shared by the low-rank product kernel and (after it, on the same stream) the
// recompression kernels' mixed-precision SVD.
inline int64_t scratch_per_cta() {
  return kScratchPerCta > kSvdScratchPerCta ? kScratchPerCta : kSvdScratchPerCta;
}

int choose_precision(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, double eps_in = -1.0) {
  int prec = ctx->opts.precision;
  if (prec != CLR_PREC_AUTO) return prec;
  // A-priori statistical error model of the split products (relative RMS error of one
  // product term, including FP32 accumulation): bf16x3 ~ 2^-16.5, bf16x6 ~ 2^-23.  The
  // expected ||dC||_F is about u ||A||_F ||B||_F / sqrt(K); the product tolerance is
  // 10 eps ||A||_F ||B||_F.  Take the cheapest mode with a factor-4 margin.
  // The exact-slice products err by ~2^-48 relative to the rows' and columns' largest entries
  // (per K segment) per term; 2^-44 allows for the spread between those and the RMS entry.
  const double e0 = eps_in >= 0.0 ? eps_in : ctx->opts.eps_lr;
  const double eps = e0 > 0 ? e0 : 1e-8;
  const double sk = std::sqrt((double)a->n_cols);
  if (std::ldexp(1.0, -16) * 0.6 / sk * 4.0 <= 10.0 * eps) return CLR_PREC_BF16X3;
  if (std::ldexp(1.0, -23) / sk * 4.0 <= 10.0 * eps) return CLR_PREC_BF16X6;
  if (std::ldexp(1.0, -44) / sk * 4.0 <= 10.0 * eps) return CLR_PREC_OZAKI;
  (void)b;
  return CLR_PREC_FP64;
}

}  // namespace

// =============================================================================================
// Errors, options, contexts
// =============================================================================================
extern "C" const char* clr_strerror(int s) {
  switch (s) {
    case CLR_OK: return "ok";
    case CLR_EINVAL: return "invalid argument";
    case CLR_ENOMEM: return "out of device memory";
    case CLR_ENOCONV: return "Newton-Schulz did not converge";
    case CLR_ETIMEOUT: return "device-side wait timed out";
    case CLR_ECUDA: return "CUDA error";
    case CLR_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

extern "C" const char* clr_last_error(clr_ctx_t ctx) { return ctx ? ctx->err.c_str() : ""; }

extern "C" void clr_opts_default(clr_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps_lr = 1e-8;
  o->eps_sp = 0.0;
  o->precision = CLR_PREC_FP64;
  o->recompress_dense = 0;
  o->ns_max_iter = 50;
  o->ns_tol = 1e-6;
  o->ns_alpha = 0.0;
  o->ns_power_steps = 30;
  o->ns_fp64_tail = 0;
  o->ns_ladder_switch = 1e-3;
  o->jacobi_max_sweeps = 40;
}

extern "C" int clr_create(clr_ctx_t* out, int device, const clr_opts* opts) {
  if (!out) return CLR_EINVAL;
  *out = nullptr;
  clr_ctx_t ctx = new (std::nothrow) clr_ctx_s;
  if (!ctx) return CLR_ENOMEM;
  if (opts) ctx->opts = *opts; else clr_opts_default(&ctx->opts);
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    delete ctx;
    return CLR_ECUDA;
  }
  ctx->device = device;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_major, cudaDevAttrComputeCapabilityMajor, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
  if (e != cudaSuccess || ctx->cc_major != 10 || ctx->cc_minor != 3) {
    delete ctx;
    return CLR_ECUDA;
  }
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                       cudaEnableDefault, &q);
  if (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ctx->encode_fn = fn;
  std::memset(&ctx->last_counters, 0, sizeof(ctx->last_counters));
  ctx->wsets.emplace_back(new WorkSet);
  ctx->cur = ctx->wsets[0].get();
  *out = ctx;
  return CLR_OK;
}

extern "C" int clr_destroy(clr_ctx_t ctx) {
  if (!ctx) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  for (auto& pe : ctx->prof_events) cudaEventDestroy(pe.e);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->up) cudaStreamDestroy(ctx->up);
  if (ctx->lay) cudaStreamDestroy(ctx->lay);
  for (cudaStream_t d : ctx->dn)
    if (d) cudaStreamDestroy(d);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (auto& w : ctx->wsets) w->release();
  for (clr_mat_t& m : ctx->snap) {
    if (m) free_mat(m);
    m = nullptr;
  }
  ctx->small.release();
  ctx->upload.release();
  ctx->jstats.release();
  delete ctx;
  return CLR_OK;
}

extern "C" int clr_set_opts(clr_ctx_t ctx, const clr_opts* o) {
  if (!ctx || !o) return CLR_EINVAL;
  if (!(o->eps_lr >= 0.0) || !(o->eps_sp >= 0.0) || o->precision < 0 || o->precision > 4)
    return fail(ctx, CLR_EINVAL, "bad options");
  ctx->opts = *o;
  return CLR_OK;
}

extern "C" int clr_get_opts(clr_ctx_t ctx, clr_opts* o) {
  if (!ctx || !o) return CLR_EINVAL;
  *o = ctx->opts;
  return CLR_OK;
}

// =============================================================================================
// Matrices
// =============================================================================================
extern "C" int clr_mat_create(clr_ctx_t ctx, int n_rt, const int32_t* rs, int n_ct,
                              const int32_t* cs, clr_mat_t* out) {
  if (!ctx || !out) return CLR_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  return alloc_mat(ctx, n_rt, rs, n_ct, cs, out);
}

extern "C" int clr_mem_trim(clr_ctx_t ctx) {
  if (!ctx) return CLR_EINVAL;
  pool().trim(ctx->device);
  return CLR_OK;
}

extern "C" int64_t clr_mem_cached(void) { return (int64_t)pool().cached(); }

extern "C" int clr_mat_free(clr_ctx_t ctx, clr_mat_t m) {
  if (!m) return CLR_EINVAL;
  if (ctx) cudaSetDevice(ctx->device);
  free_mat(m);
  return CLR_OK;
}

extern "C" int clr_mat_shape(clr_mat_t m, int64_t* nrow, int64_t* ncol, int* nrt, int* nct) {
  if (!m) return CLR_EINVAL;
  if (nrow) *nrow = m->n_rows;
  if (ncol) *ncol = m->n_cols;
  if (nrt) *nrt = m->nr;
  if (nct) *nct = m->nc;
  return CLR_OK;
}

extern "C" int clr_mat_from_dense(clr_ctx_t ctx, const double* a, int64_t lda, int a_on_host,
                                  int n_rt, const int32_t* rs, int n_ct, const int32_t* cs,
                                  double eps_lr, double drop_norm, void* stream,
                                  clr_mat_t* out) {
  if (!ctx || !a || !out) return CLR_EINVAL;
  *out = nullptr;
  if (!(eps_lr >= 0.0) || !(drop_norm >= 0.0)) return fail(ctx, CLR_EINVAL, "bad thresholds");
  cudaSetDevice(ctx->device);
  clr_mat_t m = nullptr;
  int st = alloc_mat(ctx, n_rt, rs, n_ct, cs, &m);
  if (st) return st;
  if (lda < m->n_cols) {
    free_mat(m);
    return fail(ctx, CLR_EINVAL, "lda < n_cols");
  }
  cudaStream_t s = as_stream(stream);
  const double* src = a;
  DevBuf& staging = ctx->upload;
  // Page-locked host input read once (the dense path): the layout kernel reads it in place
  // through the host-device link (on Grace-Blackwell, NVLink-C2C), with no staging copy.  The
  // SVD path reads each block many times and stages it in device memory first.
  bool direct = false;
  if (a_on_host && eps_lr == 0.0) {
    const double* dp = host_device_ptr(a);
    if (dp) {
      src = dp;
      direct = true;
    }
  }
  if (a_on_host && !direct) {
    const size_t bytes = (size_t)m->n_rows * m->n_cols * sizeof(double);
    cudaError_t e = staging.ensure(bytes);
    if (e == cudaSuccess)
      e = lda == m->n_cols
              ? cudaMemcpyAsync(staging.p, a, bytes, cudaMemcpyHostToDevice, s)
              : cudaMemcpy2DAsync(staging.p, m->n_cols * sizeof(double), a,
                                  lda * sizeof(double), m->n_cols * sizeof(double), m->n_rows,
                                  cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      free_mat(m);
      return cuda_fail(ctx, e, "from_dense upload");
    }
    src = (const double*)staging.p;
    lda = m->n_cols;
  }
  cudaError_t e = ctx->cur->ws.ensure(2 * (size_t)m->n_rows * m->n_cols * sizeof(double));
  if (e == cudaSuccess)
    e = ctx->cur->scratch.ensure((size_t)grid_of(ctx, 2) * scratch_per_cta() * sizeof(double));
  if (e != cudaSuccess) {
    free_mat(m);
    return cuda_fail(ctx, e, "from_dense workspace");
  }
  st = ensure_counters(ctx, ctx->cur);
  if (st) {
    free_mat(m);
    return st;
  }
  PlanCounters* pc = (PlanCounters*)ctx->cur->counters.p;
  cudaMemsetAsync(pc, 0, kPlanCountersClear, s);
  if (eps_lr == 0.0) {
    // every kept block is dense: a coalesced layout copy, then norms decide what is dropped
    launch_rowmajor_to_pool(m->view(), m->d_row_idx, src, lda, s);
    launch_block_norms_dense(m->view(), s);
    launch_dense_kinds(m->view(), drop_norm, &pc->err, s);
  } else {
    // blocks visited largest first (SVD cost ~ m n min(m, n)), so the dynamic distribution
    // ends with the small ones
    std::vector<int> order(m->nr * m->nc);
    for (int t = 0; t < (int)order.size(); ++t) order[t] = t;
    auto cost = [&](int t) {
      const int64_t a = m->row_sizes[t / m->nc], b = m->col_sizes[t % m->nc];
      return a * b * std::min(a, b);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    e = ctx->cur->order.ensure(order.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->cur->order.p, order.data(), order.size() * sizeof(int),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      free_mat(m);
      return cuda_fail(ctx, e, "from_dense order");
    }
    launch_compress_dense(m->view(), nullptr, nullptr, (const int*)ctx->cur->order.p, src, lda,
                          (double*)ctx->cur->ws.p, (double*)ctx->cur->scratch.p,
                          eps_lr, drop_norm, 0, ctx->opts.build_rrqr ? 1 : 0,
                          ctx->opts.svd_no_prereduce ? 0 : 1,
                          ctx->opts.jacobi_max_sweeps, grid_of(ctx, 2), &pc->err, &pc->sched[2],
                          jst(ctx), s);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_mat(m);
    return cuda_fail(ctx, e, "from_dense");
  }
  st = take_device_error(ctx);  // 3: a block with non-finite values
  if (st) {
    free_mat(m);
    if (st == CLR_EINVAL) ctx->err = "non-finite input (or an earlier device error)";
    return st;
  }
  *out = m;
  return CLR_OK;
}

extern "C" int clr_mat_from_blocks(clr_ctx_t ctx, int n_rt, const int32_t* rs, int n_ct,
                                   const int32_t* cs, const int32_t* kinds,
                                   const int32_t* ranks, const double* pool_host, void* stream,
                                   clr_mat_t* out) {
  if (!ctx || !kinds || !ranks || !pool_host || !out) return CLR_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  // validate kinds and ranks on the host
  for (int I = 0; I < n_rt; ++I)
    for (int J = 0; J < n_ct; ++J) {
      const int k = kinds[I * n_ct + J], r = ranks[I * n_ct + J];
      const int lim = std::min(rs[I], cs[J]) / 2;
      if (k < 0 || k > 2) return fail(ctx, CLR_EINVAL, "bad block kind");
      if (k == CLR_KIND_LR && (r < 1 || r > lim))
        return fail(ctx, CLR_EINVAL, "low-rank block rank out of [1, floor(min(m,n)/2)]");
    }
  clr_mat_t m = nullptr;
  int st = alloc_mat(ctx, n_rt, rs, n_ct, cs, &m);
  if (st) return st;
  std::vector<int> rk(ranks, ranks + (size_t)n_rt * n_ct);
  for (int I = 0; I < n_rt; ++I)
    for (int J = 0; J < n_ct; ++J) {
      const int b = I * n_ct + J;
      if (kinds[b] == CLR_KIND_DENSE) rk[b] = std::min(rs[I], cs[J]);
      if (kinds[b] == CLR_KIND_ZERO) rk[b] = 0;
    }
  cudaStream_t s = as_stream(stream);
  const size_t nb = (size_t)n_rt * n_ct;
  cudaError_t e = cudaMemcpyAsync(m->d_kind, kinds, nb * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->d_rank, rk.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->d_pool, pool_host, (size_t)m->n_rows * m->n_cols * sizeof(double),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    launch_block_norms(m->view(), s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_mat(m);
    return cuda_fail(ctx, e, "from_blocks");
  }
  *out = m;
  return CLR_OK;
}

extern "C" int clr_mat_to_dense(clr_ctx_t ctx, clr_mat_t m, double* out, int64_t ldo,
                                int out_on_host, void* stream) {
  if (!ctx || !m || !out) return CLR_EINVAL;
  if (ldo < m->n_cols) return fail(ctx, CLR_EINVAL, "ldo < n_cols");
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  if (!out_on_host) {
    launch_pool_to_rowmajor(m->view(), m->d_row_idx, m->d_col_idx, out, ldo, s);
    CLR_CHECK_LAUNCH("to_dense");
    return CLR_OK;
  }
  if (double* dp = const_cast<double*>(host_device_ptr(out))) {
    // page-locked output: written in place through the host-device link
    launch_pool_to_rowmajor(m->view(), m->d_row_idx, m->d_col_idx, dp, ldo, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "to_dense");
    return CLR_OK;
  }
  DevBuf& tmp = ctx->upload;
  const size_t bytes = (size_t)m->n_rows * m->n_cols * sizeof(double);
  cudaError_t e = tmp.ensure(bytes);
  if (e == cudaSuccess) {
    launch_pool_to_rowmajor(m->view(), m->d_row_idx, m->d_col_idx, (double*)tmp.p, m->n_cols, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = ldo == m->n_cols
            ? cudaMemcpyAsync(out, tmp.p, bytes, cudaMemcpyDeviceToHost, s)
            : cudaMemcpy2DAsync(out, ldo * sizeof(double), tmp.p, m->n_cols * sizeof(double),
                                m->n_cols * sizeof(double), m->n_rows, cudaMemcpyDeviceToHost,
                                s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "to_dense");
  return CLR_OK;
}

extern "C" int clr_mat_get_blocks(clr_ctx_t ctx, clr_mat_t m, int32_t* kinds, int32_t* ranks,
                                  double* norms, double* pool_host, void* stream) {
  if (!ctx || !m) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  const size_t nb = (size_t)m->nr * m->nc;
  if (kinds) CLR_CUDA(cudaMemcpyAsync(kinds, m->d_kind, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (ranks) CLR_CUDA(cudaMemcpyAsync(ranks, m->d_rank, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (norms) CLR_CUDA(cudaMemcpyAsync(norms, m->d_norm, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (pool_host)
    CLR_CUDA(cudaMemcpyAsync(pool_host, m->d_pool, (size_t)m->n_rows * m->n_cols * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
  CLR_CUDA(cudaStreamSynchronize(s));
  return CLR_OK;
}

extern "C" int clr_mat_info(clr_ctx_t ctx, clr_mat_t m, clr_info* info, void* stream) {
  if (!ctx || !m || !info) return CLR_EINVAL;
  const size_t nb = (size_t)m->nr * m->nc;
  std::vector<int> kinds(nb), ranks(nb);
  std::vector<double> norms(nb);
  int st = clr_mat_get_blocks(ctx, m, kinds.data(), ranks.data(), norms.data(), nullptr, stream);
  if (st) return st;
  std::memset(info, 0, sizeof(*info));
  info->n_rows = m->n_rows;
  info->n_cols = m->n_cols;
  info->n_row_clusters = m->nr;
  info->n_col_clusters = m->nc;
  double fro = 0.0;
  const int nbins = CLR_MAX_CLUSTER / 2 + 2;
  for (int I = 0; I < m->nr; ++I)
    for (int J = 0; J < m->nc; ++J) {
      const size_t b = (size_t)I * m->nc + J;
      const int k = kinds[b];
      if (k < 0 || k > 2) return fail(ctx, CLR_ECUDA, "corrupt block kind");
      info->n_blocks[k]++;
      fro += norms[b] * norms[b];
      if (k == CLR_KIND_LR) {
        info->max_rank = std::max(info->max_rank, ranks[b]);
        info->sum_rank += ranks[b];
        info->stored_doubles += (int64_t)(m->row_sizes[I] + m->col_sizes[J]) * ranks[b];
        info->rank_hist[std::min(ranks[b], nbins - 2)]++;
      } else if (k == CLR_KIND_DENSE) {
        info->stored_doubles += (int64_t)m->row_sizes[I] * m->col_sizes[J];
        info->rank_hist[nbins - 1]++;
      } else {
        info->rank_hist[0]++;
      }
    }
  info->frob_norm = std::sqrt(fro);
  return CLR_OK;
}

extern "C" int clr_mat_copy(clr_ctx_t ctx, clr_mat_t src, clr_mat_t dst, void* stream) {
  if (!ctx || !src || !dst) return CLR_EINVAL;
  if (src->row_sizes != dst->row_sizes || src->col_sizes != dst->col_sizes)
    return fail(ctx, CLR_EINVAL, "copy: clusters differ");
  if (src == dst) return CLR_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  const size_t nb = (size_t)src->nr * src->nc;
  CLR_CUDA(cudaMemcpyAsync(dst->d_kind, src->d_kind, nb * sizeof(int), cudaMemcpyDeviceToDevice, s));
  CLR_CUDA(cudaMemcpyAsync(dst->d_rank, src->d_rank, nb * sizeof(int), cudaMemcpyDeviceToDevice, s));
  CLR_CUDA(cudaMemcpyAsync(dst->d_norm, src->d_norm, nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CLR_CUDA(cudaMemcpyAsync(dst->d_pool, src->d_pool, (size_t)src->n_rows * src->n_cols * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
  return CLR_OK;
}

extern "C" int clr_mat_transpose(clr_ctx_t ctx, clr_mat_t src, clr_mat_t* out, void* stream) {
  if (!ctx || !src || !out) return CLR_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  clr_mat_t t = nullptr;
  int st = alloc_mat(ctx, src->nc, src->col_sizes.data(), src->nr, src->row_sizes.data(), &t);
  if (st) return st;
  launch_transpose(src->view(), t->view(), as_stream(stream));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_mat(t);
    return cuda_fail(ctx, e, "transpose");
  }
  *out = t;
  return CLR_OK;
}

extern "C" int clr_matvec(clr_ctx_t ctx, clr_mat_t a, const double* x, double* y, void* stream) {
  if (!ctx || !a || !x || !y) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  launch_matvec(a->view(), x, y, as_stream(stream));
  CLR_CHECK_LAUNCH("matvec");
  return CLR_OK;
}

// =============================================================================================
// The product
// =============================================================================================
namespace {

// *fused_norms: set when the dense kernel's epilogue formed the sums of squares of the
// route-DENSE tiles (then only their square roots remain to be taken).
int run_split_dd(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c, const Plan& p, int prec,
                 bool recompress_dense, cudaStream_t s, bool* fused_norms) {
  const int terms = prec == CLR_PREC_BF16X3 ? 2 : 3;
  const int64_t M_pad = (c->n_rows + 127) / 128 * 128;
  const int64_t N_pad = (c->n_cols + 255) / 256 * 256;
  const int64_t K_pad = (a->n_cols + 127) / 128 * 128;  // staging tiles are 128 wide
  CLR_CUDA(ctx->cur->panels_a.ensure((size_t)terms * M_pad * K_pad * 2));
  CLR_CUDA(ctx->cur->panels_b.ensure((size_t)terms * N_pad * K_pad * 2));
  CLR_CUDA(ctx->cur->tile_flags.ensure((size_t)(M_pad / 128) * (N_pad / 256)));
  MatView av = a->view(), bv = b->view(), cv = c->view();
  const int* idx_m = c->d_row_idx;
  const int* idx_n = c->d_col_idx;
  const int* idx_k = a->d_col_idx;
  WorkSet* w = ctx->cur;
  const bool reuse = ctx->reuse_a && w->staged_a == (const void*)a && w->staged_terms == terms &&
                     w->staged_m == M_pad && w->staged_k == K_pad &&
                     w->staged_buf == (const void*)w->panels_a.p;
  if (!reuse) {
    launch_split_stage(av, idx_m, idx_k, w->panels_a.p, terms, M_pad, K_pad, 1, s);
    w->staged_a = ctx->reuse_a ? (const void*)a : nullptr;
    w->staged_buf = w->panels_a.p;
    w->staged_terms = terms;
    w->staged_m = M_pad;
    w->staged_k = K_pad;
  }
  launch_split_stage(bv, idx_k, idx_n, w->panels_b.p, terms, N_pad, K_pad, 0, s);
  CLR_CHECK_LAUNCH("split staging");
  prof_launches(ctx, reuse ? 2 : 4);  // dense and low-rank passes per staged operand
  prof_mark(ctx, s, PH_STAGE);
  SplitGemmArgs g;
  g.A = &av;
  g.B = &bv;
  g.C = &cv;
  g.p = &p;
  g.terms = terms;
  g.a_panels = ctx->cur->panels_a.p;
  g.b_panels = ctx->cur->panels_b.p;
  g.M_pad = M_pad;
  g.N_pad = N_pad;
  g.K_pad = K_pad;
  g.row_tile_of = idx_m;
  g.col_tile_of = idx_n;
  g.tile_active = (unsigned char*)ctx->cur->tile_flags.p;
  g.n_sm = ctx->n_sm;
  g.err = &p.counters->err;
  g.encode_fn = ctx->encode_fn;
  g.wait_ns = ctx->opts.wait_timeout_us > 0 ? 1000ull * (unsigned long long)ctx->opts.wait_timeout_us
                                            : 2000000000ull;
  // norms in the epilogue when the dense tiles are final (not re-tested) and the clusters are
  // wide enough for its per-warp grouping
  const bool fuse = !recompress_dense &&
                    *std::min_element(c->row_sizes.begin(), c->row_sizes.end()) >= 32 &&
                    *std::min_element(c->col_sizes.begin(), c->col_sizes.end()) >= 16;
  g.norm_sq = fuse ? c->d_norm : nullptr;
  *fused_norms = fuse;
  std::string why;
  int st = split_gemm_dd(g, s, &why);
  if (st) return fail(ctx, st, "split GEMM: " + why);
  CLR_CHECK_LAUNCH("split GEMM");
  prof_launches(ctx, 2);  // tile flags + GEMM
  if (ctx->prof_on) {
    ctx->prof.dense_launches++;
    // tensor flops issued: every active 128 x 256 tile runs the full K for each term pair;
    // counted exactly for all-dense operands, an upper bound otherwise
    const double pairs = terms == 2 ? 3.0 : 6.0;
    ctx->prof.dense_tensor_flops += 2.0 * pairs * (double)c->n_rows * (double)c->n_cols *
                                    (double)K_pad;
  }
  prof_mark(ctx, s, PH_DENSE);
  return CLR_OK;
}

// Dense x dense products by exact slices on the tensor cores (CLR_PREC_OZAKI): the dense blocks
// of A and B are staged as 7 bf16 digit planes with per-row exponents, and the exact-slice GEMM
// writes the route-DENSE tiles; low-rank contributions follow in FP64 (low-rank kernel).
// Exact slices, before the plan: digit panels of A and B (dense blocks and reconstructed
// low-rank blocks) with their exponents per K segment, and the routing rule of densely
// accumulated low-rank sums.  Such a sum goes to the tensor-core GEMM when the expected error of
// its sliced evaluation -- about 1.2 2^-48 per term of a segment relative to 2^(e_i + f_j)
// (truncation of both operands and the dropped slice pairs, rounding independently), i.e.
// 1.2 2^-48 sqrt(K_seg sum_s sa[I][s] sb[J][s]) over the tile -- is, times 4, within eps/16.
int stage_ozaki(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c, double eps_lr,
                cudaStream_t s, OzDaccRule* rule) {
  const int64_t M_pad = (c->n_rows + 127) / 128 * 128;
  const int64_t N_pad = (c->n_cols + 63) / 64 * 64;
  const int64_t K_pad = (a->n_cols + 127) / 128 * 128;
  const int n_seg = (int)((K_pad + kOzakiSegK - 1) / kOzakiSegK);
  WorkSet* w = ctx->cur;
  CLR_CUDA(w->panels_a.ensure((size_t)kOzakiSlices * M_pad * K_pad * 2));
  CLR_CUDA(w->panels_b.ensure((size_t)kOzakiSlices * N_pad * K_pad * 2));
  const size_t exp_bytes = ((size_t)n_seg * (M_pad + N_pad) * sizeof(int) + 255) / 256 * 256;
  CLR_CUDA(w->oz_exps.ensure(exp_bytes + (size_t)n_seg * (c->nr + c->nc) * sizeof(double)));
  w->staged_a = nullptr;   // the panels no longer hold a split staging
  MatView av = a->view(), bv = b->view();
  int* ea = (int*)w->oz_exps.p;
  int* eb = ea + (size_t)n_seg * M_pad;
  double* sa = (double*)((char*)w->oz_exps.p + exp_bytes);
  double* sb = sa + (size_t)n_seg * c->nr;
  // one reconstruction image, used by A's staging and then (stream-ordered) by B's
  CLR_CUDA(w->oz_recon.ensure((size_t)std::max(a->n_rows * a->n_cols, b->n_rows * b->n_cols) *
                              sizeof(double)));
  double* recon = (double*)w->oz_recon.p;
  launch_ozaki_stage(av, c->d_row_idx, a->d_col_idx, w->panels_a.p, ea, recon, M_pad, K_pad, 1,
                     s);
  launch_ozaki_stage(bv, a->d_col_idx, c->d_col_idx, w->panels_b.p, eb, recon, N_pad, K_pad, 0,
                     s);
  launch_ozaki_scale_sums(ea, M_pad, c->d_row_off, c->nr, n_seg, sa, s);
  launch_ozaki_scale_sums(eb, N_pad, c->d_col_off, c->nc, n_seg, sb, s);
  CLR_CHECK_LAUNCH("exact-slice staging");
  prof_launches(ctx, 12);  // per operand: reconstruction, 2 exponent, 2 digit kernels; 2 sums
  prof_mark(ctx, s, PH_STAGE);
  const double u = 4.0 * 1.2 * std::ldexp(1.0, -48);
  const double budget = eps_lr / 16.0;
  rule->sa = sa;
  rule->sb = sb;
  rule->n_seg = n_seg;
  rule->bound2 = budget * budget / (u * u * (double)kOzakiSegK);
  return CLR_OK;
}

// Exact slices, after the plan: the GEMM over the tiles of route-DENSE and DACC_G C tiles.
int run_ozaki_gemm(clr_ctx_t ctx, clr_mat_t a, clr_mat_t c, const Plan& p, cudaStream_t s) {
  const int64_t M_pad = (c->n_rows + 127) / 128 * 128;
  const int64_t N_pad = (c->n_cols + 63) / 64 * 64;
  const int64_t K_pad = (a->n_cols + 127) / 128 * 128;
  const int n_seg = (int)((K_pad + kOzakiSegK - 1) / kOzakiSegK);
  WorkSet* w = ctx->cur;
  const size_t n_gemm_tiles = (size_t)(M_pad / 128) * (N_pad / kOzakiTileN);
  const size_t flag_bytes = (n_gemm_tiles + 15) / 16 * 16;
  CLR_CUDA(w->tile_flags.ensure(flag_bytes + (n_gemm_tiles + 1) * sizeof(int)));
  MatView cv = c->view();
  int* ea = (int*)w->oz_exps.p;
  OzakiGemmArgs g;
  g.C = &cv;
  g.p = &p;
  g.a_panels = w->panels_a.p;
  g.b_panels = w->panels_b.p;
  g.ea = ea;
  g.eb = ea + (size_t)n_seg * M_pad;
  g.M_pad = M_pad;
  g.N_pad = N_pad;
  g.K_pad = K_pad;
  g.row_tile_of = c->d_row_idx;
  g.col_tile_of = c->d_col_idx;
  g.tile_active = (unsigned char*)w->tile_flags.p;
  g.active_list = (int*)((char*)w->tile_flags.p + flag_bytes);
  g.n_sm = ctx->n_sm;
  g.err = &p.counters->err;
  g.wait_ns = ctx->opts.wait_timeout_us > 0
                  ? 1000ull * (unsigned long long)ctx->opts.wait_timeout_us : 2000000000ull;
  g.encode_fn = ctx->encode_fn;
  std::string why;
  const int st = ozaki_gemm_dd(g, s, &why);
  if (st) return fail(ctx, st, "exact-slice GEMM: " + why);
  CLR_CHECK_LAUNCH("exact-slice GEMM");
  // tile flags, their compaction, one GEMM launch per K pass
  prof_launches(ctx, 2 + (int)((K_pad + kOzakiPassK - 1) / kOzakiPassK));
  if (ctx->prof_on) ctx->prof.dense_launches++;
  prof_mark(ctx, s, PH_DENSE);
  return CLR_OK;
}

int multiply_into(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c, double alpha,
                  const Tuning& tune, clr_product_stats* stats, cudaStream_t s) {
  const int prec = tune.prec;
  const double eps_lr = tune.eps >= 0.0 ? tune.eps : ctx->opts.eps_lr;
  if (!same_clusters(a->col_sizes, b->row_sizes))
    return fail(ctx, CLR_EINVAL, "inner clusters of A and B differ");
  if (!same_clusters(c->row_sizes, a->row_sizes) || !same_clusters(c->col_sizes, b->col_sizes))
    return fail(ctx, CLR_EINVAL, "C clusters do not match A rows / B columns");
  if (c == a || c == b) return fail(ctx, CLR_EINVAL, "C aliases an operand");
  if (!std::isfinite(alpha)) return fail(ctx, CLR_EINVAL, "alpha not finite");
  Plan p;
  int st = make_plan(ctx, a->nr, b->nc, a->nc, &p);
  if (st) return st;
  p.row_off = c->d_row_off;
  p.col_off = c->d_col_off;
  p.c_cost = c->d_cost;
  CLR_CUDA(ctx->cur->ws.ensure(2 * (size_t)c->n_rows * c->n_cols * sizeof(double)));
  const int lr_grid = grid_of(ctx, tune.lr_mult);
  CLR_CUDA(ctx->cur->scratch.ensure((size_t)lr_grid * scratch_per_cta() * sizeof(double)));
  MatView av = a->view(), bv = b->view(), cv = c->view();
  const clr_opts& o = ctx->opts;
  const bool recompress_dense =
      tune.recompress >= 0 ? tune.recompress != 0 : o.recompress_dense != 0;
  prof_mark(ctx, s, PH_START);
  // split precision: densely accumulated low-rank sums go to the tensor-core GEMM where its
  // error bound u sum_K ||A_IK|| ||B_KJ|| stays below eps / 16 (u: 2^-15 bf16x3, 2^-22 bf16x6)
  const double u_split = prec == CLR_PREC_BF16X3 ? std::ldexp(1.0, -15)
                         : prec == CLR_PREC_BF16X6 ? std::ldexp(1.0, -22) : 0.0;
  const double dacc_bound = u_split > 0.0 ? eps_lr / (16.0 * u_split) : 0.0;
  bool fused_norms = false;
  OzDaccRule oz_rule;
  if (prec == CLR_PREC_OZAKI) {
    st = stage_ozaki(ctx, a, b, c, eps_lr, s, &oz_rule);
    if (st) return st;
  }
  launch_plan(av, bv, p, o.eps_sp, recompress_dense, dacc_bound, oz_rule, s);
  launch_set_route_kinds(cv, p, s);
  CLR_CHECK_LAUNCH("plan");
  prof_launches(ctx, 4);
  prof_mark(ctx, s, PH_PLAN);
  if (prec == CLR_PREC_FP64) {
    launch_dd_fp64(av, bv, cv, p, grid_of(ctx, 4), s);
    CLR_CHECK_LAUNCH("dense x dense (FP64)");
    prof_launches(ctx, 1);
    if (ctx->prof_on) ctx->prof.dense_launches++;
    prof_mark(ctx, s, PH_DENSE);
  } else if (prec == CLR_PREC_OZAKI) {
    st = run_ozaki_gemm(ctx, a, c, p, s);
    if (st) return st;
  } else {
    st = run_split_dd(ctx, a, b, c, p, prec, recompress_dense, s, &fused_norms);
    if (st) return st;
  }
  // the tensor-core GEMMs form the whole sum of the tiles they serve (route DENSE and DACC_G:
  // the low-rank blocks are staged as reconstructions): the low-rank kernel skips those
  const bool dense_by_gemm = prec != CLR_PREC_FP64;
  launch_lr_products(av, bv, cv, p, (double*)ctx->cur->ws.p, (double*)ctx->cur->scratch.p,
                     kScratchPerCta, dense_by_gemm, lr_grid, s);
  CLR_CHECK_LAUNCH("low-rank products");
  prof_launches(ctx, 1);
  prof_mark(ctx, s, PH_LOWRANK);
  launch_compress_qr(cv, p.l_qr_s, &p.counters->n_qr, p.t_rsum, (double*)ctx->cur->ws.p,
                     (double*)ctx->cur->scratch.p, eps_lr, o.jacobi_max_sweeps,
                     lr_grid, &p.counters->err, &p.counters->sched[1], jst(ctx, 1), s);
  prof_mark(ctx, s, PH_COMPRESS_QR);
  launch_compress_dense(cv, p.l_dcomp_s, &p.counters->n_dcomp, nullptr, nullptr, 0,
                        (double*)ctx->cur->ws.p, (double*)ctx->cur->scratch.p,
                        eps_lr, 0.0, 0, 0, o.svd_no_prereduce ? 0 : 1, o.jacobi_max_sweeps,
                        lr_grid, &p.counters->err,
                        &p.counters->sched[2], jst(ctx), s);
  CLR_CHECK_LAUNCH("recompression");
  prof_launches(ctx, 2);
  prof_mark(ctx, s, PH_COMPRESS);
  if (!recompress_dense) {
    if (fused_norms)
      launch_sqrt_dense_norms(cv, p, s);
    else
      launch_dense_tile_norms(cv, p, s);
    prof_launches(ctx, 1);
  }
  if (alpha != 1.0) {
    launch_scale_blocks(cv, alpha, s);
    prof_launches(ctx, 1);
  }
  CLR_CHECK_LAUNCH("finalize");
  prof_mark(ctx, s, PH_FINALIZE);
  if (ctx->prof_on) ctx->prof.products++;
  if (stats) {
    PlanCounters pc;
    CLR_CUDA(cudaMemcpyAsync(&pc, p.counters, sizeof(pc), cudaMemcpyDeviceToHost, s));
    CLR_CUDA(cudaStreamSynchronize(s));
    ctx->last_counters = pc;
    for (int q = 0; q < 4; ++q) stats->n_triples[q] = (int64_t)pc.by_kind[q];
    stats->flops = (int64_t)pc.flops;
    for (int q = 0; q < 3; ++q) stats->n_tiles[q] = (int64_t)pc.by_mode[q];
    stats->max_rank_sum = (int64_t)pc.max_rsum;
    stats->precision = prec;
    stats->n_tiles_tensor =
        prec == CLR_PREC_FP64 ? 0 : (int32_t)(pc.by_mode[1] + pc.n_gemm_dacc);
    st = take_device_error(ctx);
    if (st) return st;
  }
  return CLR_OK;
}

}  // namespace

extern "C" int clr_profile_enable(clr_ctx_t ctx, int on) {
  if (!ctx) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  for (auto& pe : ctx->prof_events) ctx->event_pool.push_back(pe.e);
  ctx->prof_events.clear();
  std::memset(&ctx->prof, 0, sizeof(ctx->prof));
  ctx->prof_on = on != 0;
  if (ctx->prof_on) {
    const size_t bytes = kJstatsBlocks * kJstatsBlock * sizeof(unsigned long long);
    CLR_CUDA(ctx->jstats.ensure(bytes));
    CLR_CUDA(cudaMemset(ctx->jstats.p, 0, bytes));
  }
  return CLR_OK;
}

extern "C" int clr_profile_read(clr_ctx_t ctx, clr_profile* out) {
  if (!ctx || !out) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  if (!ctx->prof_events.empty()) {
    CLR_CUDA(cudaDeviceSynchronize());
    std::map<cudaStream_t, cudaEvent_t> prev;  // last event per stream
    for (auto& pe : ctx->prof_events) {
      auto it = prev.find(pe.s);
      if (pe.phase != PH_START && it != prev.end()) {
        float ms = 0.f;
        CLR_CUDA(cudaEventElapsedTime(&ms, it->second, pe.e));
        double* slot = pe.phase == PH_PLAN ? &ctx->prof.ms_plan
                     : pe.phase == PH_STAGE ? &ctx->prof.ms_stage
                     : pe.phase == PH_DENSE ? &ctx->prof.ms_dense
                     : pe.phase == PH_LOWRANK ? &ctx->prof.ms_lowrank
                     : pe.phase == PH_COMPRESS_QR ? &ctx->prof.ms_compress_qr
                     : pe.phase == PH_COMPRESS ? &ctx->prof.ms_compress_dense
                     : &ctx->prof.ms_finalize;
        *slot += ms;
        if (pe.phase == PH_COMPRESS_QR || pe.phase == PH_COMPRESS) ctx->prof.ms_compress += ms;
      }
      prev[pe.s] = pe.e;
    }
    for (auto& pe : ctx->prof_events) ctx->event_pool.push_back(pe.e);
    ctx->prof_events.clear();
  }
  if (ctx->jstats.p) {
    unsigned long long j[kJstatsBlocks * kJstatsBlock];
    CLR_CUDA(cudaMemcpy(j, ctx->jstats.p, sizeof(j), cudaMemcpyDeviceToHost));
    const unsigned long long* q = j + kJstatsBlock;   // the QR route's block
    ctx->prof.svd_blocks = (int64_t)(j[0] + q[0]);
    ctx->prof.svd_sweeps_fp32 = (int64_t)(j[1] + q[1]);
    ctx->prof.svd_sweeps_fp64 = (int64_t)(j[2] + q[2]);
    ctx->prof.svd_early_dense = (int64_t)j[3];
    ctx->prof.svd_flops_fp64 = (double)(j[4] + q[4]);
    ctx->prof.svd_flops_fp32 = (double)(j[5] + q[5]);
    ctx->prof.svd_prereduced = (int64_t)j[6];
    ctx->prof.svd_flops_fp64_qr = (double)q[4];
    ctx->prof.svd_flops_fp32_qr = (double)q[5];
    const unsigned long long* pc = j + 2 * kJstatsBlock;   // per-path SM cycles and counts
    for (int path = 0; path < 4; ++path) {
      ctx->prof.svd_path_cycles[path] = (double)pc[2 * path];
      ctx->prof.svd_path_blocks[path] = (int64_t)pc[2 * path + 1];
    }
    const unsigned long long* fc = j + 3 * kJstatsBlock;  // full-SVD stages (kFullStage*)
    for (int st = 0; st < 7; ++st) ctx->prof.svd_full_cycles[st] = (double)fc[st];
    ctx->prof.svd_full_blocks = (int64_t)fc[7];
    ctx->prof.svd_full_dense = (int64_t)j[7];
    const unsigned long long* rc = j + 4 * kJstatsBlock;  // pre-reduced path stages
    for (int st = 0; st < 7; ++st) ctx->prof.svd_pre_cycles[st] = (double)rc[st];
    ctx->prof.svd_pre_blocks = (int64_t)rc[7];
  }
  *out = ctx->prof;
  return CLR_OK;
}

extern "C" int clr_multiply_into(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c,
                                 double alpha, clr_product_stats* stats, void* stream) {
  if (!ctx || !a || !b || !c) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  Tuning t;
  t.prec = choose_precision(ctx, a, b);
  return multiply_into(ctx, a, b, c, alpha, t, stats, as_stream(stream));
}

extern "C" int clr_multiply(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t* c,
                            void* stream) {
  if (!ctx || !a || !b || !c) return CLR_EINVAL;
  *c = nullptr;
  cudaSetDevice(ctx->device);
  clr_mat_t out = nullptr;
  int st = alloc_mat(ctx, a->nr, a->row_sizes.data(), b->nc, b->col_sizes.data(), &out);
  if (st) return st;
  Tuning t;
  t.prec = choose_precision(ctx, a, b);
  st = multiply_into(ctx, a, b, out, 1.0, t, nullptr, as_stream(stream));
  if (st) {
    free_mat(out);
    return st;
  }
  *c = out;
  return CLR_OK;
}

extern "C" int clr_multiply_backward(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t cbar,
                                     clr_mat_t* abar, clr_mat_t* bbar, void* stream) {
  // Adjoint of C = A B (Section 4.1's block product, truncation treated as the identity):
  // Abar = Cbar B^T and Bbar = A^T Cbar, each a CLR product recompressed at eps_lr.
  if (!ctx || !a || !b || !cbar || (!abar && !bbar)) return CLR_EINVAL;
  if (abar) *abar = nullptr;
  if (bbar) *bbar = nullptr;
  if (!same_clusters(a->col_sizes, b->row_sizes))
    return fail(ctx, CLR_EINVAL, "inner clusters of A and B differ");
  if (!same_clusters(cbar->row_sizes, a->row_sizes) ||
      !same_clusters(cbar->col_sizes, b->col_sizes))
    return fail(ctx, CLR_EINVAL, "Cbar clusters do not match A rows / B columns");
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  MatGuard g;
  Tuning t;
  int st = CLR_OK;
  clr_mat_t ab = nullptr, bb = nullptr;
  if (abar) {
    clr_mat_t bt = nullptr;
    if ((st = alloc_mat(ctx, b->nc, b->col_sizes.data(), b->nr, b->row_sizes.data(), &bt)))
      return st;
    g.v.push_back(bt);
    launch_transpose(b->view(), bt->view(), s);
    CLR_CHECK_LAUNCH("transpose");
    if ((st = alloc_mat(ctx, a->nr, a->row_sizes.data(), a->nc, a->col_sizes.data(), &ab)))
      return st;
    g.v.push_back(ab);
    t.prec = choose_precision(ctx, cbar, bt);
    if ((st = multiply_into(ctx, cbar, bt, ab, 1.0, t, nullptr, s))) return st;
  }
  if (bbar) {
    clr_mat_t at = nullptr;
    if ((st = alloc_mat(ctx, a->nc, a->col_sizes.data(), a->nr, a->row_sizes.data(), &at)))
      return st;
    g.v.push_back(at);
    launch_transpose(a->view(), at->view(), s);
    CLR_CHECK_LAUNCH("transpose");
    if ((st = alloc_mat(ctx, b->nr, b->row_sizes.data(), b->nc, b->col_sizes.data(), &bb)))
      return st;
    g.v.push_back(bb);
    t.prec = choose_precision(ctx, at, cbar);
    if ((st = multiply_into(ctx, at, cbar, bb, 1.0, t, nullptr, s))) return st;
  }
  // the transposes go back to the allocator only once the products that read them are done
  CLR_CUDA(cudaStreamSynchronize(s));
  if ((st = take_device_error(ctx))) return st;
  if (abar) *abar = g.keep(ab);
  if (bbar) *bbar = g.keep(bb);
  return CLR_OK;
}

extern "C" int clr_lincomb(clr_ctx_t ctx, double a, clr_mat_t x, double b, clr_mat_t y,
                           double diag, clr_mat_t out, void* stream) {
  if (!ctx || !x || !y || !out) return CLR_EINVAL;
  if (x->row_sizes != y->row_sizes || x->col_sizes != y->col_sizes ||
      out->row_sizes != x->row_sizes || out->col_sizes != x->col_sizes)
    return fail(ctx, CLR_EINVAL, "lincomb: clusters differ");
  if (out == x || out == y) return fail(ctx, CLR_EINVAL, "lincomb: output aliases an input");
  if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(diag))
    return fail(ctx, CLR_EINVAL, "lincomb: coefficient not finite");
  if (diag != 0.0 && x->row_sizes != x->col_sizes)
    return fail(ctx, CLR_EINVAL, "lincomb: diagonal shift needs square clusters");
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  Plan p;
  int st = make_plan(ctx, x->nr, x->nc, 1, &p);
  if (st) return st;
  p.row_off = out->d_row_off;
  p.col_off = out->d_col_off;
  CLR_CUDA(ctx->cur->ws.ensure(2 * (size_t)x->n_rows * x->n_cols * sizeof(double)));
  const int grid = grid_of(ctx, 2);
  CLR_CUDA(ctx->cur->scratch.ensure((size_t)grid * scratch_per_cta() * sizeof(double)));
  const clr_opts& o = ctx->opts;
  MatView xv = x->view(), yv = y->view(), ov = out->view();
  launch_lincomb_plan(a, xv, b, yv, diag, ov, p, (double*)ctx->cur->ws.p, o.recompress_dense, s);
  launch_compress_qr(ov, p.l_qr_s, &p.counters->n_qr, p.t_rsum, (double*)ctx->cur->ws.p,
                     (double*)ctx->cur->scratch.p, o.eps_lr,
                     o.jacobi_max_sweeps, grid, &p.counters->err, &p.counters->sched[1],
                     jst(ctx, 1), s);
  launch_compress_dense(ov, p.l_dcomp_s, &p.counters->n_dcomp, nullptr, nullptr, 0,
                        (double*)ctx->cur->ws.p, (double*)ctx->cur->scratch.p,
                        o.eps_lr, 0.0, 0, 0, o.svd_no_prereduce ? 0 : 1, o.jacobi_max_sweeps,
                        grid, &p.counters->err,
                        &p.counters->sched[2], jst(ctx), s);
  CLR_CHECK_LAUNCH("lincomb");
  return CLR_OK;
}

// =============================================================================================
// Newton–Schulz (Section 4.2)
// =============================================================================================
namespace {

__global__ void fill_kernel(double* v, int64_t n, double val) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = val;
}

// v <- w / ||w|| and dot = v^T w (single CTA, deterministic).
__global__ void __launch_bounds__(1024) normalize_kernel(const double* w, double* v, int64_t n,
                                                         double* norm_out) {
  __shared__ double red[32];
  __shared__ double tot;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(w[i], w[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    tot = t;
    if (norm_out) *norm_out = sqrt(t);
  }
  __syncthreads();
  const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
  if (v)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = w[i] * inv;
}

__global__ void __launch_bounds__(1024) dot_kernel(const double* a, const double* b, int64_t n,
                                                   double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    *out = t;
  }
}

// alpha = 1 / (1.01 lambda), lambda the Rayleigh quotient after `steps` power iterations from
// the normalised all-ones vector (reading of Section 4.2: ||alpha M - I||_2 <= 1).
int estimate_alpha(clr_ctx_t ctx, clr_mat_t s_mat, int steps, cudaStream_t s, double* alpha) {
  const int64_t n = s_mat->n_rows;
  CLR_CUDA(ctx->small.ensure((size_t)(3 * n + 4) * sizeof(double)));
  double* v = (double*)ctx->small.p;
  double* w = v + n;
  double* scal = w + n;
  fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, n, 1.0 / std::sqrt((double)n));
  MatView sv = s_mat->view();
  for (int it = 0; it < steps; ++it) {
    launch_matvec(sv, v, w, s);
    normalize_kernel<<<1, 1024, 0, s>>>(w, v, n, nullptr);
  }
  launch_matvec(sv, v, w, s);
  dot_kernel<<<1, 1024, 0, s>>>(v, w, n, scal);
  CLR_CHECK_LAUNCH("alpha estimate");
  double lam = 0.0;
  CLR_CUDA(cudaMemcpyAsync(&lam, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CLR_CUDA(cudaStreamSynchronize(s));
  if (!(lam > 0.0) || !std::isfinite(lam))
    return fail(ctx, CLR_EINVAL, "alpha estimate: matrix is not positive definite");
  *alpha = 1.0 / (1.01 * lam);
  return CLR_OK;
}

int identity_distance(clr_ctx_t ctx, clr_mat_t x, cudaStream_t s, double* out) {
  const size_t nb = (size_t)x->nr * x->nc;
  DevBuf& buf = ctx->small;
  const size_t need = (size_t)(3 * x->n_rows + 4 + 1 + nb) * sizeof(double);
  if (buf.bytes < need) CLR_CUDA(buf.ensure(need));
  double* part = (double*)buf.p + 3 * x->n_rows + 4;
  launch_identity_distance(x->view(), part, s);
  CLR_CHECK_LAUNCH("identity distance");
  double sq = 0.0;
  CLR_CUDA(cudaMemcpyAsync(&sq, part, sizeof(double), cudaMemcpyDeviceToHost, s));
  CLR_CUDA(cudaStreamSynchronize(s));
  const int st = take_device_error(ctx);
  if (st) return st;
  *out = std::sqrt(std::max(sq, 0.0) / (double)x->n_rows);
  return CLR_OK;
}

}  // namespace

namespace {

// Truncation of the residual's two products: at most 1/100 of the tolerance, so that their
// truncation error (at most about 11 eps sqrt(#tiles / N) for ||Z||_2 <= 10, far less in
// practice) cannot decide whether the residual meets ns_tol.
double residual_eps(const clr_opts& o) {
  return o.ns_tol > 0.0 ? std::min(o.eps_lr, 1e-2 * o.ns_tol) : o.eps_lr;
}

}  // namespace

extern "C" int clr_ns_residual(clr_ctx_t ctx, clr_mat_t s_mat, clr_mat_t z, double* out,
                               void* stream) {
  if (!ctx || !s_mat || !z || !out) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  MatGuard g;
  clr_mat_t zs = nullptr, zsz = nullptr;
  int st = alloc_mat(ctx, z->nr, z->row_sizes.data(), s_mat->nc, s_mat->col_sizes.data(), &zs);
  if (st) return st;
  g.v.push_back(zs);
  st = alloc_mat(ctx, z->nr, z->row_sizes.data(), z->nc, z->col_sizes.data(), &zsz);
  if (st) return st;
  g.v.push_back(zsz);
  // FP64-accurate products (the residual is the stated error, so it is not taken in split
  // precision): FP64, or exact slices when the context runs them, whose error per entry is at
  // most K 2^-39 2^(e_i + f_j) (|a_ik| < 2^e_i, |b_kj| < 2^f_j), far below any stated error
  // these iterates reach.  Densely accumulated tiles are not re-tested for low rank: Z S and
  // Z S Z are only summed, and their tiles stay as accurate as the products make them.
  Tuning t;
  t.prec = ctx->opts.precision == CLR_PREC_OZAKI ? CLR_PREC_OZAKI : CLR_PREC_FP64;
  t.eps = residual_eps(ctx->opts);
  t.recompress = 0;
  st = multiply_into(ctx, z, s_mat, zs, 1.0, t, nullptr, s);
  if (st) return st;
  st = multiply_into(ctx, zs, z, zsz, 1.0, t, nullptr, s);
  if (st) return st;
  return identity_distance(ctx, zsz, s, out);
}

extern "C" int clr_check(clr_ctx_t ctx, void* stream) {
  if (!ctx) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  CLR_CUDA(cudaStreamSynchronize(as_stream(stream)));
  if (ctx->side) CLR_CUDA(cudaStreamSynchronize(ctx->side));
  return take_device_error(ctx);
}

extern "C" int clr_sqrt_inv(clr_ctx_t ctx, clr_mat_t s_mat, clr_mat_t* z_out,
                            clr_ns_stats* stats, clr_tape_t* tape_out, void* stream) {
  if (!ctx || !s_mat || !z_out) return CLR_EINVAL;
  *z_out = nullptr;
  if (tape_out) *tape_out = nullptr;
  if (s_mat->row_sizes != s_mat->col_sizes)
    return fail(ctx, CLR_EINVAL, "S must have equal row and column clusters");
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  const clr_opts& o = ctx->opts;
  if (o.ns_max_iter < 0 || o.ns_max_iter >= CLR_NS_MAX_HISTORY)
    return fail(ctx, CLR_EINVAL, "ns_max_iter out of range");
  double alpha = o.ns_alpha;
  int st = CLR_OK;
  if (!(alpha > 0.0)) {
    st = estimate_alpha(ctx, s_mat, o.ns_power_steps, s, &alpha);
    if (st) return st;
  }
  const int nr = s_mat->nr;
  const int32_t* sz = s_mat->row_sizes.data();
  MatGuard g;
  clr_mat_t mats[7];
  for (int i = 0; i < 7; ++i) {
    st = alloc_mat(ctx, nr, sz, nr, sz, &mats[i]);
    if (st) return st;
    g.v.push_back(mats[i]);
  }
  clr_mat_t Y = mats[0], Z = mats[1], X = mats[2], X2 = mats[3], T = mats[4], Yn = mats[5],
            Zn = mats[6];
  std::unique_ptr<clr_tape_s> tape;
  if (tape_out) {
    tape.reset(new clr_tape_s);
    tape->alpha = alpha;
    tape->sizes = s_mat->row_sizes;
    tape->prec = choose_precision(ctx, s_mat, s_mat);
  }
  st = clr_mat_copy(ctx, s_mat, Y, s);
  if (st) return st;
  // Z_0 = I: 0 * S + 0 * S + 1 * I
  st = clr_lincomb(ctx, 0.0, s_mat, 0.0, s_mat, 1.0, Z, s);
  if (st) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  for (clr_mat_t& m : ctx->snap) {
    if (m) free_mat(m);
    m = nullptr;
  }
  Tuning tn;
  tn.prec = choose_precision(ctx, s_mat, s_mat);
  int& prec = tn.prec;
  int it = 0;
  bool proxy_met = false;
  std::vector<double> proxies;
  std::vector<int> precs;
  while (true) {
    st = multiply_into(ctx, Y, Z, X, alpha, tn, nullptr, s);
    if (st) break;
    double px = 0.0;
    st = identity_distance(ctx, X, s, &px);
    if (st) break;
    proxies.push_back(px);
    precs.push_back(prec);
    if (!std::isfinite(px)) {
      st = fail(ctx, CLR_ENOCONV, "Newton-Schulz diverged (non-finite residual)");
      break;
    }
    if (o.ns_tol > 0.0 && px <= o.ns_tol) {
      proxy_met = true;
      break;
    }
    if (it >= o.ns_max_iter) break;
    if (o.ns_fp64_tail && px <= o.ns_ladder_switch) prec = CLR_PREC_FP64;
    if (tape) {
      clr_mat_t yc = nullptr, zc = nullptr;
      st = alloc_mat(ctx, nr, sz, nr, sz, &yc);
      if (st) break;
      st = alloc_mat(ctx, nr, sz, nr, sz, &zc);
      if (st) { free_mat(yc); break; }
      tape->y.push_back(yc);
      tape->z.push_back(zc);
      if ((st = clr_mat_copy(ctx, Y, yc, s)) || (st = clr_mat_copy(ctx, Z, zc, s))) break;
    }
    st = multiply_into(ctx, X, X, X2, 1.0, tn, nullptr, s);
    if (st) break;
    st = clr_lincomb(ctx, -10.0 / 8.0, X, 3.0 / 8.0, X2, 15.0 / 8.0, T, s);
    if (st) break;
    // Z T and T Y are independent: T Y runs on the side stream with the second workspace set,
    // so that the SMs one product's longest tiles leave idle take the other's work.  While
    // profiling they run one after the other, so that the per-phase event intervals time one
    // kernel each.
    if (ctx->prof_on) {
      st = multiply_into(ctx, T, Y, Yn, 1.0, tn, nullptr, s);
      if (!st) st = multiply_into(ctx, Z, T, Zn, 1.0, tn, nullptr, s);
      if (st) break;
    } else {
      st = fork_side(ctx, s);
      if (st) break;
      {
        WorkSet* saved = ctx->cur;
        ctx->cur = ctx->wsets[1].get();
        st = multiply_into(ctx, T, Y, Yn, 1.0, tn, nullptr, ctx->side);
        ctx->cur = saved;
      }
      if (!st) st = multiply_into(ctx, Z, T, Zn, 1.0, tn, nullptr, s);
      const int sj = join_side(ctx, s);
      if (st || (st = sj)) break;
    }
    std::swap(Z, Zn);
    std::swap(Y, Yn);
    ++it;
    if (it == o.ns_snapshot_iter) {
      const clr_mat_t src[4] = {X, T, Y, Z};
      for (int k = 0; k < 4 && !st; ++k) {
        st = alloc_mat(ctx, nr, sz, nr, sz, &ctx->snap[k]);
        if (!st) st = clr_mat_copy(ctx, src[k], ctx->snap[k], s);
      }
      if (st) break;
    }
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tape) {
    tape->iters = (int)tape->y.size();
  }
  if (st) {
    if (tape)
      for (size_t i = 0; i < tape->y.size(); ++i) {
        free_mat(tape->y[i]);
        free_mat(tape->z[i]);
      }
    return st;
  }
  // Z_out = sqrt(alpha) Z
  clr_mat_t zo = g.keep(Z);
  auto drop = [&](int code) {
    free_mat(zo);
    if (tape)
      for (size_t i = 0; i < tape->y.size(); ++i) {
        free_mat(tape->y[i]);
        free_mat(tape->z[i]);
      }
    return code;
  };
  launch_scale_blocks(zo->view(), std::sqrt(alpha), s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return drop(cuda_fail(ctx, e, "scale"));
  // The stated error: the residual of the returned Z (FP64 products, Section 4.2's
  // convergence target), whenever a tolerance is set or statistics are wanted.
  double res = NAN;
  float ms_res = 0.f;
  if (o.ns_tol > 0.0 || stats) {
    cudaEvent_t r0, r1;
    cudaEventCreate(&r0);
    cudaEventCreate(&r1);
    cudaEventRecord(r0, s);
    const int rs = clr_ns_residual(ctx, s_mat, zo, &res, stream);
    cudaEventRecord(r1, s);
    cudaEventSynchronize(r1);
    cudaEventElapsedTime(&ms_res, r0, r1);
    cudaEventDestroy(r0);
    cudaEventDestroy(r1);
    if (rs) return drop(rs);
  }
  const bool residual_met = o.ns_tol > 0.0 && res <= o.ns_tol;
  const bool converged = o.ns_tol == 0.0 || residual_met;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iters = it;
    stats->converged = converged ? 1 : 0;
    stats->alpha = alpha;
    for (size_t i = 0; i < proxies.size() && i < CLR_NS_MAX_HISTORY; ++i) {
      stats->proxy[i] = proxies[i];
      stats->precision_used[i] = precs[i];
    }
    stats->ms_total = ms;
    stats->residual = res;
    stats->proxy_met = proxy_met ? 1 : 0;
    stats->residual_met = residual_met ? 1 : 0;
    stats->ms_residual = ms_res;
  }
  *z_out = zo;
  if (tape_out) *tape_out = tape.release();
  if (!converged) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             proxy_met ? "Newton-Schulz: ||X - I|| met ns_tol but the residual %.3e exceeds it "
                         "(truncation at eps_lr holds it above the tolerance)"
                       : "Newton-Schulz did not reach ns_tol within ns_max_iter (residual %.3e)",
             res);
    ctx->err = msg;
    return CLR_ENOCONV;
  }
  return CLR_OK;
}

extern "C" int clr_ns_snapshot(clr_ctx_t ctx, int which, clr_mat_t* out) {
  if (!ctx || !out || which < 0 || which > 3) return CLR_EINVAL;
  *out = nullptr;
  if (!ctx->snap[which]) return fail(ctx, CLR_EINVAL, "no NS snapshot held");
  *out = ctx->snap[which];
  ctx->snap[which] = nullptr;
  return CLR_OK;
}

extern "C" int clr_tape_free(clr_ctx_t ctx, clr_tape_t tape) {
  if (!tape) return CLR_EINVAL;
  if (ctx) cudaSetDevice(ctx->device);
  for (clr_mat_t m : tape->y) free_mat(m);
  for (clr_mat_t m : tape->z) free_mat(m);
  delete tape;
  return CLR_OK;
}

extern "C" int clr_sqrt_inv_backward(clr_ctx_t ctx, clr_tape_t tape, clr_mat_t zbar,
                                     clr_mat_t* sbar, void* stream) {
  // Reverse sweep of Section 4.2's recurrences (alpha held constant; truncation treated as
  // the identity, every adjoint product a CLR product at eps_lr):
  //   Z_{n+1} = Z_n T_n      ->  Zb_n  = Zb_{n+1} T_n^T,       Tb_n  = Z_n^T Zb_{n+1}
  //   Y_{n+1} = T_n Y_n      ->  Yb_n  = T_n^T Yb_{n+1},       Tb_n += Yb_{n+1} Y_n^T
  //   T_n = (15I-10X+3X^2)/8 ->  Xb_n  = (-10 Tb_n + 3 (Tb_n X_n^T + X_n^T Tb_n)) / 8
  //   X_n = alpha Y_n Z_n    ->  Yb_n += alpha Xb_n Z_n^T,     Zb_n += alpha Y_n^T Xb_n
  // starting from Zb = sqrt(alpha) zbar (the output is sqrt(alpha) Z), Yb = 0; dL/dS = Yb_0.
  if (!ctx || !tape || !zbar || !sbar) return CLR_EINVAL;
  *sbar = nullptr;
  if (tape->sizes.empty() || zbar->row_sizes != tape->sizes || zbar->col_sizes != tape->sizes)
    return fail(ctx, CLR_EINVAL, "zbar clusters differ from S");
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  const int nr = (int)tape->sizes.size();
  const int32_t* sz = tape->sizes.data();
  MatGuard g;
  enum { X, X2, T, TT, XT, YT, ZT, TB, XB, ZB, YB, ZBN, YBN, W1, W2, NW };
  clr_mat_t m[NW];
  for (int i = 0; i < NW; ++i) {
    int st = alloc_mat(ctx, nr, sz, nr, sz, &m[i]);
    if (st) return st;
    g.v.push_back(m[i]);
  }
  const double alpha = tape->alpha;
  Tuning tn;
  tn.prec = tape->prec;
  auto mul = [&](clr_mat_t a, clr_mat_t b, clr_mat_t c, double sc) {
    return multiply_into(ctx, a, b, c, sc, tn, nullptr, s);
  };
  auto tr = [&](clr_mat_t a, clr_mat_t t) {
    launch_transpose(a->view(), t->view(), s);
    return cudaGetLastError() == cudaSuccess ? CLR_OK : CLR_ECUDA;
  };
  int st = clr_lincomb(ctx, std::sqrt(alpha), zbar, 0.0, zbar, 0.0, m[ZB], s);
  if (st) return st;
  st = clr_lincomb(ctx, 0.0, zbar, 0.0, zbar, 0.0, m[YB], s);  // Yb = 0
  if (st) return st;
  for (int n = tape->iters - 1; n >= 0; --n) {
    clr_mat_t Yn = tape->y[n], Zn = tape->z[n];
    if ((st = mul(Yn, Zn, m[X], alpha))) return st;                           // X = a Y Z
    if ((st = mul(m[X], m[X], m[X2], 1.0))) return st;                        // X^2
    if ((st = clr_lincomb(ctx, -10.0 / 8.0, m[X], 3.0 / 8.0, m[X2], 15.0 / 8.0, m[T], s)))
      return st;                                                               // T
    if ((st = tr(m[T], m[TT])) || (st = tr(m[X], m[XT])) || (st = tr(Yn, m[YT])) ||
        (st = tr(Zn, m[ZT])))
      return st;
    // Tb = Z^T Zb + Yb Y^T
    if ((st = mul(m[ZT], m[ZB], m[W1], 1.0)) || (st = mul(m[YB], m[YT], m[W2], 1.0)) ||
        (st = clr_lincomb(ctx, 1.0, m[W1], 1.0, m[W2], 0.0, m[TB], s)))
      return st;
    // Zb_n = Zb T^T ; Yb_n = T^T Yb
    if ((st = mul(m[ZB], m[TT], m[ZBN], 1.0)) || (st = mul(m[TT], m[YB], m[YBN], 1.0))) return st;
    // Xb = (-10 Tb + 3 (Tb X^T + X^T Tb)) / 8
    if ((st = mul(m[TB], m[XT], m[W1], 1.0)) || (st = mul(m[XT], m[TB], m[W2], 1.0)) ||
        (st = clr_lincomb(ctx, 1.0, m[W1], 1.0, m[W2], 0.0, m[X2], s)) ||
        (st = clr_lincomb(ctx, -10.0 / 8.0, m[TB], 3.0 / 8.0, m[X2], 0.0, m[XB], s)))
      return st;
    // Yb_n += a Xb Z^T ; Zb_n += a Y^T Xb
    if ((st = mul(m[XB], m[ZT], m[W1], alpha)) ||
        (st = clr_lincomb(ctx, 1.0, m[YBN], 1.0, m[W1], 0.0, m[YB], s)))
      return st;
    if ((st = mul(m[YT], m[XB], m[W2], alpha)) ||
        (st = clr_lincomb(ctx, 1.0, m[ZBN], 1.0, m[W2], 0.0, m[ZB], s)))
      return st;
  }
  *sbar = g.keep(m[YB]);
  return CLR_OK;
}

// =============================================================================================
// Autotuner and batched products
// =============================================================================================
namespace {

// Shape key of a product: sizes, cluster counts, block-kind counts of both operands and the
// truncation threshold.  Reads the operands' kinds (synchronises the stream).
int shape_key(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, double eps, cudaStream_t s,
              std::string* key) {
  std::vector<int> ka((size_t)a->nr * a->nc), kb((size_t)b->nr * b->nc);
  CLR_CUDA(cudaMemcpyAsync(ka.data(), a->d_kind, ka.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  CLR_CUDA(cudaMemcpyAsync(kb.data(), b->d_kind, kb.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  CLR_CUDA(cudaStreamSynchronize(s));
  long long cnt[2][3] = {{0, 0, 0}, {0, 0, 0}};
  for (int k : ka) cnt[0][k & 3 ? (k < 3 ? k : 0) : 0]++;
  for (int k : kb) cnt[1][k & 3 ? (k < 3 ? k : 0) : 0]++;
  char buf[256];
  snprintf(buf, sizeof(buf), "%lldx%lldx%lld/%dx%dx%d/d%lld,%lld/l%lld,%lld/e%.3g/s%.3g",
           (long long)a->n_rows, (long long)a->n_cols, (long long)b->n_cols, a->nr, a->nc, b->nc,
           cnt[0][1], cnt[1][1], cnt[0][2], cnt[1][2], eps, ctx->opts.eps_sp);
  *key = buf;
  return CLR_OK;
}

// Candidate precisions: the configured one, or under CLR_PREC_AUTO every mode whose a-priori
// error model meets the tolerance (FP64 always does).
std::vector<int> precision_candidates(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, double eps) {
  if (ctx->opts.precision != CLR_PREC_AUTO) return {ctx->opts.precision};
  const int cheapest = choose_precision(ctx, a, b, eps);
  std::vector<int> out;
  if (cheapest == CLR_PREC_BF16X3) out.push_back(CLR_PREC_BF16X3);
  if (cheapest == CLR_PREC_BF16X3 || cheapest == CLR_PREC_BF16X6) out.push_back(CLR_PREC_BF16X6);
  if (cheapest != CLR_PREC_FP64) out.push_back(CLR_PREC_OZAKI);
  out.push_back(CLR_PREC_FP64);
  return out;
}

int time_product(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c, const Tuning& t,
                 cudaStream_t s, double* ms) {
  int st = multiply_into(ctx, a, b, c, 1.0, t, nullptr, s);  // warm-up (also sizes workspaces)
  if (st) return st;
  cudaEvent_t e0, e1;
  CLR_CUDA(cudaEventCreate(&e0));
  CLR_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, s);
  st = multiply_into(ctx, a, b, c, 1.0, t, nullptr, s);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float f = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune timing");
  *ms = f;
  return CLR_OK;
}

// Fastest (precision, CTAs per SM) for this shape, measured once per shape key and cached.
int autotune(clr_ctx_t ctx, clr_mat_t a, clr_mat_t b, clr_mat_t c, double eps,
             cudaStream_t s, Tuning* out) {
  std::string key;
  int st = shape_key(ctx, a, b, eps, s, &key);
  if (st) return st;
  auto it = ctx->tune_cache.find(key);
  if (it != ctx->tune_cache.end()) {
    *out = it->second.first;
    out->eps = eps;
    return CLR_OK;
  }
  Tuning best;
  double best_ms = -1.0;
  for (int prec : precision_candidates(ctx, a, b, eps))
    for (int mult : {1, 2, 4}) {
      Tuning t;
      t.prec = prec;
      t.lr_mult = mult;
      t.eps = eps;
      double ms = 0.0;
      st = time_product(ctx, a, b, c, t, s, &ms);
      if (st) return st;
      if (best_ms < 0.0 || ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  ctx->tune_cache[key] = {best, best_ms};
  *out = best;
  return CLR_OK;
}

}  // namespace

extern "C" int clr_autotune_save(clr_ctx_t ctx, const char* path) {
  if (!ctx || !path) return CLR_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return fail(ctx, CLR_EINVAL, "cannot open autotune file for writing");
  for (auto& kv : ctx->tune_cache)
    fprintf(f, "%s %d %d %.6f\n", kv.first.c_str(), kv.second.first.prec,
            kv.second.first.lr_mult, kv.second.second);
  fclose(f);
  return CLR_OK;
}

extern "C" int clr_autotune_load(clr_ctx_t ctx, const char* path) {
  if (!ctx || !path) return CLR_EINVAL;
  FILE* f = fopen(path, "r");
  if (!f) return fail(ctx, CLR_EINVAL, "cannot open autotune file");
  char key[256];
  int prec = 0, mult = 0;
  double ms = 0.0;
  int n = 0;
  while (fscanf(f, "%255s %d %d %lf", key, &prec, &mult, &ms) == 4) {
    if (prec < 0 || prec > 4 || prec == CLR_PREC_AUTO || mult < 1 || mult > 8) continue;
    Tuning t;
    t.prec = prec;
    t.lr_mult = mult;
    ctx->tune_cache[key] = {t, ms};
    ++n;
  }
  fclose(f);
  return n >= 0 ? CLR_OK : CLR_EINVAL;
}

extern "C" int clr_autotune_entries(clr_ctx_t ctx) {
  return ctx ? (int)ctx->tune_cache.size() : CLR_EINVAL;
}

struct clr_batch_s {
  int n = 0;
  std::vector<clr_mat_t> a, b, c;
  std::vector<Tuning> tune;
  std::vector<int> branch;
  std::vector<std::unique_ptr<WorkSet>> wsets;  // one per branch, owned by the batch
  std::vector<cudaStream_t> streams;            // origin + branches
  std::vector<cudaEvent_t> events;              // fork + joins
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t last_run = nullptr;  // recorded after each launch on the caller's stream
  ~clr_batch_s() {
    if (last_run) cudaEventDestroy(last_run);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
    for (auto& w : wsets) w->release();
    for (clr_mat_t m : c) free_mat(m);
  }
};

extern "C" int clr_batch_create(clr_ctx_t ctx, int n, const clr_mat_t* a, const clr_mat_t* b,
                                const double* eps, int tune_on, void* stream, clr_batch_t* out) {
  if (!ctx || n < 1 || !a || !b || !out) return CLR_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  std::unique_ptr<clr_batch_s> bt(new (std::nothrow) clr_batch_s);
  if (!bt) return fail(ctx, CLR_ENOMEM, "host allocation");
  bt->n = n;
  for (int i = 0; i < n; ++i) {
    if (!a[i] || !b[i]) return CLR_EINVAL;
    if (a[i]->col_sizes != b[i]->row_sizes)
      return fail(ctx, CLR_EINVAL, "batch: inner clusters of A and B differ");
    bt->a.push_back(a[i]);
    bt->b.push_back(b[i]);
    clr_mat_t ci = nullptr;
    int st = alloc_mat(ctx, a[i]->nr, a[i]->row_sizes.data(), b[i]->nc, b[i]->col_sizes.data(), &ci);
    if (st) return st;
    bt->c.push_back(ci);
  }
  // tuning (uncaptured, on the context's own workspaces)
  WorkSet* saved = ctx->cur;
  for (int i = 0; i < n; ++i) {
    const double ei = eps ? eps[i] : ctx->opts.eps_lr;
    if (!(ei >= 0.0)) return fail(ctx, CLR_EINVAL, "batch: eps must be >= 0");
    Tuning t;
    t.prec = choose_precision(ctx, a[i], b[i], ei);
    t.eps = ei;
    if (tune_on) {
      int st = autotune(ctx, a[i], b[i], bt->c[i], ei, s, &t);
      if (st) return st;
    }
    bt->tune.push_back(t);
  }
  // branches: longest-processing-time assignment on a dense-equivalent cost estimate
  const int nb = std::min(n, 4);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto cost = [&](int i) {
    return (double)a[i]->n_rows * (double)a[i]->n_cols * (double)b[i]->n_cols;
  };
  std::sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::vector<double> load(nb, 0.0);
  bt->branch.assign(n, 0);
  for (int i : order) {
    const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    bt->branch[i] = br;
    load[br] += cost(i);
  }
  for (int br = 0; br < nb; ++br) bt->wsets.emplace_back(new WorkSet);
  // size each branch's workspaces (and warm up) with one uncaptured run per product
  for (int i = 0; i < n; ++i) {
    ctx->cur = bt->wsets[bt->branch[i]].get();
    int st = multiply_into(ctx, a[i], b[i], bt->c[i], 1.0, bt->tune[i], nullptr, s);
    if (st) {
      ctx->cur = saved;
      return st;
    }
  }
  ctx->cur = saved;
  CLR_CUDA(cudaStreamSynchronize(s));
  {
    const int st = take_device_error(ctx, &bt->wsets);
    if (st) return st;
  }
  // capture every product into one graph: fork to nb branches, join on the origin stream
  bt->streams.resize(nb + 1, nullptr);
  for (auto& st : bt->streams) CLR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  bt->events.resize(nb + 1, nullptr);
  for (auto& e : bt->events) CLR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaStream_t origin = bt->streams[0];
  CLR_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  int st = CLR_OK;
  cudaEventRecord(bt->events[0], origin);
  for (int br = 0; br < nb; ++br) cudaStreamWaitEvent(bt->streams[br + 1], bt->events[0], 0);
  for (int i = 0; i < n && !st; ++i) {
    ctx->cur = bt->wsets[bt->branch[i]].get();
    st = multiply_into(ctx, a[i], b[i], bt->c[i], 1.0, bt->tune[i], nullptr,
                       bt->streams[bt->branch[i] + 1]);
  }
  for (int br = 0; br < nb; ++br) {
    cudaEventRecord(bt->events[br + 1], bt->streams[br + 1]);
    cudaStreamWaitEvent(origin, bt->events[br + 1], 0);
  }
  ctx->capturing = false;
  ctx->cur = saved;
  cudaError_t e = cudaStreamEndCapture(origin, &bt->graph);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch capture");
  e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph instantiate");
  CLR_CUDA(cudaEventCreateWithFlags(&bt->last_run, cudaEventDisableTiming));
  *out = bt.release();
  return CLR_OK;
}

extern "C" int clr_batch_run(clr_ctx_t ctx, clr_batch_t batch, void* stream) {
  if (!ctx || !batch || !batch->exec) return CLR_EINVAL;
  cudaSetDevice(ctx->device);
  CLR_CUDA(cudaGraphLaunch(batch->exec, as_stream(stream)));
  CLR_CUDA(cudaEventRecord(batch->last_run, as_stream(stream)));
  return CLR_OK;
}

extern "C" int clr_batch_output(clr_batch_t batch, int i, clr_mat_t* c) {
  if (!batch || !c || i < 0 || i >= batch->n) return CLR_EINVAL;
  *c = batch->c[i];
  return CLR_OK;
}

extern "C" int clr_batch_tuning(clr_batch_t batch, int i, int* precision, int* lr_mult,
                                int* branch) {
  if (!batch || i < 0 || i >= batch->n) return CLR_EINVAL;
  if (precision) *precision = batch->tune[i].prec;
  if (lr_mult) *lr_mult = batch->tune[i].lr_mult;
  if (branch) *branch = batch->branch[i];
  return CLR_OK;
}

extern "C" int clr_batch_free(clr_ctx_t ctx, clr_batch_t batch) {
  if (!batch) return CLR_EINVAL;
  if (ctx) cudaSetDevice(ctx->device);
  // the graph runs on the caller's stream: wait for its last launch before the outputs and
  // workspaces go back to the allocator
  if (batch->last_run) cudaEventSynchronize(batch->last_run);
  for (cudaStream_t s : batch->streams) cudaStreamSynchronize(s);
  delete batch;
  return CLR_OK;
}

extern "C" int clr_multiply_batched(clr_ctx_t ctx, int n, const clr_mat_t* a,
                                    const clr_mat_t* b, clr_mat_t* c, void* stream) {
  // one graph launch for all n products (tuned when precision is CLR_PREC_AUTO); the outputs
  // are handed to the caller
  if (!ctx || n < 0 || (n > 0 && (!a || !b || !c))) return CLR_EINVAL;
  for (int i = 0; i < n; ++i) c[i] = nullptr;
  if (n == 0) return CLR_OK;
  clr_batch_t bt = nullptr;
  int st = clr_batch_create(ctx, n, a, b, nullptr, ctx->opts.precision == CLR_PREC_AUTO, stream,
                            &bt);
  if (st) return st;
  st = clr_batch_run(ctx, bt, stream);
  if (st == CLR_OK) {
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "batched products");
  }
  if (st == CLR_OK) st = take_device_error(ctx, &bt->wsets);
  if (st == CLR_OK)
    for (int i = 0; i < n; ++i) {
      c[i] = bt->c[i];
      bt->c[i] = nullptr;
    }
  bt->c.clear();
  clr_batch_free(ctx, bt);
  return st;
}

// =============================================================================================
// Streamed product of page-locked host matrices
// =============================================================================================
namespace {

// Cuts n_t clusters (sizes sz) into at most `parts` runs of whole clusters with balanced
// element counts: the returned boundaries are cluster indices, first 0, last n_t.
std::vector<int> cluster_cuts(int n_t, const int32_t* sz, int parts) {
  int64_t total = 0;
  for (int i = 0; i < n_t; ++i) total += sz[i];
  if (parts > n_t) parts = n_t;
  std::vector<int> cut(1, 0);
  int64_t acc = 0;
  for (int j = 0; j < n_t; ++j) {
    acc += sz[j];
    if ((int)cut.size() < parts && acc * parts >= total * (int64_t)cut.size() && j + 1 < n_t)
      cut.push_back(j + 1);
  }
  cut.push_back(n_t);
  return cut;
}

}  // namespace

extern "C" int clr_multiply_host_stream(clr_ctx_t ctx, const double* a, int64_t lda,
                                        const double* b, int64_t ldb, double* c, int64_t ldc,
                                        int n_rt, const int32_t* rs, int n_kt, const int32_t* ks,
                                        int n_ct, const int32_t* cs, int n_chunks,
                                        void* stream) {
  if (!ctx || !a || !b || !c || !rs || !ks || !cs || n_rt < 1 || n_kt < 1 || n_ct < 1 ||
      n_chunks < 1)
    return CLR_EINVAL;
  int64_t k = 0, n = 0;
  for (int i = 0; i < n_kt; ++i) k += ks[i];
  for (int i = 0; i < n_ct; ++i) n += cs[i];
  if (lda < k || ldb < n || ldc < n) return fail(ctx, CLR_EINVAL, "leading dimension too small");
  if (!host_device_ptr(a) || !host_device_ptr(b) || !host_device_ptr(c))
    return fail(ctx, CLR_EINVAL, "host buffers must be page-locked");
  cudaSetDevice(ctx->device);
  cudaStream_t s = as_stream(stream);
  // A in two row chunks, B and C in n_chunks column chunks (whole clusters); the product of
  // row chunk i and column chunk j is C's tile (i, j)
  const std::vector<int> rcut = cluster_cuts(n_rt, rs, 2), ccut = cluster_cuts(n_ct, cs, n_chunks);
  const int nra = (int)rcut.size() - 1, ncb = (int)ccut.size() - 1;
  std::vector<int64_t> row0(nra + 1, 0), col0(ncb + 1, 0);
  for (int i = 0; i < nra; ++i) {
    row0[i + 1] = row0[i];
    for (int r = rcut[i]; r < rcut[i + 1]; ++r) row0[i + 1] += rs[r];
  }
  for (int j = 0; j < ncb; ++j) {
    col0[j + 1] = col0[j];
    for (int q = ccut[j]; q < ccut[j + 1]; ++q) col0[j + 1] += cs[q];
  }
  int64_t up_max = 0, c_max = 0;
  for (int i = 0; i < nra; ++i) up_max = std::max(up_max, (row0[i + 1] - row0[i]) * k);
  for (int j = 0; j < ncb; ++j) up_max = std::max(up_max, k * (col0[j + 1] - col0[j]));
  for (int i = 0; i < nra; ++i)
    for (int j = 0; j < ncb; ++j)
      c_max = std::max(c_max, (row0[i + 1] - row0[i]) * (col0[j + 1] - col0[j]));
  // every matrix and buffer up front: alloc_mat's synchronous metadata uploads would otherwise
  // wait for the work already in flight and serialise the pipeline
  MatGuard g;
  int st = CLR_OK;
  std::vector<clr_mat_t> am(nra, nullptr), bm(ncb, nullptr), cm((size_t)nra * ncb, nullptr);
  for (int i = 0; i < nra && !st; ++i) {
    st = alloc_mat(ctx, rcut[i + 1] - rcut[i], rs + rcut[i], n_kt, ks, &am[i]);
    if (!st) g.v.push_back(am[i]);
  }
  for (int j = 0; j < ncb && !st; ++j) {
    st = alloc_mat(ctx, n_kt, ks, ccut[j + 1] - ccut[j], cs + ccut[j], &bm[j]);
    if (!st) g.v.push_back(bm[j]);
  }
  for (int i = 0; i < nra && !st; ++i)
    for (int j = 0; j < ncb && !st; ++j) {
      clr_mat_t& m = cm[(size_t)i * ncb + j];
      st = alloc_mat(ctx, rcut[i + 1] - rcut[i], rs + rcut[i], ccut[j + 1] - ccut[j],
                     cs + ccut[j], &m);
      if (!st) g.v.push_back(m);
    }
  if (st) return st;
  if ((st = fork_side(ctx, s))) return st;
  // streams: up (host-to-device copies), lay (their layout into the chunk matrices), the two
  // compute streams (s and side), dn[0..1] (each C tile's layout and device-to-host copy), so
  // that no copy waits for a kernel it does not depend on
  for (cudaStream_t* ps : {&ctx->up, &ctx->lay, &ctx->dn[0], &ctx->dn[1]})
    if (!*ps && cudaStreamCreateWithFlags(ps, cudaStreamNonBlocking) != cudaSuccess)
      return fail(ctx, CLR_ECUDA, "stream creation");
  for (cudaStream_t ps : {ctx->up, ctx->lay, ctx->dn[0], ctx->dn[1]})
    CLR_CUDA(cudaStreamWaitEvent(ps, ctx->ev_fork, 0));
  for (int sl = 0; sl < 2; ++sl) {
    WorkSet* w = ctx->wsets[sl].get();
    CLR_CUDA(w->host_c.ensure((size_t)c_max * sizeof(double)));   // download staging dn[sl]
    CLR_CUDA(w->host_b.ensure((size_t)up_max * sizeof(double)));   // upload staging, alternating
    w->staged_a = nullptr;
  }
  WorkSet* w0 = ctx->wsets[0].get();
  CLR_CUDA(w0->host_err.ensure(sizeof(int)));
  CLR_CUDA(cudaMemsetAsync(w0->host_err.p, 0, sizeof(int), ctx->lay));
  // per uploaded operand chunk (A row chunks, then B column chunks): copied (on up) and laid
  // out (on lay: the event the products wait for); per C tile: its product done
  const int n_up = nra + ncb, n_tiles = nra * ncb;
  std::vector<cudaEvent_t> ev(n_up, nullptr), ev_cp(n_up, nullptr), ev_pr(n_tiles, nullptr);
  struct EvGuard {
    std::vector<cudaEvent_t>* v[3];
    ~EvGuard() {
      for (auto* vv : v)
        for (cudaEvent_t e : *vv)
          if (e) cudaEventDestroy(e);
    }
  } eg{{&ev, &ev_cp, &ev_pr}};
  for (auto* vv : {&ev, &ev_cp, &ev_pr})
    for (auto& e : *vv)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
        return fail(ctx, CLR_ECUDA, "events");
  // uploads in the order the products need them: A_0, B_0, A_1, B_1, B_2, ...; upload u goes
  // through staging buffer u % 2, whose previous layout (upload u - 2) it waits for
  int n_issued = 0;
  std::vector<int> order_of;   // upload index of the n-th issued upload
  auto upload = [&](clr_mat_t M, const double* src, int64_t ld, int64_t rows, int64_t cols,
                    int u) -> int {
    WorkSet* wb = ctx->wsets[n_issued & 1].get();
    cudaError_t e = cudaSuccess;
    if (n_issued >= 2) e = cudaStreamWaitEvent(ctx->up, ev[order_of[n_issued - 2]], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(wb->host_b.p, cols * sizeof(double), src, ld * sizeof(double),
                            cols * sizeof(double), rows, cudaMemcpyHostToDevice, ctx->up);
    if (e == cudaSuccess) e = cudaEventRecord(ev_cp[u], ctx->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->lay, ev_cp[u], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream upload");
    launch_rowmajor_to_pool(M->view(), M->d_row_idx, (const double*)wb->host_b.p, cols, ctx->lay);
    launch_block_norms_dense(M->view(), ctx->lay);
    launch_dense_kinds(M->view(), 0.0, (int*)w0->host_err.p, ctx->lay);
    e = cudaEventRecord(ev[u], ctx->lay);
    ++n_issued;
    return e == cudaSuccess ? CLR_OK : cuda_fail(ctx, e, "stream upload");
  };
  for (int q = 0; q < std::max(nra, ncb) && !st; ++q) {
    if (q < nra) {
      order_of.push_back(q);
      st = upload(am[q], a + row0[q] * lda, lda, row0[q + 1] - row0[q], k, q);
    }
    if (!st && q < ncb) {
      order_of.push_back(nra + q);
      st = upload(bm[q], b + col0[q], ldb, k, col0[q + 1] - col0[q], nra + q);
    }
  }
  WorkSet* saved = ctx->cur;
  ctx->reuse_a = true;  // each stream keeps its row chunk of A: its bf16 panels are staged once
  Tuning t;
  if (!st) t.prec = choose_precision(ctx, am[0], am[0]);
  int n_done = 0;
  for (int j = 0; j < ncb && !st; ++j)
    for (int i = 0; i < nra && !st; ++i) {
      const int sl = nra > 1 ? (i & 1) : (j & 1);
      cudaStream_t ss = sl ? ctx->side : s;
      WorkSet* w = ctx->wsets[sl].get();
      ctx->cur = w;
      cudaError_t e = cudaStreamWaitEvent(ss, ev[i], 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ss, ev[nra + j], 0);
      if (e != cudaSuccess) {
        st = cuda_fail(ctx, e, "stream order");
        break;
      }
      clr_mat_t Cq = cm[(size_t)i * ncb + j];
      if ((st = multiply_into(ctx, am[i], bm[j], Cq, 1.0, t, nullptr, ss))) break;
      // C's tile back on a download stream (alternating, each with its staging buffer): layout
      // to row-major, copy engine device -> host, while the compute stream goes on
      const int d = n_done & 1;
      cudaStream_t sd = ctx->dn[d];
      e = cudaEventRecord(ev_pr[n_done], ss);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(sd, ev_pr[n_done], 0);
      if (e != cudaSuccess) {
        st = cuda_fail(ctx, e, "stream order");
        break;
      }
      ++n_done;
      WorkSet* wd = ctx->wsets[d].get();
      const int64_t nk = col0[j + 1] - col0[j];
      launch_pool_to_rowmajor(Cq->view(), Cq->d_row_idx, Cq->d_col_idx, (double*)wd->host_c.p,
                              nk, sd);
      e = cudaMemcpy2DAsync(c + row0[i] * ldc + col0[j], ldc * sizeof(double), wd->host_c.p,
                            nk * sizeof(double), nk * sizeof(double), row0[i + 1] - row0[i],
                            cudaMemcpyDeviceToHost, sd);
      if (e != cudaSuccess) st = cuda_fail(ctx, e, "stream download");
    }
  // join the helper streams and the side stream back into s
  cudaError_t ej = cudaSuccess;
  for (cudaStream_t ps : {ctx->up, ctx->lay, ctx->dn[0], ctx->dn[1]}) {
    if (ej == cudaSuccess) ej = cudaEventRecord(ctx->ev_join, ps);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, ctx->ev_join, 0);
  }
  const int sj = join_side(ctx, s);
  ctx->reuse_a = false;
  for (int sl = 0; sl < 2; ++sl) ctx->wsets[sl]->staged_a = nullptr;
  ctx->cur = saved;
  cudaError_t e = cudaStreamSynchronize(s);
  if (st) return st;
  if (sj) return sj;
  if (ej != cudaSuccess) return cuda_fail(ctx, ej, "streamed product");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "streamed product");
  int flag = 0;
  CLR_CUDA(cudaMemcpy(&flag, w0->host_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) return fail(ctx, CLR_EINVAL, "non-finite input in A or B");
  return take_device_error(ctx);
}

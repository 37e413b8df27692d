// Internal definitions shared by the liblgc translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/lgc.h"

#define LGC_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) {                                \
      lgc::set_last_cuda_error(e_, #expr, __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? LGC_ENOMEM : LGC_ECUDA; \
    }                                                       \
  } while (0)

#define LGC_TRY(expr)            \
  do {                           \
    int s_ = (expr);             \
    if (s_ < 0) return s_;       \
  } while (0)

namespace lgc {

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

constexpr int kBlock = 256;
constexpr int kWarp = 32;
// Bound on linear-probing steps.  Tables are kept at most half full, so a
// probe sequence this long means the table is corrupt or full.
constexpr uint32_t kMaxProbe = 1u << 20;

// Device-side error flags (bit mask in Counters::err).
constexpr int kErrTableFull = 1;
constexpr int kErrFrontierOverflow = 2;
constexpr int kErrDuplicate = 4;  // a sweep input names a vertex twice

// ---------------------------------------------------------------------------
// Hash table slot: key = vertex + 1 (0 = empty, so a zero memset clears the
// table), aux = per-algorithm integer (sweep rank), val = the sparse set's
// double.  Key and value share one 16-byte slot, so a probe and the
// following atomic add touch the same 32-byte sector.
// ---------------------------------------------------------------------------
struct __align__(16) Slot {
  int32_t key;
  int32_t aux;
  double val;
};

// A sparse set (vertex -> double, missing keys read as 0), in one of two
// representations chosen by the host per table:
//  - hashed: open addressing with linear probing over `cap` Slots (at most
//    half full), slot = probe position;
//  - dense: dval[v] indexed by the vertex id itself plus a presence bitmap
//    (bit v of bits[] says v is a key), slot = v.  Used once a set may hold
//    n/8 keys or more: no probing, and a value array that fits in L2 at the
//    sizes where hashing would not.
// `p` is an optional second double per slot (PR-Nibble's p) in either form.
struct Table {
  Slot* s = nullptr;
  double* p = nullptr;  // optional second value per slot (PR-Nibble's p)
  int64_t cap = 0;      // hashed: power of two; dense: n
  int shift = 32;       // hashed: 32 - log2(cap)
  int dense = 0;
  double* dval = nullptr;   // dense values, n entries
  uint32_t* bits = nullptr; // dense presence bitmap, ceil(n/32) words
};

__host__ __device__ inline uint32_t hash_slot(int32_t v, int shift) {
  // Fibonacci hashing: multiply by 2^32 / golden ratio, keep the top bits.
  return shift >= 32 ? 0u : (uint32_t)((uint32_t)v * 0x9E3779B1u) >> shift;
}

// Returns the slot of vertex v, inserting it if absent; *inserted = 1 if
// this call created the key.  Returns -1 (and sets the error flag) if the
// probe bound is exceeded.
__device__ inline int64_t ht_find_or_insert(const Table& T, int32_t v, int* inserted, int* err) {
  const uint32_t mask = (uint32_t)(T.cap - 1);
  const int32_t k = v + 1;
  uint32_t h = hash_slot(v, T.shift);
  for (uint32_t probe = 0; probe < kMaxProbe && probe <= mask; probe++) {
    int32_t cur = *((volatile int32_t*)&T.s[h].key);
    if (cur == k) return h;
    if (cur == 0) {
      int32_t prev = atomicCAS(&T.s[h].key, 0, k);
      if (prev == 0) {
        *inserted = 1;
        return h;
      }
      if (prev == k) return h;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, kErrTableFull);
  return -1;
}

// Lookup only; -1 if absent.
__device__ inline int64_t ht_find(const Table& T, int32_t v) {
  const uint32_t mask = (uint32_t)(T.cap - 1);
  const int32_t k = v + 1;
  uint32_t h = hash_slot(v, T.shift);
  for (uint32_t probe = 0; probe < kMaxProbe && probe <= mask; probe++) {
    int32_t cur = T.s[h].key;
    if (cur == k) return h;
    if (cur == 0) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// Representation-independent accessors.  T.dense is uniform across a launch.
__device__ inline int64_t tb_find_or_insert(const Table& T, int32_t v, int* inserted, int* err) {
  if (T.dense) {
    const uint32_t m = 1u << (v & 31);
    uint32_t* w = &T.bits[v >> 5];
    if (!(*(volatile uint32_t*)w & m)) {
      const uint32_t old = atomicOr(w, m);
      if (!(old & m)) *inserted = 1;
    }
    return v;
  }
  return ht_find_or_insert(T, v, inserted, err);
}

__device__ inline int64_t tb_find(const Table& T, int32_t v) {
  if (T.dense) return (T.bits[v >> 5] >> (v & 31)) & 1u ? v : -1;
  return ht_find(T, v);
}

__device__ inline double* tb_val(const Table& T, int64_t slot) {
  return T.dense ? &T.dval[slot] : &T.s[slot].val;
}

// Per-round device counters, read back by the host once per round.
struct Counters {
  int32_t next_size;   // entries appended to the next frontier
  int32_t err;         // kErr* bits
  int64_t next_edges;  // sum of degrees of the next frontier
  int64_t inserted;    // keys inserted into the destination table
  int64_t aux;         // algorithm-specific
};

// Warp-aggregated append of (v, slot, degree) to a frontier list.  Every
// lane of the calling group must call it (pred selects the appending lanes).
__device__ inline void frontier_append(bool pred, int32_t v, int32_t slot, int64_t d,
                                       int32_t* fv, int32_t* fs, Counters* C, int32_t cap) {
  const unsigned active = __activemask();
  const unsigned mask = __ballot_sync(active, pred);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  const int rank = __popc(mask & ((1u << lane) - 1));
  const unsigned dd = pred ? (unsigned)d : 0u;  // degrees < 2^31
  const unsigned lo = __reduce_add_sync(active, dd & 0xFFFFu);
  const unsigned hi = __reduce_add_sync(active, dd >> 16);
  int32_t base = 0;
  if (lane == leader) {
    base = atomicAdd(&C->next_size, __popc(mask));
    atomicAdd((unsigned long long*)&C->next_edges,
              (unsigned long long)lo + ((unsigned long long)hi << 16));
  }
  base = __shfl_sync(active, base, leader);
  if (pred) {
    int32_t pos = base + rank;
    if (pos < cap) {
      fv[pos] = v;
      fs[pos] = slot;
    } else {
      atomicOr(&C->err, kErrFrontierOverflow);
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side objects
// ---------------------------------------------------------------------------
struct Serve;  // request loop (serve.cu)

}  // namespace lgc

struct lgc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  lgc_alloc_fns alloc_fns = {nullptr, nullptr, nullptr};  // caller's allocator, if set
  bool own_stream = false;
  bool result_on_device = false;
  bool trace = false;
  int table_form = 0;   // LGC_OPT_TABLE_FORM
  int pull_policy = 0;  // LGC_OPT_PULL: 0 automatic, 1 never, 2 every deterministic round
  int sms = 152;              // multiprocessors of the device
  bool device_rounds = true;  // LGC_OPT_DEVICE_ROUNDS
  int pull_batch = 0;          // LGC_OPT_PULL_BATCH: 0 = the graph's tuned value
  int pull_group = 0;          // LGC_OPT_PULL_GROUP: 0 = the graph's tuned value
  int pull_share = 0;          // LGC_OPT_PULL_SHARE: 0 = the graph's tuned value
  int64_t batch_handoff = 0;   // LGC_OPT_BATCH_HANDOFF: 0 default, -1 never
  int hk_threshold_sign = 1;   // LGC_OPT_HK_THRESHOLD_SIGN: +1 (e^t, default) or -1 (e^-t)
  int sweep_cross = 0;  // LGC_OPT_SWEEP_CROSS: 0 automatic, 1 edge-balanced, 2 vertex-centric
  int64_t serve_mem_budget = 40ll << 30;
  int64_t serve_max_batch = 64;
  int64_t serve_lane_seeds = 1024;  // LGC_OPT_SERVE_LANE
  // the radix sort's per-tile status words (see prim.cu), their pass epoch,
  // its histogram and tile counters, and a failed-wait flag in mapped pinned
  // host memory (the device writes it; the host reads it after a sync)
  unsigned long long* sort_status = nullptr;
  int64_t sort_status_cap = 0;
  uint32_t sort_epoch = 0;
  unsigned long long* sort_aux = nullptr;
  uint64_t lb_ticket = 0;  // tickets taken so far from the auxiliary block's counter
  int* h_sort_err = nullptr;
  int* d_sort_err = nullptr;
  // small pinned host block for per-round read-back
  lgc::Counters* h_counters = nullptr;
  lgc::Counters* d_counters = nullptr;
  int64_t* h_scratch = nullptr;  // pinned, 8 int64
  // residual of the last PR-Nibble call (host svec), kept under LGC_OPT_TRACE
  lgc_svec* last_residual = nullptr;
  // trace of the last call
  std::vector<int64_t> trace_sizes;
  std::vector<int32_t> trace_ids;
  // endpoints of the last rand-HK-PR call (device, owned)
  int32_t* d_endpoints = nullptr;
  int64_t n_endpoints = 0;
  lgc::Serve* serve = nullptr;
  // measurement
  int64_t n_launches = 0;
  bool profile = false;
  struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> event_pool;
  lgc_kernel_profile prof[LGC_PROF_COUNT] = {};
};

// Work item of a pull round: edges [beg, beg + len) of heavy vertex w, the
// item's vertex being heavy[h] and having nparts items in all.
struct __align__(32) PullItem {
  int64_t beg;
  int32_t w, h, len, nparts;
  int64_t pad;
};

// A vertex of degree 1..kPullLight for the atomic pull gather: its list
// [beg, beg + d).  The graph keeps them grouped by degree (highest first), so
// the threads of a warp walk lists of one length.
struct __align__(16) LightItem {
  int64_t beg;
  int32_t w, d;
};

// A 256-edge segment of a big vertex's list (deterministic pull rounds):
// edges [beg, beg + len) of vertex w, the big vertex's index `big`.
struct __align__(32) DetSeg {
  int64_t beg;
  int32_t w, len, big, pad0;
  int64_t pad1;
};

struct lgc_graph {
  lgc_ctx* ctx = nullptr;
  uint64_t serial = 0;  // unique per graph of the process (a freed graph's address may recur)
  int64_t n = 0, nnz = 0;
  int64_t* off = nullptr;  // device, n + 1
  int32_t* col = nullptr;  // device, nnz
  int32_t* deg = nullptr;  // device, n (int32 degree, read where off[] pairs would cost more)
  int32_t max_deg = 0;
  std::vector<int32_t> hdeg;  // host copy of deg (seeds are checked without a device read)
  int pull_batch = 8;          // edges per lane per batch in heavy pull gathers (tuned)
  int pull_group = 32;         // lanes per work item in heavy pull gathers (tuned)
  int pull_share = 16;         // bytes per gathered share in atomic pull gathers (tuned)
  int64_t batch_handoff = 0;   // batched PR-Nibble hand-off threshold (tuned; 0: untuned)
  int pull_light = 32;         // atomic pull rounds: degree <= pull_light one thread each (tuned)
  // vertices of degree > pull_light in ascending id, for the atomic pull edge phase
  int32_t* heavy = nullptr;
  int64_t nheavy = 0;
  // their adjacency cut into work items of at most kPullItem edges (one
  // 32-byte record each, so a warp learns everything about its item from one
  // load)
  PullItem* items = nullptr;
  int64_t nitems = 0;
  // vertices of degree in (kPullLight, kDetBig], longest lists first (one
  // lane each folds its list in the deterministic pull)
  int32_t* det_mid = nullptr;
  int64_t ndet_mid = 0;
  // vertices of degree > kDetBig, whose deterministic fold runs segment-
  // parallel: their ids, the first of their segments (nbig + 1 prefix), and
  // the 256-edge segments
  int32_t* big_w = nullptr;
  int64_t* big_seg0 = nullptr;
  int64_t nbig = 0;
  DetSeg* segs = nullptr;
  int64_t nsegs = 0;
  // vertices of degree 1..pull_light grouped by degree (atomic pull rounds)
  LightItem* light = nullptr;
  int64_t nlight = 0;
  // the deterministic pull's own list of vertices of degree 1..kPullLight
  // (its light lists fold in one thread, so its bin stays at kPullLight);
  // the atomic list itself while pull_light == kPullLight
  LightItem* light_det = nullptr;
  int64_t nlight_det = 0;
};

namespace lgc {
// A pull round handles vertices of degree <= kPullLight with one thread each
// and the rest in work items of at most kPullItem edges.
constexpr int kPullLight = 32;  // default of lgc_graph::pull_light; the deterministic bin
constexpr int kDetBig = 1024;  // longer lists fold segment-parallel in deterministic mode
constexpr int kDetSeg = 256;
constexpr int kPullItem = 4096;
}  // namespace lgc

namespace lgc {

// Stream-ordered device allocation (CUDA memory pool of the device; freed
// memory is cached by the pool).
int dalloc(lgc_ctx* ctx, void** p, size_t bytes);
void dfree(lgc_ctx* ctx, void* p);

template <class T>
int dalloc_t(lgc_ctx* ctx, T** p, size_t count) {
  return dalloc(ctx, (void**)p, count * sizeof(T));
}

// A growable device buffer.
template <class T>
struct DBuf {
  T* ptr = nullptr;
  size_t cap = 0;
  int reserve(lgc_ctx* ctx, size_t count) {
    if (count <= cap) return LGC_OK;
    size_t nc = cap ? cap : 1024;
    while (nc < count) nc *= 2;
    if (ptr) dfree(ctx, ptr);
    ptr = nullptr;
    cap = 0;
    LGC_TRY(dalloc_t(ctx, &ptr, nc));
    cap = nc;
    return LGC_OK;
  }
  // As reserve, keeping the first `keep` elements when it reallocates.
  int reserve_keep(lgc_ctx* ctx, size_t count, size_t keep) {
    if (count <= cap) return LGC_OK;
    size_t nc = cap ? cap : 1024;
    while (nc < count) nc *= 2;
    T* np = nullptr;
    LGC_TRY(dalloc_t(ctx, &np, nc));
    if (keep && ptr &&
        cudaMemcpyAsync(np, ptr, sizeof(T) * keep, cudaMemcpyDeviceToDevice, ctx->stream) !=
            cudaSuccess) {
      dfree(ctx, np);
      return LGC_ECUDA;
    }
    if (ptr) dfree(ctx, ptr);
    ptr = np;
    cap = nc;
    return LGC_OK;
  }
  void release(lgc_ctx* ctx) {
    if (ptr) dfree(ctx, ptr);
    ptr = nullptr;
    cap = 0;
  }
};

// Allocates a cleared hashed table with capacity >= min_cap (power of two).
int table_create(lgc_ctx* ctx, Table* T, int64_t min_cap, bool with_p);
// Allocates a cleared dense table over n vertices.
int table_create_dense(lgc_ctx* ctx, Table* T, int64_t n, bool with_p);
// Converts a hashed table to the dense form over n vertices; frontier slots
// fs[0..nf) are re-resolved (they become the vertex ids).
int table_to_dense(lgc_ctx* ctx, Table* T, int64_t n, const int32_t* fv, int32_t* fs,
                   int64_t nf);
// Makes *T an empty table able to take `need` keys: dense if need >= n/8,
// else hashed at load <= 1/2 (reusing the allocation when it fits).
int table_fresh(lgc_ctx* ctx, Table* T, int64_t need, int64_t n, bool with_p);
// A set that may reach n/8 keys is kept dense.
inline bool want_dense(const lgc_ctx* ctx, int64_t need, int64_t n) {
  if (ctx->table_form == 1) return false;
  if (ctx->table_form == 2) return true;
  return need >= n / 8 && n >= 1024;
}
void table_destroy(lgc_ctx* ctx, Table* T);
int table_clear(lgc_ctx* ctx, Table* T);
// Rehashes into a table of capacity >= new_cap; the frontier slots fs[0..nf)
// (if given) are re-resolved from their vertex ids fv.
int table_grow(lgc_ctx* ctx, Table* T, int64_t new_cap, const int32_t* fv, int32_t* fs,
               int64_t nf);
int64_t pow2_at_least(int64_t x);

// Library-owned outputs carry their context for release.
// Host memory for results: page-locked blocks from a process-wide pool (so
// device-to-host copies run at the link's full speed and a host result does
// not depend on the context that made it), ordinary heap memory if
// page-locking fails.  Freed blocks are kept for reuse, up to 4 GB.
void* host_alloc(size_t bytes);
void host_free(void* p);

struct SvecBox {
  lgc_svec pub;
  lgc_ctx* ctx;
};
struct ClusterBox {
  lgc_cluster pub;
  lgc_ctx* ctx;
};
// Builds an lgc_svec from device arrays (copied into a fresh allocation,
// on the device or the host according to on_device).
int make_svec(lgc_ctx* ctx, const int32_t* d_idx, const double* d_val, int64_t nnz,
              bool on_device, lgc_svec** out);

// Extracts {(key - 1, value) : value > 0} from a table, sorted by vertex id.
// vals == nullptr uses T.s[].val, else vals[slot].
int table_extract_sorted(lgc_ctx* ctx, const Table& T, const double* vals, int64_t n_vertices,
                         int32_t** d_idx, double** d_val, int64_t* nnz,
                         bool positive_only = true);

// Algorithm drivers (diffuse.cu, rwalk.cu, sweep.cu).  ctx supplies the
// stream and scratch; g is read-only and may be shared by several contexts.
int run_prnibble(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_prnibble_params* prm,
                 lgc_svec** p, lgc_stats* st, lgc_svec** r_out);
int run_nibble(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_nibble_params* prm, lgc_svec** p,
               lgc_stats* st);
int run_hkpr(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_hkpr_params* prm, lgc_svec** p,
             lgc_stats* st);
int run_rand_hkpr(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_rand_hkpr_params* prm,
                  lgc_svec** p, lgc_stats* st);
int autotune_pull(lgc_ctx* ctx, lgc_graph* g);
int rebuild_pull_lists(lgc_ctx* ctx, lgc_graph* g, int L);
int run_prnibble_set(lgc_ctx* ctx, lgc_graph* g, int64_t k, const int32_t* seeds,
                     const double* weights, double beta, const lgc_prnibble_params* prm,
                     lgc_svec** p, lgc_stats* st_out, lgc_svec** r_out);
// Continues PR-Nibble for one seed from the state batched rounds left: its
// hashed table src (r in the slot values, p in src.p; copied, same capacity
// so the frontier's slots stay valid), its frontier d_fv/d_fs (nf entries,
// ascending in deterministic mode) with degree sum E, the table's key count,
// and the rounds, pushes and pushed edges run so far.  The result and the
// counters are those of one uninterrupted run (status_detail
// LGC_EMAXROUNDS when the round limit ended it).
int run_prnibble_from(lgc_ctx* ctx, lgc_graph* g, const Table& src, const int32_t* d_fv,
                      const int32_t* d_fs, int64_t nf, int64_t E, int64_t count,
                      const lgc_prnibble_params* prm, const lgc_stats& so_far, lgc_svec** p,
                      lgc_stats* st_out);
int run_sweep(lgc_ctx* ctx, lgc_graph* g, const lgc_svec* p, lgc_cluster** out);
int run_sweep_batch(lgc_ctx* ctx, lgc_graph* g, int64_t B, const lgc_svec* const* ps,
                    lgc_cluster** out);
// d(x) of a seed, checked: LGC_EINVAL unless 0 <= x < n and d(x) >= 1.
int validate_seed(lgc_ctx* ctx, lgc_graph* g, int32_t x, int64_t* dx);
int ctx_init(lgc_ctx* ctx, int device, cudaStream_t stream);
void ctx_fini(lgc_ctx* ctx);

double now_seconds();

// Profiling scope: records CUDA events around the launches made between
// begin and end when ctx->profile is set, and counts launches always.
struct ProfScope {
  lgc_ctx* ctx;
  int kernel;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(lgc_ctx* c, int k, double b);
  ~ProfScope();
};
cudaEvent_t take_event(lgc_ctx* ctx);
// Folds completed event pairs into ctx->prof (synchronizes the stream).
void profile_collect(lgc_ctx* ctx);

}  // namespace lgc

// Counts one kernel launch on ctx.
#define LGC_COUNT_LAUNCH(ctx) ((ctx)->n_launches++)

namespace lgc {
// The flags of the context's look-back launches (one-launch scans, sorts
// and compactions), once: LGC_ETIMEOUT if a look-back wait gave up, else
// LGC_ECUDA if a partial sum left the status words' range or a launch's
// tiles were out of step.  Call after the context's stream has synchronised.
inline int sort_check(lgc_ctx* ctx) {
  volatile int* e = ctx->h_sort_err;
  if (e && *e) {
    const int f = *e;
    *e = 0;
    return (f & 1) ? LGC_ETIMEOUT : LGC_ECUDA;
  }
  return LGC_OK;
}
}  // namespace lgc

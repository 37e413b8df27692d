// Host helpers: memory, hash tables, sparse-vector outputs.
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <new>

#include <unordered_map>

#include "common.cuh"
#include "prim.cuh"

namespace lgc {

static thread_local char g_last_err[256];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_err, sizeof g_last_err, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file,
           line);
}

int validate_seed(lgc_ctx* ctx, lgc_graph* g, int32_t x, int64_t* dx) {
  (void)ctx;
  if (!g || x < 0 || x >= g->n) return LGC_EINVAL;
  *dx = g->hdeg[x];
  return *dx >= 1 ? LGC_OK : LGC_EINVAL;
}

int ctx_init(lgc_ctx* ctx, int device, cudaStream_t stream) {
  ctx->device = device;
  LGC_CUDA_TRY(cudaSetDevice(device));
  LGC_CUDA_TRY(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device));
  if (stream) {
    ctx->stream = stream;
    ctx->own_stream = false;
  } else {
    LGC_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  // keep freed device memory in the pool between calls
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  LGC_CUDA_TRY(cudaHostAlloc((void**)&ctx->h_counters, sizeof(Counters), cudaHostAllocDefault));
  LGC_CUDA_TRY(cudaHostAlloc((void**)&ctx->h_scratch, 8 * sizeof(int64_t), cudaHostAllocDefault));
  LGC_CUDA_TRY(cudaMalloc((void**)&ctx->d_counters, sizeof(Counters)));
  LGC_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(Counters), ctx->stream));
  LGC_CUDA_TRY(cudaHostAlloc((void**)&ctx->h_sort_err, sizeof(int), cudaHostAllocMapped));
  *ctx->h_sort_err = 0;
  LGC_CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->d_sort_err, ctx->h_sort_err, 0));
  return LGC_OK;
}

void ctx_fini(lgc_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  profile_collect(ctx);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  ctx->event_pool.clear();
  if (ctx->d_endpoints) cudaFree(ctx->d_endpoints);
  dfree(ctx, ctx->sort_status);
  dfree(ctx, ctx->sort_aux);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->h_sort_err) cudaFreeHost(ctx->h_sort_err);
  ctx->sort_status = nullptr;
  ctx->sort_aux = nullptr;
  ctx->sort_status_cap = 0;
  ctx->h_sort_err = nullptr;
  ctx->d_sort_err = nullptr;
  if (ctx->d_counters) cudaFree(ctx->d_counters);
  if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
  if (ctx->h_scratch) cudaFreeHost(ctx->h_scratch);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  ctx->d_endpoints = nullptr;
  ctx->d_counters = nullptr;
  ctx->h_counters = nullptr;
  ctx->h_scratch = nullptr;
  ctx->stream = nullptr;
}

cudaEvent_t take_event(lgc_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

ProfScope::ProfScope(lgc_ctx* c, int k, double b) : ctx(c), kernel(k), bytes(b) {
  if (ctx->profile) {
    a = take_event(ctx);
    if (a) cudaEventRecord(a, ctx->stream);
  }
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b = take_event(ctx);
  if (!b) return;
  cudaEventRecord(b, ctx->stream);
  ctx->prof_pending.push_back({kernel, a, b, bytes});
}

void profile_collect(lgc_ctx* ctx) {
  if (ctx->prof_pending.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->prof[r.kernel].launches += 1;
      ctx->prof[r.kernel].ms += ms;
      ctx->prof[r.kernel].bytes += r.bytes;
    } else {
      cudaGetLastError();
    }
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  ctx->prof_pending.clear();
}

double now_seconds() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

int dalloc(lgc_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->alloc_fns.alloc) {
    *p = ctx->alloc_fns.alloc(bytes, (void*)ctx->stream, ctx->alloc_fns.user);
    return *p ? LGC_OK : LGC_ENOMEM;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? LGC_ENOMEM : LGC_ECUDA;
  }
  return LGC_OK;
}

void dfree(lgc_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->alloc_fns.free) ctx->alloc_fns.free(p, (void*)ctx->stream, ctx->alloc_fns.user);
  else cudaFreeAsync(p, ctx->stream);
}

int64_t pow2_at_least(int64_t x) {
  int64_t c = 1;
  while (c < x) c <<= 1;
  return c;
}

int table_create(lgc_ctx* ctx, Table* T, int64_t min_cap, bool with_p) {
  int64_t cap = pow2_at_least(min_cap < 64 ? 64 : min_cap);
  int lg = 0;
  while (((int64_t)1 << lg) < cap) lg++;
  if (lg > 31) return LGC_EINVAL;
  *T = Table();
  T->cap = cap;
  T->shift = 32 - lg;
  LGC_TRY(dalloc_t(ctx, &T->s, (size_t)cap));
  if (with_p) {
    int s = dalloc_t(ctx, &T->p, (size_t)cap);
    if (s != LGC_OK) {
      dfree(ctx, T->s);
      T->s = nullptr;
      return s;
    }
  }
  return table_clear(ctx, T);
}

int table_create_dense(lgc_ctx* ctx, Table* T, int64_t n, bool with_p) {
  *T = Table();
  T->dense = 1;
  T->cap = n;
  int s = dalloc_t(ctx, &T->dval, (size_t)n);
  if (s == LGC_OK) s = dalloc_t(ctx, &T->bits, (size_t)((n + 31) / 32));
  if (s == LGC_OK && with_p) s = dalloc_t(ctx, &T->p, (size_t)n);
  if (s != LGC_OK) {
    table_destroy(ctx, T);
    return s;
  }
  return table_clear(ctx, T);
}

void table_destroy(lgc_ctx* ctx, Table* T) {
  dfree(ctx, T->s);
  dfree(ctx, T->p);
  dfree(ctx, T->dval);
  dfree(ctx, T->bits);
  *T = Table();
}

int table_clear(lgc_ctx* ctx, Table* T) {
  if (T->dense) {
    LGC_CUDA_TRY(cudaMemsetAsync(T->dval, 0, sizeof(double) * T->cap, ctx->stream));
    LGC_CUDA_TRY(cudaMemsetAsync(T->bits, 0, sizeof(uint32_t) * ((T->cap + 31) / 32),
                                 ctx->stream));
  } else {
    LGC_CUDA_TRY(cudaMemsetAsync(T->s, 0, sizeof(Slot) * T->cap, ctx->stream));
  }
  if (T->p) LGC_CUDA_TRY(cudaMemsetAsync(T->p, 0, sizeof(double) * T->cap, ctx->stream));
  return LGC_OK;
}

int table_fresh(lgc_ctx* ctx, Table* T, int64_t need, int64_t n, bool with_p) {
  if (want_dense(ctx, need, n)) {
    if (T->dense && T->cap == n && (T->p != nullptr) == with_p) return table_clear(ctx, T);
    table_destroy(ctx, T);
    return table_create_dense(ctx, T, n, with_p);
  }
  const int64_t want = pow2_at_least(2 * (need < 32 ? 32 : need));
  if (!T->dense && T->s && T->cap >= want && T->cap <= 8 * want && (T->p != nullptr) == with_p)
    return table_clear(ctx, T);
  table_destroy(ctx, T);
  return table_create(ctx, T, want, with_p);
}

namespace {

__global__ void rehash_kernel(Table from, Table to, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < from.cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    Slot s = from.s[i];
    if (s.key == 0) continue;
    int ins = 0;
    int64_t j = ht_find_or_insert(to, s.key - 1, &ins, err);
    if (j < 0) continue;
    to.s[j].aux = s.aux;
    to.s[j].val = s.val;
    if (from.p) to.p[j] = from.p[i];
  }
}

__global__ void to_dense_kernel(Table from, Table to) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < from.cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    Slot s = from.s[i];
    if (s.key == 0) continue;
    const int32_t v = s.key - 1;
    to.dval[v] = s.val;
    if (from.p) to.p[v] = from.p[i];
    atomicOr(&to.bits[v >> 5], 1u << (v & 31));
  }
}

__global__ void reresolve_kernel(Table T, const int32_t* fv, int32_t* fs, int64_t nf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x)
    fs[i] = (int32_t)tb_find(T, fv[i]);
}

__global__ void extract_kernel(Table T, const double* vals, Counters* C, uint32_t* keys,
                               double* out, int positive_only) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T.cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t k = T.s[i].key;
    double v = vals ? vals[i] : T.s[i].val;
    if (k != 0 && (v > 0.0 || !positive_only)) {
      int pos = atomicAdd(&C->next_size, 1);
      keys[pos] = (uint32_t)(k - 1);
      out[pos] = v;
    }
  }
}

// Dense extraction in vertex order: count the kept keys of each bitmap word,
// then (after a scan of the counts) write them in ascending id.
__device__ inline uint32_t dense_kept(const Table& T, const double* vals, int64_t w, int64_t n,
                                      int positive_only) {
  uint32_t m = T.bits[w];
  if (positive_only) {
    uint32_t k = 0;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int64_t v = w * 32 + b;
      if (v < n && (vals ? vals[v] : T.dval[v]) > 0.0) k |= 1u << b;
    }
    return k;
  }
  return m;
}

__global__ void dense_count_kernel(Table T, const double* vals, int64_t n, int positive_only,
                                   int64_t* cnt) {
  const int64_t words = (n + 31) / 32;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popc(dense_kept(T, vals, w, n, positive_only));
}

__global__ void dense_write_kernel(Table T, const double* vals, int64_t n, int positive_only,
                                   const int64_t* pos, uint32_t* keys, double* out) {
  const int64_t words = (n + 31) / 32;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t m = dense_kept(T, vals, w, n, positive_only);
    int64_t at = pos[w];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int64_t v = w * 32 + b;
      keys[at] = (uint32_t)v;
      out[at] = vals ? vals[v] : T.dval[v];
      at++;
    }
  }
}

}  // namespace

int table_to_dense(lgc_ctx* ctx, Table* T, int64_t n, const int32_t* fv, int32_t* fs,
                   int64_t nf) {
  if (T->dense) return LGC_OK;
  Table nt;
  LGC_TRY(table_create_dense(ctx, &nt, n, T->p != nullptr));
  to_dense_kernel<<<grid_for(T->cap), kBlock, 0, ctx->stream>>>(*T, nt);
  LGC_COUNT_LAUNCH(ctx);
  if (nf > 0 && fv && fs) {
    reresolve_kernel<<<grid_for(nf), kBlock, 0, ctx->stream>>>(nt, fv, fs, nf);
    LGC_COUNT_LAUNCH(ctx);
  }
  LGC_CUDA_TRY(cudaGetLastError());
  table_destroy(ctx, T);
  *T = nt;
  return LGC_OK;
}

int table_grow(lgc_ctx* ctx, Table* T, int64_t new_cap, const int32_t* fv, int32_t* fs,
               int64_t nf) {
  Table nt;
  LGC_TRY(table_create(ctx, &nt, new_cap, T->p != nullptr));
  LGC_CUDA_TRY(cudaMemsetAsync(&ctx->d_counters->err, 0, sizeof(int), ctx->stream));
  rehash_kernel<<<grid_for(T->cap), kBlock, 0, ctx->stream>>>(*T, nt, &ctx->d_counters->err);
  LGC_COUNT_LAUNCH(ctx);
  if (nf > 0 && fv && fs) {
    reresolve_kernel<<<grid_for(nf), kBlock, 0, ctx->stream>>>(nt, fv, fs, nf);
    LGC_COUNT_LAUNCH(ctx);
  }
  LGC_CUDA_TRY(cudaGetLastError());
  table_destroy(ctx, T);
  *T = nt;
  return LGC_OK;
}

int table_extract_sorted(lgc_ctx* ctx, const Table& T, const double* vals, int64_t n_vertices,
                         int32_t** d_idx, double** d_val, int64_t* nnz, bool positive_only) {
  cudaStream_t st = ctx->stream;
  *d_idx = nullptr;
  *d_val = nullptr;
  *nnz = 0;
  if (T.dense) {
    const int64_t n = T.cap, words = (n + 31) / 32;
    int64_t *cnt = nullptr, *tot = nullptr;
    uint32_t* k = nullptr;
    double* v = nullptr;
    int s = dalloc_t(ctx, &cnt, words);
    if (s == LGC_OK) s = dalloc_t(ctx, &tot, 1);
    if (s == LGC_OK) {
      dense_count_kernel<<<grid_for(words), kBlock, 0, st>>>(T, vals, n, positive_only, cnt);
      LGC_COUNT_LAUNCH(ctx);
      s = scan_i64(ctx, cnt, cnt, words, false, tot);
    }
    int64_t count = 0;
    if (s == LGC_OK) {
      if (cudaMemcpyAsync(ctx->h_scratch, tot, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        s = LGC_ECUDA;
      else
        count = ctx->h_scratch[0];
    }
    if (s == LGC_OK) s = dalloc_t(ctx, &k, count);
    if (s == LGC_OK) s = dalloc_t(ctx, &v, count);
    if (s == LGC_OK) {
      dense_write_kernel<<<grid_for(words), kBlock, 0, st>>>(T, vals, n, positive_only, cnt, k, v);
      LGC_COUNT_LAUNCH(ctx);
      if (cudaGetLastError() != cudaSuccess) s = LGC_ECUDA;
    }
    dfree(ctx, cnt);
    dfree(ctx, tot);
    if (s != LGC_OK) {
      dfree(ctx, k);
      dfree(ctx, v);
      return s;
    }
    *d_idx = (int32_t*)k;
    *d_val = v;
    *nnz = count;
    return LGC_OK;
  }
  LGC_CUDA_TRY(cudaMemsetAsync(&ctx->d_counters->next_size, 0, sizeof(int32_t), st));
  // at most min(cap, n) keys
  int64_t maxk = T.cap < n_vertices ? T.cap : n_vertices;
  uint32_t *k = nullptr, *kt = nullptr;
  double *v = nullptr, *vt = nullptr;
  int s = dalloc_t(ctx, &k, maxk);
  if (s == LGC_OK) s = dalloc_t(ctx, &kt, maxk);
  if (s == LGC_OK) s = dalloc_t(ctx, &v, maxk);
  if (s == LGC_OK) s = dalloc_t(ctx, &vt, maxk);
  if (s == LGC_OK) {
    extract_kernel<<<grid_for(T.cap), kBlock, 0, st>>>(T, vals, ctx->d_counters, k, v,
                                                        positive_only ? 1 : 0);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaGetLastError() != cudaSuccess) s = LGC_ECUDA;
  }
  int32_t count = 0;
  if (s == LGC_OK) {
    if (cudaMemcpyAsync(ctx->h_scratch, &ctx->d_counters->next_size, sizeof(int32_t),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = LGC_ECUDA;
    else
      count = *(int32_t*)ctx->h_scratch;
  }
  if (s == LGC_OK) s = radix_sort_u32_f64(ctx, k, v, kt, vt, count, bits_for(n_vertices));
  dfree(ctx, kt);
  dfree(ctx, vt);
  if (s != LGC_OK) {
    dfree(ctx, k);
    dfree(ctx, v);
    return s;
  }
  *d_idx = (int32_t*)k;
  *d_val = v;
  *nnz = count;
  return LGC_OK;
}

namespace {
struct HostPool {
  std::mutex mu;
  std::unordered_map<void*, std::pair<size_t, bool>> info;  // block -> (size class, pinned)
  std::map<size_t, std::vector<void*>> spare;
  size_t spare_bytes = 0;
};
// never destroyed: host results may be freed while the process exits
HostPool& host_pool() {
  static HostPool* p = new HostPool();
  return *p;
}
constexpr size_t kHostSpareMax = size_t{4} << 30;
}  // namespace

void* host_alloc(size_t bytes) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  HostPool& P = host_pool();
  {
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.spare.find(c);
    if (it != P.spare.end() && !it->second.empty()) {
      void* q = it->second.back();
      it->second.pop_back();
      P.spare_bytes -= c;
      return q;
    }
  }
  void* q = nullptr;
  bool pinned = true;
  if (cudaHostAlloc(&q, c, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    q = malloc(c);
    pinned = false;
    if (!q) return nullptr;
  }
  std::lock_guard<std::mutex> lk(P.mu);
  P.info[q] = {c, pinned};
  return q;
}

void host_free(void* q) {
  if (!q) return;
  HostPool& P = host_pool();
  std::unique_lock<std::mutex> lk(P.mu);
  auto it = P.info.find(q);
  if (it == P.info.end()) return;  // not ours
  const size_t c = it->second.first;
  const bool pinned = it->second.second;
  if (pinned && P.spare_bytes + c <= kHostSpareMax) {
    P.spare[c].push_back(q);
    P.spare_bytes += c;
    return;
  }
  P.info.erase(it);
  lk.unlock();
  if (pinned) cudaFreeHost(q);
  else free(q);
}

int make_svec(lgc_ctx* ctx, const int32_t* d_idx, const double* d_val, int64_t nnz,
              bool on_device, lgc_svec** out) {
  *out = nullptr;
  SvecBox* b = new (std::nothrow) SvecBox();
  if (!b) return LGC_ENOMEM;
  b->ctx = ctx;
  b->pub.nnz = nnz;
  b->pub.on_device = on_device ? 1 : 0;
  if (on_device) {
    int s = dalloc_t(ctx, &b->pub.idx, nnz);
    if (s == LGC_OK) s = dalloc_t(ctx, &b->pub.val, nnz);
    if (s != LGC_OK) {
      dfree(ctx, b->pub.idx);
      delete b;
      return s;
    }
    if (nnz) {
      LGC_CUDA_TRY(cudaMemcpyAsync(b->pub.idx, d_idx, 4 * nnz, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
      LGC_CUDA_TRY(cudaMemcpyAsync(b->pub.val, d_val, 8 * nnz, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    }
  } else {
    b->pub.idx = (int32_t*)host_alloc(4 * (nnz ? nnz : 1));
    b->pub.val = (double*)host_alloc(8 * (nnz ? nnz : 1));
    if (!b->pub.idx || !b->pub.val) {
      host_free(b->pub.idx);
      host_free(b->pub.val);
      delete b;
      return LGC_ENOMEM;
    }
    if (nnz) {
      LGC_CUDA_TRY(cudaMemcpyAsync(b->pub.idx, d_idx, 4 * nnz, cudaMemcpyDeviceToHost,
                                   ctx->stream));
      LGC_CUDA_TRY(cudaMemcpyAsync(b->pub.val, d_val, 8 * nnz, cudaMemcpyDeviceToHost,
                                   ctx->stream));
      LGC_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
  }
  *out = &b->pub;
  return LGC_OK;
}

}  // namespace lgc

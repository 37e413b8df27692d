// Public C ABI (include/lgc.h): contexts, graphs, entry points, releases,
// and the request loop behind lgc_submit / lgc_poll.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>

#include "batch.cuh"
#include "common.cuh"
#include "prim.cuh"

using namespace lgc;

namespace {

__global__ void degree_kernel(const int64_t* __restrict__ off, int64_t n,
                              int32_t* __restrict__ deg, int* maxdeg) {
  int m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = off[v + 1] - off[v];
    deg[v] = (int32_t)d;
    m = max(m, (int)d);
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, m);
}

// Flags: 1 offsets not monotone / out of range, 2 column out of range,
// 4 self loop, 8 adjacency not strictly ascending (unsorted or duplicate),
// 16 asymmetric (w lists v does not hold for v lists w).
__global__ void validate_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                int64_t n, int64_t nnz, int* flags) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[v], e = off[v + 1];
    if (b < 0 || e < b || e > nnz) {
      atomicOr(flags, 1);
      continue;
    }
    for (int64_t k = b; k < e; k++) {
      const int32_t w = col[k];
      if (w < 0 || w >= n) {
        atomicOr(flags, 2);
        continue;
      }
      if (w == v) atomicOr(flags, 4);
      if (k > b && col[k - 1] >= w) atomicOr(flags, 8);
      // binary search v in w's list
      int64_t lo = off[w], hi = off[w + 1];
      bool found = false;
      if (lo >= 0 && hi <= nnz && lo <= hi) {
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          int32_t c = col[mid];
          if (c == v) {
            found = true;
            break;
          }
          if (c < v) lo = mid + 1;
          else hi = mid;
        }
      }
      if (!found) atomicOr(flags, 16);
    }
  }
}

__global__ void heavy_flag_kernel(const int32_t* __restrict__ deg, int64_t n, int light,
                                  int64_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = deg[v] > light ? 1 : 0;
}

__global__ void heavy_write_kernel(const int32_t* __restrict__ deg, int64_t n, int light,
                                   const int64_t* __restrict__ pos, int32_t* __restrict__ out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (deg[v] > light) out[pos[v]] = (int32_t)v;
}

__global__ void items_count_kernel(const int32_t* __restrict__ heavy, int64_t nh,
                                   const int32_t* __restrict__ deg, int64_t* __restrict__ cnt) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh;
       h += (int64_t)gridDim.x * blockDim.x)
    cnt[h] = ((int64_t)deg[heavy[h]] + kPullItem - 1) / kPullItem;
}

__global__ void items_fill_kernel(const int32_t* __restrict__ heavy, int64_t nh,
                                  const int64_t* __restrict__ off, const int64_t* __restrict__ pos,
                                  PullItem* __restrict__ items) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh;
       h += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = heavy[h];
    const int64_t o0 = off[w], d = off[w + 1] - o0;
    const int32_t parts = (int32_t)((d + kPullItem - 1) / kPullItem);
    for (int32_t k = 0; k < parts; k++) {
      PullItem it;
      it.beg = o0 + (int64_t)k * kPullItem;
      it.w = w;
      it.h = (int32_t)h;
      it.len = (int32_t)min((int64_t)kPullItem, d - (int64_t)k * kPullItem);
      it.nparts = parts;
      it.pad = 0;
      items[pos[h] + k] = it;
    }
  }
}

__global__ void gather_off_kernel(const int32_t* __restrict__ ids, int64_t k,
                                  const int64_t* __restrict__ off, int64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = off[ids[i]];
}

// The deterministic pull's vertices of degree (kPullLight, kDetBig], and those
// of degree > kDetBig with their 256-edge segments (built on the host from the
// degree copy; only their list starts are read back).
int build_big_segments(lgc_ctx* ctx, lgc_graph* g) {
  cudaStream_t s = ctx->stream;
  {
    std::vector<int32_t> mid;
    for (int64_t v = 0; v < g->n; v++)
      if (g->hdeg[v] > kPullLight && g->hdeg[v] <= kDetBig) mid.push_back((int32_t)v);
    std::stable_sort(mid.begin(), mid.end(),
                     [&](int32_t a, int32_t b) { return g->hdeg[a] > g->hdeg[b]; });
    g->ndet_mid = (int64_t)mid.size();
    if (g->ndet_mid > 0) {
      LGC_TRY(dalloc_t(ctx, &g->det_mid, g->ndet_mid));
      LGC_CUDA_TRY(cudaMemcpyAsync(g->det_mid, mid.data(), 4 * g->ndet_mid,
                                   cudaMemcpyHostToDevice, s));
      LGC_CUDA_TRY(cudaStreamSynchronize(s));  // mid goes out of scope
    }
  }
  std::vector<int32_t> bw;
  for (int64_t v = 0; v < g->n; v++)
    if (g->hdeg[v] > kDetBig) bw.push_back((int32_t)v);
  g->nbig = (int64_t)bw.size();
  if (g->nbig == 0) return LGC_OK;
  std::vector<int64_t> starts(g->nbig), seg0(g->nbig + 1, 0);
  int64_t* d_starts = nullptr;
  LGC_TRY(dalloc_t(ctx, &g->big_w, g->nbig));
  LGC_TRY(dalloc_t(ctx, &d_starts, g->nbig));
  LGC_CUDA_TRY(cudaMemcpyAsync(g->big_w, bw.data(), 4 * g->nbig, cudaMemcpyHostToDevice, s));
  gather_off_kernel<<<grid_for(g->nbig), kBlock, 0, s>>>(g->big_w, g->nbig, g->off, d_starts);
  LGC_COUNT_LAUNCH(ctx);
  LGC_CUDA_TRY(cudaMemcpyAsync(starts.data(), d_starts, 8 * g->nbig, cudaMemcpyDeviceToHost, s));
  LGC_CUDA_TRY(cudaStreamSynchronize(s));
  dfree(ctx, d_starts);
  for (int64_t b = 0; b < g->nbig; b++)
    seg0[b + 1] = seg0[b] + (g->hdeg[bw[b]] + kDetSeg - 1) / kDetSeg;
  g->nsegs = seg0[g->nbig];
  std::vector<DetSeg> segs(g->nsegs);
  for (int64_t b = 0; b < g->nbig; b++) {
    const int64_t d = g->hdeg[bw[b]];
    for (int64_t k = 0; k < seg0[b + 1] - seg0[b]; k++) {
      DetSeg& S = segs[seg0[b] + k];
      S = DetSeg{};
      S.beg = starts[b] + k * kDetSeg;
      S.w = bw[b];
      S.len = (int32_t)std::min<int64_t>(kDetSeg, d - k * kDetSeg);
      S.big = (int32_t)b;
    }
  }
  LGC_TRY(dalloc_t(ctx, &g->big_seg0, g->nbig + 1));
  LGC_TRY(dalloc_t(ctx, &g->segs, g->nsegs));
  LGC_CUDA_TRY(cudaMemcpyAsync(g->big_seg0, seg0.data(), 8 * (g->nbig + 1),
                               cudaMemcpyHostToDevice, s));
  LGC_CUDA_TRY(cudaMemcpyAsync(g->segs, segs.data(), sizeof(DetSeg) * g->nsegs,
                               cudaMemcpyHostToDevice, s));
  LGC_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
  return LGC_OK;
}

__global__ void light_items_kernel(const int32_t* __restrict__ order, int64_t k,
                                   const int64_t* __restrict__ off, LightItem* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = order[i];
    const int64_t o0 = off[w];
    out[i] = LightItem{o0, w, (int32_t)(off[w + 1] - o0)};
  }
}

// The vertices of degree 1..L grouped by degree, highest first, ids
// ascending within a degree (a counting sort of the host degree copy), into
// *out (*nout entries).
int build_light_list(lgc_ctx* ctx, lgc_graph* g, int L, LightItem** out, int64_t* nout) {
  cudaStream_t s = ctx->stream;
  const int64_t n = g->n;
  std::vector<int64_t> cnt(L + 2, 0), at(L + 2, 0);
  int64_t k = 0;
  for (int64_t v = 0; v < n; v++)
    if (g->hdeg[v] >= 1 && g->hdeg[v] <= L) cnt[g->hdeg[v]]++;
  for (int d = L; d >= 1; d--) {
    at[d] = k;
    k += cnt[d];
  }
  *nout = k;
  if (k == 0) return LGC_OK;
  std::vector<int32_t> order;
  try {
    order.resize(k);
  } catch (...) {
    return LGC_ENOMEM;
  }
  for (int64_t v = 0; v < n; v++) {
    const int32_t d = g->hdeg[v];
    if (d >= 1 && d <= L) order[at[d]++] = (int32_t)v;
  }
  int32_t* d_order = nullptr;
  LGC_TRY(dalloc_t(ctx, &d_order, k));
  int st = dalloc_t(ctx, out, k);
  if (st == LGC_OK &&
      cudaMemcpyAsync(d_order, order.data(), 4 * k, cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = LGC_ECUDA;
  if (st == LGC_OK) {
    light_items_kernel<<<grid_for(k), kBlock, 0, s>>>(d_order, k, g->off, *out);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      st = LGC_ECUDA;  // (the host order goes out of scope)
  }
  dfree(ctx, d_order);
  return st;
}

// The atomic pull's light list (degree <= pull_light) and the deterministic
// pull's (degree <= kPullLight), shared while the two bins agree.
int build_light_items(lgc_ctx* ctx, lgc_graph* g) {
  LGC_TRY(build_light_list(ctx, g, g->pull_light, &g->light, &g->nlight));
  if (g->pull_light == kPullLight) {
    g->light_det = g->light;
    g->nlight_det = g->nlight;
    return LGC_OK;
  }
  return build_light_list(ctx, g, kPullLight, &g->light_det, &g->nlight_det);
}

// The vertices of degree > kPullLight, ascending, for pull rounds, and their
// adjacency cut into work items.
int build_heavy_list(lgc_ctx* ctx, lgc_graph* g) {
  cudaStream_t s = ctx->stream;
  const int64_t n = g->n;
  if (n == 0) return LGC_OK;
  int64_t *flag = nullptr, *tot = nullptr;
  int st = dalloc_t(ctx, &flag, n);
  if (st == LGC_OK) st = dalloc_t(ctx, &tot, 1);
  if (st == LGC_OK) {
    heavy_flag_kernel<<<grid_for(n), kBlock, 0, s>>>(g->deg, n, g->pull_light, flag);
    LGC_COUNT_LAUNCH(ctx);
    st = scan_i64(ctx, flag, flag, n, false, tot);
  }
  if (st == LGC_OK) {
    if (cudaMemcpyAsync(ctx->h_scratch, tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = LGC_ECUDA;
  }
  if (st == LGC_OK) {
    g->nheavy = ctx->h_scratch[0];
    st = dalloc_t(ctx, &g->heavy, g->nheavy);
  }
  if (st == LGC_OK && g->nheavy > 0) {
    heavy_write_kernel<<<grid_for(n), kBlock, 0, s>>>(g->deg, n, g->pull_light, flag, g->heavy);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaGetLastError() != cudaSuccess) st = LGC_ECUDA;
  }
  // work items of at most kPullItem edges over the heavy vertices' lists
  const int64_t nh = g->nheavy;
  if (st == LGC_OK && nh > 0) {
    items_count_kernel<<<grid_for(nh), kBlock, 0, s>>>(g->heavy, nh, g->deg, flag);
    LGC_COUNT_LAUNCH(ctx);
    st = scan_i64(ctx, flag, flag, nh, false, tot);
  }
  if (st == LGC_OK && nh > 0) {
    if (cudaMemcpyAsync(ctx->h_scratch, tot, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = LGC_ECUDA;
  }
  if (st == LGC_OK && nh > 0) {
    g->nitems = ctx->h_scratch[0];
    st = dalloc_t(ctx, &g->items, g->nitems);
  }
  if (st == LGC_OK && nh > 0) {
    items_fill_kernel<<<grid_for(nh), kBlock, 0, s>>>(g->heavy, nh, g->off, flag, g->items);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaGetLastError() != cudaSuccess) st = LGC_ECUDA;
  }
  dfree(ctx, flag);
  dfree(ctx, tot);
  return st;
}

}  // namespace

namespace lgc {

// Rebuilds the degree-binned vertex lists of the pull rounds for the atomic
// light threshold L: vertices of degree 1..L one thread each (grouped by
// degree), the others in work items.  The deterministic lists keep their own
// bins whatever L is: degree 1..kPullLight one thread each, (kPullLight,
// kDetBig] one lane each, longer ones segment-parallel.
int rebuild_pull_lists(lgc_ctx* ctx, lgc_graph* g, int L) {
  if (L < 4 || L > 256) return LGC_EINVAL;
  if (g->light_det != g->light) dfree(ctx, g->light_det);
  for (void* p : {(void*)g->heavy, (void*)g->items, (void*)g->big_w, (void*)g->big_seg0,
                  (void*)g->segs, (void*)g->det_mid, (void*)g->light})
    dfree(ctx, p);
  g->light_det = nullptr;
  g->nlight_det = 0;
  g->heavy = nullptr;
  g->items = nullptr;
  g->big_w = nullptr;
  g->big_seg0 = nullptr;
  g->segs = nullptr;
  g->det_mid = nullptr;
  g->light = nullptr;
  g->nheavy = g->nitems = g->nbig = g->nsegs = g->ndet_mid = g->nlight = 0;
  g->pull_light = L;
  LGC_TRY(build_heavy_list(ctx, g));
  LGC_TRY(build_big_segments(ctx, g));
  return build_light_items(ctx, g);
}

}  // namespace lgc

// ---------------------------------------------------------------------------
// request loop: continuous batching.  PR-Nibble requests go to one lane
// that runs all admitted PR-Nibble seeds' rounds together in a batch engine
// (a request that arrives while others run joins at the next round; a seed
// that finishes leaves with its result); the other requests run on worker
// contexts, each on its own stream, side by side with the lane.
// ---------------------------------------------------------------------------
namespace lgc {

struct Serve {
  struct Item {
    uint64_t ticket;
    lgc_graph* g;
    lgc_request req;
    double submit_s;
    int64_t bytes;
    int bypassed;  // times a later request was admitted before this one
  };
  lgc_ctx* owner = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Item> queue;  // worker requests
  std::deque<Item> prq;    // PR-Nibble requests for the lane
  std::map<uint64_t, lgc_result*> done;
  std::map<uint64_t, int> known;  // ticket -> 1 while queued or running
  int64_t inflight_bytes = 0;
  int inflight = 0;
  int64_t lane_bytes = 0;     // the lane's live table bytes after its last round
  int64_t lane_resident = 0;  // PR-Nibble requests admitted to the lane, not finished
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  std::vector<lgc_ctx*> wctx;
  std::thread lane;
  lgc_ctx* lane_ctx = nullptr;
  size_t max_queue = 1 << 20;
};

// A request may jump ahead of a queued one that does not fit; a queued
// request passed over this many times is admitted next, before anything
// behind it.
constexpr int kMaxBypass = 16;

// Device memory a worker request may need: its sparse sets in the form they
// take (hashed while they may stay below n/8 keys at load 1/2, else dense
// arrays with a presence bitmap), plus frontier and share arrays.
static int64_t request_bytes(const lgc_graph* g, const lgc_request& r) {
  const int64_t n = g->n;
  auto slots = [&](int64_t keys) { return pow2_at_least(2 * std::max<int64_t>(keys, 32)); };
  const int64_t dense_set = 8 * n + n / 8;  // values + presence bits
  const int64_t frontier = 16 * n;          // frontier ids, slots, shares, offsets
  switch (r.algo) {
    case LGC_ALGO_PRNIBBLE: {
      double bound = 1.0 + 1.0 / (r.pr.alpha * r.pr.eps);
      int64_t keys = bound < (double)n ? (int64_t)bound : n;
      return std::min<int64_t>(slots(keys) * 24 + keys * 24, 2 * dense_set + 8 * n + frontier);
    }
    case LGC_ALGO_NIBBLE:
      return std::min<int64_t>(2 * slots(n) * 16 + n * 24, 2 * dense_set + frontier);
    case LGC_ALGO_HKPR:
      return std::min<int64_t>(3 * slots(n) * 16 + n * 24, 3 * dense_set + frontier);
    default:
      return r.rh.n_walks * 40;
  }
}

// Takes the first queued request that fits (bounded bypass); S->mu held.
static bool take_fitting(Serve* S, std::deque<Serve::Item>& q, Serve::Item* out) {
  for (auto it = q.begin(); it != q.end(); ++it) {
    const bool fits = S->inflight == 0 ||
                      (S->inflight < S->owner->serve_max_batch &&
                       S->inflight_bytes + S->lane_bytes + it->bytes <= S->owner->serve_mem_budget);
    if (fits) {
      for (auto jt = q.begin(); jt != it; ++jt) jt->bypassed++;
      *out = *it;
      q.erase(it);
      return true;
    }
    if (it->bypassed >= kMaxBypass) return false;  // nothing may pass it any more
  }
  return false;
}

static void publish(Serve* S, uint64_t ticket, lgc_result* res) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->done[ticket] = res;
  }
  S->cv.notify_all();
}

static void serve_worker(Serve* S, lgc_ctx* wc) {
  for (;;) {
    Serve::Item it;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || take_fitting(S, S->queue, &it); });
      if (S->stop) return;
      S->inflight++;
      S->inflight_bytes += it.bytes;
    }
    lgc_result* res = new lgc_result();
    memset(res, 0, sizeof(*res));
    res->submit_s = it.submit_s;
    res->start_s = now_seconds();
    wc->result_on_device = false;
    lgc_svec* p = nullptr;
    int st = LGC_EINVAL;
    switch (it.req.algo) {
      case LGC_ALGO_PRNIBBLE:
        st = run_prnibble(wc, it.g, it.req.seed, &it.req.pr, &p, &res->stats, nullptr);
        break;
      case LGC_ALGO_NIBBLE:
        st = run_nibble(wc, it.g, it.req.seed, &it.req.nb, &p, &res->stats);
        break;
      case LGC_ALGO_HKPR:
        st = run_hkpr(wc, it.g, it.req.seed, &it.req.hk, &p, &res->stats);
        break;
      case LGC_ALGO_RAND_HKPR:
        st = run_rand_hkpr(wc, it.g, it.req.seed, &it.req.rh, &p, &res->stats);
        break;
    }
    if (st == LGC_EMAXROUNDS) st = LGC_OK;
    res->p = p;
    if (st == LGC_OK && it.req.want_sweep && p) st = run_sweep(wc, it.g, p, &res->cluster);
    cudaStreamSynchronize(wc->stream);
    res->status = st;
    res->end_s = now_seconds();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->inflight--;
      S->inflight_bytes -= it.bytes;
    }
    publish(S, it.ticket, res);
  }
}

// The PR-Nibble lane: one batch engine per (graph, mode); every pass admits
// the queued PR-Nibble requests that fit, runs one round of every engine
// with running seeds, and hands out the finished seeds' results (vectors
// extracted together, sweep cuts of all of them in one batched sweep).
struct LaneJob {
  Serve::Item item;
  double start_s;
};

static void lane_fail(Serve* S, const LaneJob& j, int st) {
  lgc_result* res = new lgc_result();
  memset(res, 0, sizeof(*res));
  res->status = st;
  res->submit_s = j.item.submit_s;
  res->start_s = j.start_s;
  res->end_s = now_seconds();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->lane_resident--;
  }
  publish(S, j.item.ticket, res);
}

static void serve_lane(Serve* S, lgc_ctx* lc) {
  struct Eng {
    BatchEngine E;
    std::map<int64_t, LaneJob> jobs;  // slot -> request
    double first_done_s = 0.0;        // when the oldest unharvested seed finished
  };
  // Finished seeds are handed out together (one extraction, one batched
  // sweep): when no seed of the engine is running any more, when they are a
  // quarter of its seeds, when admission is waiting for memory they hold, or
  // when the oldest has waited kHarvestWait seconds.
  constexpr double kHarvestWait = 0.002;
  bool admission_blocked = false;
  // engines by (graph serial, mode); an engine without requests is dropped
  // at the end of the pass that emptied it
  std::map<std::pair<uint64_t, int>, Eng*> engines;
  lc->result_on_device = false;
  for (;;) {
    std::vector<Serve::Item> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      bool busy = false;
      for (auto& kv : engines) busy = busy || kv.second->E.nf > 0;
      if (!busy) S->cv.wait(lk, [&] { return S->stop || !S->prq.empty(); });
      if (S->stop) break;
      // admission by live table memory: the lane's tables after its last
      // round plus the workers' reservations stay within the budget
      const int64_t lane_cap = S->owner->serve_lane_seeds;
      int64_t adding = 0;  // first tables of the seeds admitted in this pass
      while (!S->prq.empty() && S->lane_resident < lane_cap) {
        const Serve::Item& h = S->prq.front();
        const int64_t d = h.g->hdeg[h.req.seed];
        const int64_t first = table_bytes(pow2_at_least(std::max<int64_t>(64, 2 * (1 + d))));
        const bool fits = S->lane_resident == 0 ||
                          S->inflight_bytes + S->lane_bytes + adding + first <=
                              S->owner->serve_mem_budget;
        if (!fits) break;
        adding += first;
        admit.push_back(h);
        S->prq.pop_front();
        S->lane_resident++;
      }
      admission_blocked = !S->prq.empty();
    }
    // new seeds join their engine at the next round
    const double t_admit = now_seconds();
    std::map<std::pair<uint64_t, int>, std::vector<Serve::Item>> by_engine;
    for (const Serve::Item& it : admit) by_engine[{it.g->serial, it.req.pr.mode}].push_back(it);
    for (auto& kv : by_engine) {
      Eng*& e = engines[kv.first];
      if (!e) {
        e = new Eng();
        const int st = e->E.init(lc, kv.second[0].g, kv.first.second);
        if (st != LGC_OK) {
          for (const Serve::Item& it : kv.second) lane_fail(S, LaneJob{it, t_admit}, st);
          e->E.fini();
          delete e;
          engines.erase(kv.first);
          continue;
        }
      }
      // one at a time on a refusal, so that a bad request fails alone
      std::vector<int32_t> seeds;
      std::vector<lgc_prnibble_params> prms;
      for (const Serve::Item& it : kv.second) {
        seeds.push_back(it.req.seed);
        prms.push_back(it.req.pr);
      }
      std::vector<int64_t> slots(seeds.size());
      int st = e->E.add((int64_t)seeds.size(), seeds.data(), prms.data(), slots.data());
      if (st == LGC_OK) {
        for (size_t i = 0; i < slots.size(); i++)
          e->jobs[slots[i]] = LaneJob{kv.second[i], t_admit};
      } else {
        for (size_t i = 0; i < seeds.size(); i++) {
          int64_t sl = -1;
          const int s1 = e->E.add(1, &seeds[i], &prms[i], &sl);
          if (s1 == LGC_OK) e->jobs[sl] = LaneJob{kv.second[i], t_admit};
          else lane_fail(S, LaneJob{kv.second[i], t_admit}, s1);
        }
      }
    }
    // one round of every engine, then the finished seeds' results
    int64_t live = 0;
    for (auto& kv : engines) {
      Eng* e = kv.second;
      lgc_graph* g = e->E.g;
      if (e->E.nf > 0) {
        const int st = e->E.round();
        if (st != LGC_OK) {  // every request of this engine fails; the engine restarts
          for (auto& jv : e->jobs) lane_fail(S, jv.second, st);
          e->jobs.clear();
          e->E.fini();
          e->E = BatchEngine();
          e->E.init(lc, g, kv.first.second);
          continue;
        }
      }
      if (!e->E.done.empty() && e->first_done_s == 0.0) e->first_done_s = now_seconds();
      const int64_t ndone = (int64_t)e->E.done.size();
      const bool harvest =
          ndone > 0 && (e->E.running == 0 || 4 * ndone >= (int64_t)e->jobs.size() ||
                        admission_blocked || now_seconds() - e->first_done_s >= kHarvestWait);
      if (harvest) {
        e->first_done_s = 0.0;
        std::vector<int64_t> fin;
        fin.swap(e->E.done);
        std::vector<lgc_svec*> ps(fin.size(), nullptr);
        std::vector<lgc_stats> sts(fin.size());
        int st = e->E.extract(fin, ps.data(), sts.data());
        std::vector<lgc_cluster*> cl(fin.size(), nullptr);
        std::vector<const lgc_svec*> want;
        std::vector<size_t> at;
        for (size_t i = 0; st == LGC_OK && i < fin.size(); i++)
          if (e->jobs[fin[i]].item.req.want_sweep && ps[i]) {
            want.push_back(ps[i]);
            at.push_back(i);
          }
        std::vector<lgc_cluster*> got(want.size(), nullptr);
        if (st == LGC_OK && !want.empty())
          st = run_sweep_batch(lc, g, (int64_t)want.size(), want.data(), got.data());
        for (size_t k = 0; k < at.size(); k++) cl[at[k]] = got[k];
        const double t_end = now_seconds();
        for (size_t i = 0; i < fin.size(); i++) {
          const LaneJob j = e->jobs[fin[i]];
          e->jobs.erase(fin[i]);
          e->E.release(fin[i]);
          lgc_result* res = new lgc_result();
          memset(res, 0, sizeof(*res));
          res->status = st;
          res->p = st == LGC_OK ? ps[i] : nullptr;
          res->cluster = st == LGC_OK ? cl[i] : nullptr;
          if (st != LGC_OK) {
            lgc_svec_free(ps[i]);
            lgc_cluster_free(cl[i]);
          }
          res->stats = sts[i];
          res->submit_s = j.item.submit_s;
          res->start_s = j.start_s;
          res->end_s = t_end;
          {
            std::lock_guard<std::mutex> lk(S->mu);
            S->lane_resident--;
            S->done[j.item.ticket] = res;
          }
        }
        S->cv.notify_all();
      }
      live += e->E.table_bytes_live();
    }
    for (auto it = engines.begin(); it != engines.end();) {
      if (it->second->jobs.empty() && it->second->E.nf == 0) {
        it->second->E.fini();
        delete it->second;
        it = engines.erase(it);
      } else {
        ++it;
      }
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->lane_bytes = live;
    }
    S->cv.notify_all();  // workers may fit now
  }
  for (auto& kv : engines) {
    for (auto& jv : kv.second->jobs) lane_fail(S, jv.second, LGC_ECUDA);
    kv.second->E.fini();
    delete kv.second;
  }
}

static void serve_shutdown(lgc_ctx* ctx) {
  Serve* S = ctx->serve;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  if (S->lane.joinable()) S->lane.join();
  for (lgc_ctx* w : S->wctx) {
    ctx_fini(w);
    delete w;
  }
  if (S->lane_ctx) {
    ctx_fini(S->lane_ctx);
    delete S->lane_ctx;
  }
  for (auto& kv : S->done) lgc_result_free(kv.second);
  delete S;
  ctx->serve = nullptr;
}

}  // namespace lgc

extern "C" {

const char* lgc_strerror(int s) {
  switch (s) {
    case LGC_OK: return "ok";
    case LGC_PENDING: return "pending";
    case LGC_EINVAL: return "invalid argument";
    case LGC_ENOMEM: return "out of memory";
    case LGC_ETABLEFULL: return "hash table full";
    case LGC_EMAXROUNDS: return "maximum number of rounds reached";
    case LGC_ECUDA: return "CUDA error";
    case LGC_EBUSY: return "busy";
    case LGC_ENOTFOUND: return "not found";
    case LGC_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

int lgc_ctx_create(int device, void* cuda_stream, lgc_ctx** out) {
  return lgc_ctx_create_with_alloc(device, nullptr, cuda_stream, out);
}

int lgc_ctx_create_with_alloc(int device, const lgc_alloc_fns* fns, void* cuda_stream,
                              lgc_ctx** out) {
  if (!out) return LGC_EINVAL;
  if (fns && (!fns->alloc || !fns->free)) return LGC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return LGC_ECUDA;
  }
  if (device < 0 || device >= ndev) return LGC_EINVAL;
  lgc_ctx* ctx = new (std::nothrow) lgc_ctx();
  if (!ctx) return LGC_ENOMEM;
  if (fns) ctx->alloc_fns = *fns;
  int s = ctx_init(ctx, device, (cudaStream_t)cuda_stream);
  if (s != LGC_OK) {
    ctx_fini(ctx);
    delete ctx;
    return s;
  }
  *out = ctx;
  return LGC_OK;
}

void lgc_ctx_destroy(lgc_ctx* ctx) {
  if (!ctx) return;
  serve_shutdown(ctx);
  if (ctx->last_residual) lgc_svec_free(ctx->last_residual);
  ctx_fini(ctx);
  delete ctx;
}

int lgc_set_trace(lgc_ctx* ctx, int flags) {
  if (!ctx || (flags & ~LGC_TRACE_FRONTIERS)) return LGC_EINVAL;
  return lgc_ctx_set_option(ctx, LGC_OPT_TRACE, flags & LGC_TRACE_FRONTIERS);
}

int lgc_ctx_set_option(lgc_ctx* ctx, int option, int64_t value) {
  if (!ctx) return LGC_EINVAL;
  switch (option) {
    case LGC_OPT_RESULT_ON_DEVICE: ctx->result_on_device = value != 0; return LGC_OK;
    case LGC_OPT_TRACE: ctx->trace = value != 0; return LGC_OK;
    case LGC_OPT_PROFILE: ctx->profile = value != 0; return LGC_OK;
    case LGC_OPT_TABLE_FORM:
      if (value < 0 || value > 2) return LGC_EINVAL;
      ctx->table_form = (int)value;
      return LGC_OK;
    case LGC_OPT_PULL:
      if (value < 0 || value > 2) return LGC_EINVAL;
      ctx->pull_policy = (int)value;
      return LGC_OK;
    case LGC_OPT_DEVICE_ROUNDS:
      if (value < 0 || value > 1) return LGC_EINVAL;
      ctx->device_rounds = value != 0;
      return LGC_OK;
    case LGC_OPT_PULL_BATCH:
      if (value != 0 && value != 4 && value != 8 && value != 16) return LGC_EINVAL;
      ctx->pull_batch = (int)value;
      return LGC_OK;
    case LGC_OPT_PULL_GROUP:
      if (value != 0 && value != 8 && value != 16 && value != 32) return LGC_EINVAL;
      ctx->pull_group = (int)value;
      return LGC_OK;
    case LGC_OPT_PULL_SHARE:
      if (value != 0 && value != 8 && value != 16) return LGC_EINVAL;
      ctx->pull_share = (int)value;
      return LGC_OK;
    case LGC_OPT_BATCH_HANDOFF:
      if (value < -1) return LGC_EINVAL;
      ctx->batch_handoff = value;
      return LGC_OK;
    case LGC_OPT_HK_THRESHOLD_SIGN:
      if (value != 1 && value != -1) return LGC_EINVAL;
      ctx->hk_threshold_sign = (int)value;
      return LGC_OK;
    case LGC_OPT_SWEEP_CROSS:
      if (value < 0 || value > 2) return LGC_EINVAL;
      ctx->sweep_cross = (int)value;
      return LGC_OK;
    case LGC_OPT_SERVE_MEM_BUDGET:
      if (value <= 0) return LGC_EINVAL;
      ctx->serve_mem_budget = value;
      return LGC_OK;
    case LGC_OPT_SERVE_LANE:
      if (value < 0 || value > (1 << 20)) return LGC_EINVAL;
      if (ctx->serve) return LGC_EBUSY;  // fixed once the loop has started
      ctx->serve_lane_seeds = value;
      return LGC_OK;
    case LGC_OPT_SERVE_MAX_BATCH:
      if (value <= 0 || value > 1024) return LGC_EINVAL;
      if (ctx->serve) return LGC_EBUSY;  // fixed once the loop has started
      ctx->serve_max_batch = value;
      return LGC_OK;
    default: return LGC_EINVAL;
  }
}

int lgc_ctx_synchronize(lgc_ctx* ctx) {
  if (!ctx) return LGC_EINVAL;
  LGC_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LGC_OK;
}

int lgc_graph_create(lgc_ctx* ctx, int64_t n, const int64_t* offsets, const int32_t* cols,
                     int flags, lgc_graph** out) {
  if (!ctx || !out || n < 0 || !offsets || (n > 0 && !cols) || n >= INT32_MAX) return LGC_EINVAL;
  *out = nullptr;
  cudaStream_t s = ctx->stream;
  const bool dev = flags & LGC_GRAPH_DEVICE_INPUT;
  int64_t nnz = 0;
  LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, offsets + n, 8,
                               dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  LGC_CUDA_TRY(cudaStreamSynchronize(s));
  nnz = ctx->h_scratch[0];
  if (nnz < 0) return LGC_EINVAL;
  lgc_graph* g = new (std::nothrow) lgc_graph();
  static std::atomic<uint64_t> graphs_made{0};
  if (g) g->serial = ++graphs_made;
  if (!g) return LGC_ENOMEM;
  g->ctx = ctx;
  g->n = n;
  g->nnz = nnz;
  int st = LGC_OK;
  do {
    if ((st = dalloc_t(ctx, &g->off, n + 1)) != LGC_OK) break;
    if ((st = dalloc_t(ctx, &g->col, nnz)) != LGC_OK) break;
    if ((st = dalloc_t(ctx, &g->deg, n)) != LGC_OK) break;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(g->off, offsets, 8 * (n + 1), k, s) != cudaSuccess) {
      st = LGC_ECUDA;
      break;
    }
    if (nnz && cudaMemcpyAsync(g->col, cols, 4 * nnz, k, s) != cudaSuccess) {
      st = LGC_ECUDA;
      break;
    }
    int* dflags = nullptr;
    if ((st = dalloc_t(ctx, &dflags, 2)) != LGC_OK) break;
    cudaMemsetAsync(dflags, 0, 8, s);
    if (n > 0) {
      if (flags & LGC_GRAPH_VALIDATE) {
        validate_kernel<<<grid_for(n), kBlock, 0, s>>>(g->off, g->col, n, nnz, dflags);
        LGC_COUNT_LAUNCH(ctx);
      }
      degree_kernel<<<std::min(grid_for(n), (ctx->sms * 64)), kBlock, 0, s>>>(g->off, n, g->deg,
                                                                       dflags + 1);
      LGC_COUNT_LAUNCH(ctx);
    }
    cudaMemcpyAsync(ctx->h_scratch, dflags, 8, cudaMemcpyDeviceToHost, s);
    dfree(ctx, dflags);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      st = LGC_ECUDA;
      break;
    }
    int32_t* hf = (int32_t*)ctx->h_scratch;
    if (hf[0] != 0) {
      st = LGC_EINVAL;
      break;
    }
    g->max_deg = hf[1];
    try {
      g->hdeg.resize(n);
    } catch (...) {
      st = LGC_ENOMEM;
      break;
    }
    if (n && (cudaMemcpyAsync(g->hdeg.data(), g->deg, 4 * n, cudaMemcpyDeviceToHost, s) !=
                  cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess)) {
      st = LGC_ECUDA;
      break;
    }
    st = build_heavy_list(ctx, g);
    if (st == LGC_OK) st = build_big_segments(ctx, g);
    if (st == LGC_OK) st = build_light_items(ctx, g);
  } while (0);
  if (st != LGC_OK) {
    dfree(ctx, g->off);
    dfree(ctx, g->col);
    dfree(ctx, g->deg);
    dfree(ctx, g->heavy);
    dfree(ctx, g->items);
    dfree(ctx, g->big_w);
    dfree(ctx, g->big_seg0);
    dfree(ctx, g->segs);
    dfree(ctx, g->det_mid);
    if (g->light_det != g->light) dfree(ctx, g->light_det);
    dfree(ctx, g->light);
    cudaStreamSynchronize(s);
    delete g;
    return st;
  }
  *out = g;
  return LGC_OK;
}

// Waits until no queued or running request of the context's request loop
// uses g.
static void wait_graph_idle(lgc_graph* g) {
  lgc_ctx* ctx = g->ctx;
  if (!ctx->serve) return;
  Serve* S = ctx->serve;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv.wait(lk, [&] {
    for (auto& it : S->queue)
      if (it.g == g) return false;
    for (auto& it : S->prq)
      if (it.g == g) return false;
    return S->inflight == 0 && S->lane_resident == 0;
  });
}

void lgc_graph_destroy(lgc_graph* g) {
  if (!g) return;
  lgc_ctx* ctx = g->ctx;
  wait_graph_idle(g);
  dfree(ctx, g->off);
  dfree(ctx, g->col);
  dfree(ctx, g->deg);
  dfree(ctx, g->heavy);
  dfree(ctx, g->items);
  dfree(ctx, g->big_w);
  dfree(ctx, g->big_seg0);
  dfree(ctx, g->segs);
  dfree(ctx, g->det_mid);
  if (g->light_det != g->light) dfree(ctx, g->light_det);
  dfree(ctx, g->light);
  cudaStreamSynchronize(ctx->stream);
  delete g;
}

int lgc_graph_autotune(lgc_graph* g, int* pull_batch, int* pull_group, int* pull_share) {
  if (!g) return LGC_EINVAL;
  wait_graph_idle(g);  // the pull lists are rebuilt: no request may be using them
  LGC_TRY(autotune_pull(g->ctx, g));
  LGC_TRY(autotune_batch(g->ctx, g));
  if (pull_batch) *pull_batch = g->pull_batch;
  if (pull_group) *pull_group = g->pull_group;
  if (pull_share) *pull_share = g->pull_share;
  return LGC_OK;
}

int64_t lgc_graph_batch_handoff(const lgc_graph* g) { return g ? batch_handoff_of(g) : -1; }

int lgc_graph_pull_light(const lgc_graph* g) { return g ? g->pull_light : -1; }

int lgc_graph_set_pull_light(lgc_graph* g, int light) {
  if (!g || light < 4 || light > 256) return LGC_EINVAL;
  wait_graph_idle(g);
  if (light == g->pull_light) return LGC_OK;
  return rebuild_pull_lists(g->ctx, g, light);
}

int64_t lgc_graph_num_vertices(const lgc_graph* g) { return g ? g->n : -1; }
int64_t lgc_graph_num_entries(const lgc_graph* g) { return g ? g->nnz : -1; }

int lgc_prnibble(lgc_graph* g, int32_t seed, const lgc_prnibble_params* prm, lgc_svec** p,
                 lgc_stats* st) {
  if (!g || !prm || !p) return LGC_EINVAL;
  lgc_ctx* ctx = g->ctx;
  if (ctx->last_residual) {
    lgc_svec_free(ctx->last_residual);
    ctx->last_residual = nullptr;
  }
  return run_prnibble(ctx, g, seed, prm, p, st, ctx->trace ? &ctx->last_residual : nullptr);
}

int lgc_prnibble_residual(lgc_ctx* ctx, lgc_svec** r) {
  if (!ctx || !r) return LGC_EINVAL;
  *r = nullptr;
  if (!ctx->last_residual) return LGC_ENOTFOUND;
  *r = ctx->last_residual;
  ctx->last_residual = nullptr;
  return LGC_OK;
}

int lgc_prnibble_set(lgc_graph* g, int64_t k, const int32_t* seeds, const double* weights,
                     double beta, const lgc_prnibble_params* prm, lgc_svec** p, lgc_stats* st) {
  if (!g || !prm || !p) return LGC_EINVAL;
  lgc_ctx* ctx = g->ctx;
  if (ctx->last_residual) {
    lgc_svec_free(ctx->last_residual);
    ctx->last_residual = nullptr;
  }
  return run_prnibble_set(ctx, g, k, seeds, weights, beta, prm, p, st,
                          ctx->trace ? &ctx->last_residual : nullptr);
}

int lgc_nibble(lgc_graph* g, int32_t seed, const lgc_nibble_params* prm, lgc_svec** p,
               lgc_stats* st) {
  if (!g || !prm || !p) return LGC_EINVAL;
  return run_nibble(g->ctx, g, seed, prm, p, st);
}

int lgc_hkpr(lgc_graph* g, int32_t seed, const lgc_hkpr_params* prm, lgc_svec** p,
             lgc_stats* st) {
  if (!g || !prm || !p) return LGC_EINVAL;
  return run_hkpr(g->ctx, g, seed, prm, p, st);
}

int lgc_rand_hkpr(lgc_graph* g, int32_t seed, const lgc_rand_hkpr_params* prm, lgc_svec** p,
                  lgc_stats* st) {
  if (!g || !prm || !p) return LGC_EINVAL;
  return run_rand_hkpr(g->ctx, g, seed, prm, p, st);
}

int lgc_rand_hkpr_endpoints(lgc_ctx* ctx, int32_t* out, int64_t n_walks) {
  if (!ctx || !out) return LGC_EINVAL;
  if (!ctx->d_endpoints) return LGC_ENOTFOUND;
  if (n_walks != ctx->n_endpoints) return LGC_EINVAL;
  LGC_CUDA_TRY(cudaMemcpyAsync(out, ctx->d_endpoints, 4 * n_walks, cudaMemcpyDeviceToHost,
                               ctx->stream));
  LGC_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return LGC_OK;
}

int lgc_sweep(lgc_graph* g, const lgc_svec* p, lgc_cluster** out) {
  if (!g || !p || !out) return LGC_EINVAL;
  return run_sweep(g->ctx, g, p, out);
}

int lgc_sweep_batch(lgc_graph* g, int64_t B, const lgc_svec* const* p, lgc_cluster** out) {
  if (!g || !p || !out) return LGC_EINVAL;
  return run_sweep_batch(g->ctx, g, B, p, out);
}

int lgc_get_trace(lgc_ctx* ctx, int64_t* rounds, int64_t* sizes, int64_t cap_rounds,
                  int32_t* frontiers, int64_t cap_ids) {
  if (!ctx || !rounds) return LGC_EINVAL;
  *rounds = (int64_t)ctx->trace_sizes.size();
  if (sizes) {
    int64_t k = std::min<int64_t>(cap_rounds, *rounds);
    memcpy(sizes, ctx->trace_sizes.data(), 8 * k);
  }
  if (frontiers) {
    int64_t k = std::min<int64_t>(cap_ids, (int64_t)ctx->trace_ids.size());
    memcpy(frontiers, ctx->trace_ids.data(), 4 * k);
  }
  return LGC_OK;
}

int64_t lgc_launch_count(const lgc_ctx* ctx) { return ctx ? ctx->n_launches : -1; }

int lgc_profile_read(lgc_ctx* ctx, int kernel, lgc_kernel_profile* out) {
  if (!ctx || !out || kernel < 0 || kernel >= LGC_PROF_COUNT) return LGC_EINVAL;
  profile_collect(ctx);
  *out = ctx->prof[kernel];
  return LGC_OK;
}

int lgc_profile_reset(lgc_ctx* ctx) {
  if (!ctx) return LGC_EINVAL;
  profile_collect(ctx);
  for (int k = 0; k < LGC_PROF_COUNT; k++) ctx->prof[k] = lgc_kernel_profile{0, 0.0, 0.0};
  return LGC_OK;
}

int lgc_submit(lgc_ctx* ctx, lgc_graph* g, const lgc_request* req, uint64_t* ticket) {
  if (!ctx || !g || !req || !ticket) return LGC_EINVAL;
  if (req->algo < LGC_ALGO_PRNIBBLE || req->algo > LGC_ALGO_RAND_HKPR) return LGC_EINVAL;
  if (req->seed < 0 || req->seed >= g->n) return LGC_EINVAL;
  if (!ctx->serve) {
    Serve* S = new (std::nothrow) Serve();
    if (!S) return LGC_ENOMEM;
    S->owner = ctx;
    int nw = (int)std::min<int64_t>(ctx->serve_max_batch, 64);
    for (int i = 0; i < nw; i++) {
      lgc_ctx* w = new (std::nothrow) lgc_ctx();
      if (!w || ctx_init(w, ctx->device, nullptr) != LGC_OK) {
        if (w) {
          ctx_fini(w);
          delete w;
        }
        break;
      }
      w->device_rounds = false;  // cooperative launches are never run side by side
      S->wctx.push_back(w);
    }
    if (S->wctx.empty()) {
      delete S;
      return LGC_ECUDA;
    }
    if (ctx->serve_lane_seeds > 0) {
      lgc_ctx* l = new (std::nothrow) lgc_ctx();
      if (l && ctx_init(l, ctx->device, nullptr) == LGC_OK) {
        l->device_rounds = false;
        l->batch_handoff = ctx->batch_handoff;
        S->lane_ctx = l;
      } else if (l) {
        ctx_fini(l);
        delete l;
      }
    }
    for (lgc_ctx* w : S->wctx) S->workers.emplace_back(serve_worker, S, w);
    if (S->lane_ctx) S->lane = std::thread(serve_lane, S, S->lane_ctx);
    ctx->serve = S;
  }
  Serve* S = ctx->serve;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() + S->prq.size() >= S->max_queue) return LGC_EBUSY;
    Serve::Item it;
    it.ticket = S->next_ticket++;
    it.g = g;
    it.req = *req;
    it.submit_s = now_seconds();
    it.bytes = request_bytes(g, *req);
    it.bypassed = 0;
    if (req->algo == LGC_ALGO_PRNIBBLE && S->lane_ctx) S->prq.push_back(it);
    else S->queue.push_back(it);
    S->known[it.ticket] = 1;
    *ticket = it.ticket;
  }
  S->cv.notify_all();
  return LGC_OK;
}

int lgc_poll(lgc_ctx* ctx, uint64_t ticket, lgc_result** out) {
  if (!ctx || !out) return LGC_EINVAL;
  *out = nullptr;
  Serve* S = ctx->serve;
  if (!S) return LGC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it != S->done.end()) {
    *out = it->second;
    S->done.erase(it);
    S->known.erase(ticket);
    return LGC_OK;
  }
  return S->known.count(ticket) ? LGC_PENDING : LGC_ENOTFOUND;
}

int lgc_wait(lgc_ctx* ctx, uint64_t ticket, lgc_result** out) {
  if (!ctx || !out) return LGC_EINVAL;
  *out = nullptr;
  Serve* S = ctx->serve;
  if (!S) return LGC_ENOTFOUND;
  std::unique_lock<std::mutex> lk(S->mu);
  // woken by every finished request (the workers notify all after storing)
  S->cv.wait(lk, [&] { return S->stop || S->done.count(ticket) || !S->known.count(ticket); });
  auto it = S->done.find(ticket);
  if (it == S->done.end()) return LGC_ENOTFOUND;
  *out = it->second;
  S->done.erase(it);
  S->known.erase(ticket);
  return LGC_OK;
}

void lgc_svec_free(lgc_svec* p) {
  if (!p) return;
  SvecBox* b = (SvecBox*)p;
  if (p->on_device) {
    dfree(b->ctx, p->idx);
    dfree(b->ctx, p->val);
  } else {
    host_free(p->idx);
    host_free(p->val);
  }
  delete b;
}

void lgc_cluster_free(lgc_cluster* c) {
  if (!c) return;
  ClusterBox* b = (ClusterBox*)c;
  if (c->on_device) dfree(b->ctx, c->ids);
  else host_free(c->ids);
  delete b;
}

void lgc_result_free(lgc_result* r) {
  if (!r) return;
  lgc_svec_free(r->p);
  lgc_cluster_free(r->cluster);
  delete r;
}

}  // extern "C"

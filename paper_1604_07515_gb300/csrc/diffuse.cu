// Synchronous frontier diffusions: PR-Nibble (Sec. 3.3), Nibble (Sec. 3.2)
// and HK-PR (Sec. 3.4).
//
// One round = vertexMap over the frontier F (per-algorithm kernel: reads the
// frontier values, updates the vertex's own entries, computes the share it
// sends along each edge) followed by an edgeMap (generic: adds the share to
// the destination's entry of a hash table) and the filter that forms the
// next frontier.
//
// Atomic mode: the edgeMap adds with atomicAdd (the paper's fetchAdd).  The
// next frontier is formed during the edgeMap itself: the one add that takes
// a destination from below its threshold c*d(w) to at least it appends w
// (values only grow, so exactly one add crosses).  Only F and N(F) can
// change, so this equals the paper's filter over the whole sparse set.
//
// Deterministic mode: the edgeMap emits one (destination, share) record per
// edge in frontier order (the frontier is kept in ascending id), sorts the
// records stably by destination, and folds each destination's run left to
// right starting from the value it holds after the vertexMap.  That is the
// order a sequential loop over ascending sources produces, so p, r and every
// frontier are bit-identical to it.  The filter then compacts the runs whose
// result reaches the threshold; runs are in ascending id, so the next
// frontier is too.
//
// All arithmetic is IEEE binary64 with FMA contraction disabled (--fmad=false),
// each expression evaluated in the order written.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>
#include <string.h>

#include <cooperative_groups.h>

#include "common.cuh"
#include "fx128.cuh"
#include "lookback.cuh"
#include "prim.cuh"

namespace cg = cooperative_groups;

namespace lgc {

namespace {

constexpr int kEdgeItems = 4;
constexpr int kEdgeTile = kBlock * kEdgeItems;  // edges per CTA tile

enum FrontierMode { kFmNone = 0, kFmThreshold = 1, kFmInserted = 2 };

// The first index of a[0, n) (non-decreasing) whose entry exceeds x, found
// by all 32 lanes of a warp (the same result in each): every step probes the
// last entry of 32 equal chunks of the range and keeps the chunk where the
// entries start to exceed x, so a search over n entries takes about
// log32(n) dependent loads instead of log2(n).
__device__ inline int64_t warp_upper_bound(const int64_t* a, int64_t n, int64_t x) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t pos = lo + (int64_t)(lane + 1) * step - 1;
    const bool le = pos < hi && a[pos] <= x;  // true on a prefix of the lanes
    const int c = __popc(__ballot_sync(0xffffffffu, le));
    lo += (int64_t)c * step;
    if (lo >= hi) return hi;
    hi = min(hi, lo + step);
  }
  const bool le = lo + lane < hi && a[lo + lane] <= x;
  return lo + __popc(__ballot_sync(0xffffffffu, le));
}

// Stages, for the block's record range [e0, e1), the exclusive prefix sums of
// the sources owning those records into s_epos[0..cnt] (the last entry is
// the end of the last staged source) and returns cnt <= kEdgeTile.  All
// threads of the block must call it; the caller synchronizes after staging
// its own per-source arrays.
__device__ inline int stage_sources(const int64_t* epos, int64_t nf, int64_t total,
                                    int64_t e0, int64_t e1, int64_t* s_i0, int64_t* s_i1,
                                    int64_t* s_epos) {
  const int warp = threadIdx.x >> 5;
  if (warp < 2) {  // the two ends at once, each by a whole warp
    const int64_t b = warp_upper_bound(epos, nf, warp == 0 ? e0 : e1 - 1) - 1;
    if ((threadIdx.x & 31) == 0) *(warp == 0 ? s_i0 : s_i1) = b;
  }
  __syncthreads();
  const int64_t i0 = *s_i0;
  int64_t c = *s_i1 - i0 + 1;
  if (i0 < 0 || c < 0) c = 0;
  if (c > kEdgeTile) c = kEdgeTile;
  const int cnt = (int)c;
  for (int j = threadIdx.x; j <= cnt; j += kBlock)
    s_epos[j] = (i0 + j < nf) ? epos[i0 + j] : total;
  __syncthreads();
  return cnt;
}

// Source j (within the staged range) of record e and its local index *q;
// -1 if e is not a record of a staged source.
__device__ inline int find_source(const int64_t* s_epos, int cnt, int64_t e, int64_t* q) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s_epos[mid] <= e) lo = mid + 1;
    else hi = mid;
  }
  const int j = lo - 1;
  if (j < 0) return -1;
  const int64_t local = e - s_epos[j];
  if (local >= s_epos[j + 1] - s_epos[j]) return -1;
  *q = local;
  return j;
}

// Adds every thread's count n into *counter with one atomic per block (a
// per-warp atomic on one address queues when a launch has many warps).  All
// threads of the block call it, once, where every thread arrives.
__device__ inline void flush_count(int64_t n, int64_t* counter) {
  __shared__ int64_t s_cnt[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_cnt[k];
    if (t) atomicAdd((unsigned long long*)counter, (unsigned long long)t);
  }
}

__device__ inline void count_inserted(int ins, int64_t* counter) {
  const unsigned active = __activemask();
  const unsigned m = __ballot_sync(active, ins);
  if (m && (threadIdx.x & 31) == __ffs(active) - 1)
    atomicAdd((unsigned long long*)counter, (unsigned long long)__popc(m));
}

// ---------------------------------------------------------------------------
// vertexMap kernels.  Each writes, per frontier entry i: share[i], the
// record count cnt[i] (d(v), plus one self record in deterministic mode when
// the vertex itself is a key of the destination table) and foff[i] = off[v].
// ---------------------------------------------------------------------------

// PR-Nibble, Fig. alg:pr-nibble (rule 1) / alg:pr-nibble2 (rule 0).  T holds
// r in slot.val and p in T.p[slot]; r' is updated in place (every read of r
// in the round is of a frontier vertex, done here before the edgeMap).
// The vertexMap bodies take the frontier entries [i0, i1) in steps of `step`
// (a block-uniform start: the grid's stride, or a block's own chunk) and
// return the sum of the record counts this thread wrote.
__device__ inline int64_t prnibble_vmap_body(int64_t i0, int64_t i1, int64_t step,
                                             const int32_t* fv, const int32_t* fs, Table T,
                                             const int64_t* __restrict__ off, double alpha,
                                             double cs, double cn, double eps, int rule, int det,
                                             int self_append, double* share, int64_t* cnt,
                                             int64_t* foff, int32_t* nfv, int32_t* nfs,
                                             int32_t ncap, Counters* C) {
  int64_t csum = 0;
  for (int64_t base = i0; base < i1; base += step) {
    const int64_t i = base + threadIdx.x;
    bool pred = false;
    int32_t v = 0, s = 0;
    int64_t d = 0;
    if (i < i1) {
      v = fv[i];
      s = fs[i];
      const bool ok = s >= 0;  // always true unless a table overflowed (flagged)
      const double r = ok ? *tb_val(T, s) : 0.0;
      const int64_t o0 = off[v];
      d = off[v + 1] - o0;
      double sh, rbase;
      if (rule == 0) {
        if (ok) T.p[s] = T.p[s] + cs * r;
        rbase = 0.0;
        sh = (cn * r) / (double)d;
      } else {
        if (ok) T.p[s] = T.p[s] + alpha * r;
        rbase = ((1.0 - alpha) * r) / 2.0;
        sh = ((1.0 - alpha) * r) / (2.0 * (double)d);
      }
      if (ok) *tb_val(T, s) = rbase;
      share[i] = sh;
      cnt[i] = d + (det ? 1 : 0);
      csum += cnt[i];
      foff[i] = o0;
      pred = ok && self_append && rule == 1 && rbase >= eps * (double)d;
    }
    frontier_append(pred, v, s, d, nfv, nfs, C, ncap);
  }
  return csum;
}

__global__ void vmap_prnibble_kernel(int64_t nf, const int32_t* __restrict__ fv,
                                     const int32_t* __restrict__ fs, Table T,
                                     const int64_t* __restrict__ off, double alpha, double cs,
                                     double cn, double eps, int rule, int det, int self_append,
                                     double* __restrict__ share, int64_t* __restrict__ cnt,
                                     int64_t* __restrict__ foff, int32_t* nfv, int32_t* nfs,
                                     int32_t ncap, Counters* C) {
  prnibble_vmap_body((int64_t)blockIdx.x * blockDim.x, nf, (int64_t)gridDim.x * blockDim.x, fv,
                     fs, T, off, alpha, cs, cn, eps, rule, det, self_append, share, cnt, foff,
                     nfv, nfs, ncap, C);
}

// Nibble, Fig. alg:nibble: p'[v] = p[v]/2 on the frontier (S = p, D = p',
// fresh), share p[v]/(2 d(v)).
__device__ inline int64_t nibble_vmap_body(int64_t i0, int64_t i1, int64_t step,
                                           const int32_t* fv, const int32_t* fs, Table S,
                                           Table D, const int64_t* __restrict__ off, double eps,
                                           int fmode, int det, int self_append, double* share,
                                           int64_t* cnt, int64_t* foff, int32_t* nfv,
                                           int32_t* nfs, int32_t ncap, Counters* C) {
  int64_t nins = 0;  // counted once per block
  int64_t csum = 0;
  for (int64_t base = i0; base < i1; base += step) {
    const int64_t i = base + threadIdx.x;
    bool pred = false;
    int ins = 0;
    int32_t v = 0, ds = 0;
    int64_t d = 0;
    if (i < i1) {
      v = fv[i];
      const double pv = fs[i] >= 0 ? *tb_val(S, fs[i]) : 0.0;
      const int64_t o0 = off[v];
      d = off[v + 1] - o0;
      ds = (int32_t)tb_find_or_insert(D, v, &ins, &C->err);
      const double self = pv / 2.0;
      if (ds >= 0) *tb_val(D, ds) = self;
      share[i] = pv / (2.0 * (double)d);
      cnt[i] = d + (det ? 1 : 0);
      csum += cnt[i];
      foff[i] = o0;
      if (self_append && ds >= 0)
        pred = fmode == kFmInserted ? true : self >= eps * (double)d;
    }
    nins += ins;
    frontier_append(pred, v, ds, d, nfv, nfs, C, ncap);
  }
  flush_count(nins, &C->aux);
  return csum;
}

__global__ void vmap_nibble_kernel(int64_t nf, const int32_t* __restrict__ fv,
                                   const int32_t* __restrict__ fs, Table S, Table D,
                                   const int64_t* __restrict__ off, double eps, int fmode,
                                   int det, int self_append, double* __restrict__ share,
                                   int64_t* __restrict__ cnt,
                                   int64_t* __restrict__ foff, int32_t* nfv, int32_t* nfs,
                                   int32_t ncap, Counters* C) {
  nibble_vmap_body((int64_t)blockIdx.x * blockDim.x, nf, (int64_t)gridDim.x * blockDim.x, fv, fs,
                   S, D, off, eps, fmode, det, self_append, share, cnt, foff, nfv, nfs, ncap, C);
}

// HK-PR, Fig. alg:hkpr: p[v] += r[v] on the frontier; share
// t r[v]/((j+1) d(v)) or, on the last level, r[v]/d(v).
__global__ void vmap_hkpr_kernel(int64_t nf, const int32_t* __restrict__ fv,
                                 const int32_t* __restrict__ fs, Table S, Table P,
                                 const int64_t* __restrict__ off, double t, int j, int last,
                                 double* __restrict__ share, int64_t* __restrict__ cnt,
                                 int64_t* __restrict__ foff, Counters* C) {
  int64_t nins = 0;  // counted once per block
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nf;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int ins = 0;
    if (i < nf) {
      const int32_t v = fv[i];
      const double r = fs[i] >= 0 ? *tb_val(S, fs[i]) : 0.0;
      const int64_t o0 = off[v];
      const int64_t d = off[v + 1] - o0;
      const int64_t ps = tb_find_or_insert(P, v, &ins, &C->err);
      if (ps >= 0) *tb_val(P, ps) = *tb_val(P, ps) + r;
      share[i] = last ? r / (double)d : (t * r) / ((double)(j + 1) * (double)d);
      cnt[i] = d;
      foff[i] = o0;
    }
    nins += ins;
  }
  flush_count(nins, &C->aux);
}

// ---------------------------------------------------------------------------
// edgeMap, atomic mode.  Edge-balanced: CTA tile k covers edges
// [k*kEdgeTile, (k+1)*kEdgeTile) of the frontier's concatenated adjacency
// lists; the tile's sources are found by binary search in the exclusive
// prefix sums of the frontier degrees and staged in shared memory, and each
// thread then finds its edge's source there.  Consecutive threads read
// consecutive col[] entries.
// ---------------------------------------------------------------------------
// The tiles [first tile, ntiles) of the edge push with the given stride.
__device__ inline void emap_atomic_body(const int32_t* __restrict__ col,
                                        const int32_t* __restrict__ deg, const double* share,
                                        const int64_t* epos, const int64_t* foff, int64_t nf,
                                        int64_t E, Table D, double c, int fmode, int32_t* nfv,
                                        int32_t* nfs, int32_t ncap, Counters* C) {
  __shared__ int64_t s_epos[kEdgeTile + 1];
  __shared__ int64_t s_off[kEdgeTile];
  __shared__ double s_share[kEdgeTile];
  __shared__ int64_t s_i0, s_i1;
  const int64_t ntiles = (E + kEdgeTile - 1) / kEdgeTile;
  int64_t nins = 0;  // counted once per block
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kEdgeTile;
    const int64_t e1 = min(E, e0 + kEdgeTile);
    const int cntsrc = stage_sources(epos, nf, E, e0, e1, &s_i0, &s_i1, s_epos);
    const int64_t i0 = s_i0;
    for (int j = threadIdx.x; j < cntsrc; j += kBlock) {
      s_off[j] = foff[i0 + j];
      s_share[j] = share[i0 + j];
    }
    __syncthreads();
    int32_t w[kEdgeItems];
    double sh[kEdgeItems];
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) {
      const int64_t e = e0 + k * kBlock + threadIdx.x;
      w[k] = -1;
      int64_t q;
      const int j = e < e1 ? find_source(s_epos, cntsrc, e, &q) : -1;
      if (j >= 0) {
        w[k] = col[s_off[j] + q];
        sh[k] = s_share[j];
      }
    }
    // Resolve every item's slot before any atomic, so the first-probe loads
    // (or bitmap loads) of all items are in flight together.
    int32_t slot[kEdgeItems];
    int ins[kEdgeItems];
    uint32_t probe[kEdgeItems];
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) {
      ins[k] = 0;
      probe[k] = 0;
      if (w[k] >= 0)
        probe[k] = D.dense ? __ldcg(&D.bits[w[k] >> 5])
                           : (uint32_t)__ldcg(&D.s[hash_slot(w[k], D.shift)].key);
    }
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) {
      slot[k] = -1;
      if (w[k] < 0) continue;
      if (D.dense) {
        slot[k] = w[k];
        const uint32_t m = 1u << (w[k] & 31);
        if (!(probe[k] & m) && !(atomicOr(&D.bits[w[k] >> 5], m) & m)) ins[k] = 1;
      } else if ((int32_t)probe[k] == w[k] + 1) {
        slot[k] = (int32_t)hash_slot(w[k], D.shift);
      } else {
        slot[k] = (int32_t)ht_find_or_insert(D, w[k], &ins[k], &C->err);
      }
    }
    // All adds issued back to back; their returned old values decide the
    // threshold crossings.
    double old[kEdgeItems];
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++)
      old[k] = slot[k] >= 0 ? atomicAdd(tb_val(D, slot[k]), sh[k]) : 0.0;
    bool pred[kEdgeItems];
    int64_t dw[kEdgeItems];
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) {
      pred[k] = false;
      dw[k] = 0;
      if (slot[k] < 0) continue;
      if (fmode == kFmThreshold) {
        const double nv = old[k] + sh[k];
        if (nv >= c) {  // c*d(w) >= c for d(w) >= 1: cheap pre-test
          dw[k] = deg[w[k]];
          const double thr = c * (double)dw[k];
          pred[k] = old[k] < thr && nv >= thr;
        }
      } else if (fmode == kFmInserted && ins[k]) {
        dw[k] = deg[w[k]];
        pred[k] = true;
      }
    }
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) {
      nins += ins[k];
      frontier_append(pred[k], w[k], slot[k], dw[k], nfv, nfs, C, ncap);
    }
    __syncthreads();
  }
  flush_count(nins, &C->inserted);
}

__global__ void __launch_bounds__(kBlock)
    emap_atomic_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ deg,
                       const double* __restrict__ share, const int64_t* __restrict__ epos,
                       const int64_t* __restrict__ foff, int64_t nf, int64_t E_host,
                       const int64_t* __restrict__ E_dev, Table D, double c, int fmode,
                       int32_t* nfv, int32_t* nfs, int32_t ncap, Counters* C) {
  // the device-computed total bounds every edge index, whatever the host passed
  emap_atomic_body(col, deg, share, epos, foff, nf, min(E_host, *E_dev), D, c, fmode, nfv, nfs,
                   ncap, C);
}

// ---------------------------------------------------------------------------
// edgeMap for bulk rounds (atomic mode, dense destination): the adds are
// fire-and-forget reductions (no returned value, so nothing waits on them)
// and the key is marked in the presence bitmap; the next frontier is formed
// afterwards by the dense filter.  Also used for the last HK-PR level (no
// frontier) in either table form.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock)
    emap_red_kernel(const int32_t* __restrict__ col, const double* __restrict__ share,
                    const int64_t* __restrict__ epos, const int64_t* __restrict__ foff,
                    int64_t nf, int64_t E_host, const int64_t* __restrict__ E_dev, Table D,
                    Counters* C) {
  __shared__ int64_t s_epos[kEdgeTile + 1];
  __shared__ int64_t s_off[kEdgeTile];
  __shared__ double s_share[kEdgeTile];
  __shared__ int64_t s_i0, s_i1;
  const int64_t E = min(E_host, *E_dev);
  const int64_t ntiles = (E + kEdgeTile - 1) / kEdgeTile;
  int64_t nins = 0;  // counted once per block
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kEdgeTile;
    const int64_t e1 = min(E, e0 + kEdgeTile);
    const int cntsrc = stage_sources(epos, nf, E, e0, e1, &s_i0, &s_i1, s_epos);
    const int64_t i0 = s_i0;
    for (int j = threadIdx.x; j < cntsrc; j += kBlock) {
      s_off[j] = foff[i0 + j];
      s_share[j] = share[i0 + j];
    }
    __syncthreads();
    int32_t w[kEdgeItems];
    double sh[kEdgeItems];
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) {
      const int64_t e = e0 + k * kBlock + threadIdx.x;
      w[k] = -1;
      int64_t q;
      const int j = e < e1 ? find_source(s_epos, cntsrc, e, &q) : -1;
      if (j >= 0) {
        w[k] = col[s_off[j] + q];
        sh[k] = s_share[j];
      }
    }
    int ins[kEdgeItems];
    if (D.dense) {
      // nothing waits here: the add and the presence bit are both reductions
      // (results unused); the keys this round inserted are counted by the
      // caller from the bitmap's population before and after
#pragma unroll
      for (int k = 0; k < kEdgeItems; k++) {
        ins[k] = 0;
        if (w[k] < 0) continue;
        atomicAdd(&D.dval[w[k]], sh[k]);
        atomicOr(&D.bits[w[k] >> 5], 1u << (w[k] & 31));
      }
    } else {
#pragma unroll
      for (int k = 0; k < kEdgeItems; k++) {
        ins[k] = 0;
        if (w[k] < 0) continue;
        const int64_t s = ht_find_or_insert(D, w[k], &ins[k], &C->err);
        if (s >= 0) atomicAdd(&D.s[s].val, sh[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kEdgeItems; k++) nins += ins[k];
    __syncthreads();
  }
  flush_count(nins, &C->inserted);
}

// ---------------------------------------------------------------------------
// Consecutive small PR-Nibble rounds (atomic mode) in one cooperative launch:
// vertexMap, prefix sum of the frontier degrees, edge push with the
// threshold-crossing append, and the frontier swap, separated by grid-wide
// barriers, with no return to the host between rounds.  The kernel stops
// (leaving the state for the host, which continues with the same rounds
// one launch per step) when the frontier is empty, the round limit is
// reached, or the next round is not small: more than e_max edges, a next
// frontier that might not fit the buffers, or a table that might pass its
// load limit.  Each round computes exactly what the host-driven round does.
// ---------------------------------------------------------------------------
struct RoundsState {
  int32_t cur;   // frontier buffer of the current round (0 or 1)
  int32_t stop;  // 1 empty frontier, 2 round limit, 3 round not small, 4 error flagged
  int64_t count, rounds, pushes, pushed_edges;
  int32_t ptab;  // Nibble: the table holding p (0 the initial one, 1 A, 2 B)
};

__device__ inline int64_t block_sum_i64(int64_t x, int64_t* s_red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
  __syncthreads();
  int64_t t = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_red[k];
  __syncthreads();
  return t;
}

// The grid-wide exclusive prefix sum of cnt[0, nf) into epos: block b owns
// the chunk [c0, c1) of grid_chunk, writes the sum of cnt over it into
// bsum[b], and after a grid barrier grid_scan_tail scans its chunk from the
// sums of the chunks before it and returns the total (every thread of the
// grid calls it).
__device__ inline void grid_chunk(int64_t nf, int64_t* c0, int64_t* c1) {
  const int64_t chunk = (nf + gridDim.x - 1) / gridDim.x;
  *c0 = min(nf, (int64_t)blockIdx.x * chunk);
  *c1 = min(nf, *c0 + chunk);
}

__device__ inline int64_t grid_scan_tail(const int64_t* cnt, int64_t nf, int64_t* epos,
                                         const int64_t* bsum) {
  __shared__ int64_t s_red[kBlock / 32];
  __shared__ int64_t s_scan[kBlock / 32];
  const int G = gridDim.x;
  int64_t c0, c1;
  grid_chunk(nf, &c0, &c1);
  int64_t pre = 0, tot = 0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    const int64_t x = __ldcg(&bsum[b]);
    tot += x;
    if (b < (int)blockIdx.x) pre += x;
  }
  pre = block_sum_i64(pre, s_red);
  tot = block_sum_i64(tot, s_red);
  for (int64_t base = c0; base < c1; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t x = i < c1 ? cnt[i] : 0;
    int64_t inc = x;  // inclusive scan within the warp, then across warps
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((threadIdx.x & 31) >= o) inc += y;
    }
    if ((threadIdx.x & 31) == 31) s_scan[threadIdx.x >> 5] = inc;
    __syncthreads();
    int64_t wpre = 0, btot = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      if (k < (int)(threadIdx.x >> 5)) wpre += s_scan[k];
      btot += s_scan[k];
    }
    if (i < c1) epos[i] = pre + wpre + inc - x;
    pre += btot;
    __syncthreads();
  }
  return tot;
}

// Every thread keeps the round state (frontier buffer, rounds, pushes,
// keys) in registers, updated alike from the counters each round wrote once
// the grid has synchronised; the state goes to S when the kernel stops.  A
// round: the vertexMap over each block's chunk of the frontier with the
// chunk's record count | barrier | the scan | barrier | the edge push |
// barrier.  The current round's counters are cleared after the first
// barrier (nothing reads them after it), for their reuse as the next
// round's "next".
__global__ void __launch_bounds__(kBlock)
    rounds_prnibble_kernel(Table T, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ col, const int32_t* __restrict__ deg,
                           double alpha, double cs, double cn, double eps, int rule,
                           int32_t* fv0, int32_t* fs0, int32_t* fv1, int32_t* fs1, int32_t fcap,
                           double* share, int64_t* cnt, int64_t* epos, int64_t* foff,
                           int64_t* bsum, Counters* Cn, RoundsState* S, int64_t max_rounds,
                           int64_t e_max, int64_t key_limit) {
  cg::grid_group grid = cg::this_grid();
  __shared__ int64_t s_red[kBlock / 32];
  int cur = __ldcg(&S->cur);
  int64_t count = __ldcg(&S->count), rounds = __ldcg(&S->rounds);
  int64_t pushes = __ldcg(&S->pushes), pushed = __ldcg(&S->pushed_edges);
  for (;;) {
    const int nxt = cur ^ 1;
    const int64_t nf = __ldcg(&Cn[cur].next_size);
    const int64_t E = __ldcg(&Cn[cur].next_edges);
    const int err = __ldcg(&Cn[cur].err) | __ldcg(&Cn[nxt].err);
    int stop = 0;
    if (err) stop = 4;
    else if (nf == 0) stop = 1;
    else if (rounds >= max_rounds) stop = 2;
    else if (E > e_max || nf + E > fcap || count + E > key_limit) stop = 3;
    if (stop) {  // the same decision in every thread: no barrier is left waiting
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->cur = cur;
        S->stop = stop;
        S->count = count;
        S->rounds = rounds;
        S->pushes = pushes;
        S->pushed_edges = pushed;
      }
      return;
    }
    int32_t* fv = cur ? fv1 : fv0;
    int32_t* fs = cur ? fs1 : fs0;
    int32_t* nfv = cur ? fv0 : fv1;
    int32_t* nfs = cur ? fs0 : fs1;
    // vertexMap (the original rule keeps a vertex whose reduced residual
    // still reaches the threshold)
    int64_t c0, c1;
    grid_chunk(nf, &c0, &c1);
    int64_t part = prnibble_vmap_body(c0, c1, blockDim.x, fv, fs, T, off, alpha, cs, cn, eps,
                                      rule, 0, 1, share, cnt, foff, nfv, nfs, fcap, &Cn[nxt]);
    part = block_sum_i64(part, s_red);
    if (threadIdx.x == 0) bsum[blockIdx.x] = part;
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) Cn[cur] = Counters{};
    const int64_t tot = grid_scan_tail(cnt, nf, epos, bsum);
    grid.sync();
    // edge push into the same table, appending crossings to the next frontier
    emap_atomic_body(col, deg, share, epos, foff, nf, min(E, tot), T, eps, kFmThreshold, nfv,
                     nfs, fcap, &Cn[nxt]);
    grid.sync();
    rounds += 1;
    pushes += nf;
    pushed += E;
    count += __ldcg(&Cn[nxt].inserted);
    cur = nxt;
  }
}

// Nibble (Fig. alg:nibble, atomic mode) the same way: each round fills a
// fresh p' from p, so two hashed tables of capacity cap alternate as p'
// (A in device round 0, 2, ..., B in 1, 3, ...; both clear at launch) and p
// starts in T0 (any form), the table the host's rounds left.  A round runs
// the vertexMap (p'[v] = p[v]/2, appending v if that reaches the threshold),
// the scan and the edge push into p'.  When the new frontier is empty the
// run is over and p stays where it was (the method returns the previous p);
// otherwise p' becomes p and the old p, when it is A or B, is cleared in a
// fourth phase to serve as the next round's p'.  key_limit is cap / 2: a
// round whose keys (at most |F| + its edges) could pass it stops the kernel
// first.
__global__ void __launch_bounds__(kBlock)
    rounds_nibble_kernel(Table T0, Table A, Table B, const int64_t* __restrict__ off,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ deg,
                         double eps, int fmode, int32_t* fv0, int32_t* fs0, int32_t* fv1,
                         int32_t* fs1, int32_t fcap, double* share, int64_t* cnt, int64_t* epos,
                         int64_t* foff, int64_t* bsum, Counters* Cn, RoundsState* S,
                         int64_t max_rounds, int64_t e_max, int64_t key_limit) {
  cg::grid_group grid = cg::this_grid();
  __shared__ int64_t s_red[kBlock / 32];
  int cur = __ldcg(&S->cur), ptab = __ldcg(&S->ptab);
  int64_t count = __ldcg(&S->count), k = __ldcg(&S->rounds);
  int64_t pushes = __ldcg(&S->pushes), pushed = __ldcg(&S->pushed_edges);
  auto finish = [&](int stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->cur = cur;
      S->ptab = ptab;
      S->stop = stop;
      S->count = count;
      S->rounds = k;
      S->pushes = pushes;
      S->pushed_edges = pushed;
    }
  };
  for (;;) {
    const int nxt = cur ^ 1;
    const int64_t nf = __ldcg(&Cn[cur].next_size);
    const int64_t E = __ldcg(&Cn[cur].next_edges);
    const int err = __ldcg(&Cn[cur].err) | __ldcg(&Cn[nxt].err);
    int stop = 0;
    if (err) stop = 4;
    else if (nf == 0) stop = 1;
    else if (k >= max_rounds) stop = 2;
    else if (E > e_max || nf + E > fcap || nf + E > key_limit) stop = 3;
    if (stop) {  // the same decision in every thread: no barrier is left waiting
      finish(stop);
      return;
    }
    const Table P = ptab == 0 ? T0 : ptab == 1 ? A : B;
    const Table Q = (k & 1) ? B : A;  // never P: P is T0 or the other one
    int32_t* fv = cur ? fv1 : fv0;
    int32_t* fs = cur ? fs1 : fs0;
    int32_t* nfv = cur ? fv0 : fv1;
    int32_t* nfs = cur ? fs0 : fs1;
    int64_t c0, c1;
    grid_chunk(nf, &c0, &c1);
    int64_t part = nibble_vmap_body(c0, c1, blockDim.x, fv, fs, P, Q, off, eps, fmode, 0, 1,
                                    share, cnt, foff, nfv, nfs, fcap, &Cn[nxt]);
    part = block_sum_i64(part, s_red);
    if (threadIdx.x == 0) bsum[blockIdx.x] = part;
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) Cn[cur] = Counters{};
    const int64_t tot = grid_scan_tail(cnt, nf, epos, bsum);
    grid.sync();
    emap_atomic_body(col, deg, share, epos, foff, nf, min(E, tot), Q, eps, fmode, nfv, nfs, fcap,
                     &Cn[nxt]);
    grid.sync();
    k += 1;
    pushes += nf;
    pushed += E;
    if (__ldcg(&Cn[nxt].next_size) == 0) {  // the previous p is the result
      finish(1);
      return;
    }
    count = __ldcg(&Cn[nxt].aux) + __ldcg(&Cn[nxt].inserted);
    if (ptab != 0) {  // the old p (A or B) becomes the next round's p'
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.cap;
           i += (int64_t)gridDim.x * blockDim.x)
        P.s[i] = Slot{};
    }
    ptab = ((k - 1) & 1) ? 2 : 1;
    cur = nxt;
    grid.sync();
  }
}

__global__ void rounds_init_kernel(Counters* Cn, RoundsState* S, int64_t nf, int64_t E,
                                   int64_t count) {
  Cn[0] = Counters{};
  Cn[1] = Counters{};
  Cn[0].next_size = (int32_t)nf;
  Cn[0].next_edges = E;
  *S = RoundsState{};
  S->count = count;
}

// out: stop | err << 8 | ptab << 16, cur, frontier size, its edges, keys,
// rounds, pushes, pushed edges
__global__ void rounds_pack_kernel(const Counters* Cn, const RoundsState* S, int64_t* out) {
  const int cur = S->cur;
  out[0] = (int64_t)S->stop | ((int64_t)(Cn[0].err | Cn[1].err) << 8) | ((int64_t)S->ptab << 16);
  out[1] = cur;
  out[2] = Cn[cur].next_size;
  out[3] = Cn[cur].next_edges;
  out[4] = S->count;
  out[5] = S->rounds;
  out[6] = S->pushes;
  out[7] = S->pushed_edges;
}

// sign * (set bits of the bitmap) added into *out, one atomic per block.
__global__ void bits_pop_kernel(const uint32_t* __restrict__ bits, int64_t words, int sign,
                                int64_t* out) {
  __shared__ unsigned long long s_pop;
  if (threadIdx.x == 0) s_pop = 0;
  __syncthreads();
  unsigned long long c = 0;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x)
    c += __popc(bits[w]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_pop, c);
  __syncthreads();
  if (threadIdx.x == 0 && s_pop)
    atomicAdd((unsigned long long*)out, (unsigned long long)((int64_t)sign * (int64_t)s_pop));
}

// Filter of a dense set, in ascending vertex order: vertex v qualifies when it
// is a key and its value reaches c*d(v) (kFmThreshold) or always
// (kFmInserted); the qualifying vertices are compacted in one launch
// (compact_words_kernel), which also sums their degrees.
__device__ inline uint32_t dense_qualifying(const Table& D, const int32_t* __restrict__ deg,
                                            int64_t w, int64_t n, double c, int fmode) {
  uint32_t m = D.bits[w];
  if (fmode != kFmThreshold) return m;
  uint32_t q = 0;
  while (m) {
    const int b = __ffs(m) - 1;
    m &= m - 1;
    const int64_t v = w * 32 + b;
    if (v < n && D.dval[v] >= c * (double)deg[v]) q |= 1u << b;
  }
  return q;
}

// The filter's bitmap word w, for compact_words_kernel.
struct DenseQualWord {
  Table D;
  const int32_t* deg;
  int64_t n;
  double c;
  int fmode;
  __device__ uint32_t operator()(int64_t w) const {
    return dense_qualifying(D, deg, w, n, c, fmode);
  }
};

// ---------------------------------------------------------------------------
// Pull edgeMap (deterministic mode, dense rounds).  Instead of scattering
// from the frontier, every vertex w gathers from its neighbours that are in
// the frontier.  Adjacency lists are sorted, so w meets its in-frontier
// neighbours in ascending id: folding their shares left to right from w's
// current value is exactly the canonical order, with no records and no sort.
// The frontier is given as one double per vertex, sh[v]: +0.0 (all bits
// zero) for a vertex outside the frontier, its share for a frontier vertex,
// and -0.0 for a frontier vertex whose share is zero.  So one gather gives
// both membership (any bit set) and the value, and adding a member's -0.0 to
// a non-negative value changes nothing, exactly as its +0.0 share would.
// Vertices of degree <= kPullLight use one thread, the rest (ascending list
// g->heavy) are read in batches by warps.  Qualifying vertices are marked in
// qbits for an ordered compaction.
// ---------------------------------------------------------------------------
__device__ inline bool pull_member(double s) { return __double_as_longlong(s) != 0; }

__global__ void pull_scatter_kernel(int64_t nf, const int32_t* __restrict__ fv,
                                    const double* __restrict__ share, double* __restrict__ sh,
                                    int clear) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = fv[i];
    if (clear) {
      sh[v] = 0.0;
      continue;
    }
    const double x = share[i];
    sh[v] = pull_member(x) ? x : -0.0;
  }
}

__device__ inline bool pull_qualifies(double acc, int64_t d, double c, int fmode) {
  if (fmode == kFmThreshold) return acc >= c * (double)d;
  return fmode == kFmInserted;
}

// Deterministic pull, vertices of degree 1..kPullLight: one thread folds its
// list in order (acc <- RN(acc + s) from the present value), taking the
// vertices from the graph's list grouped by degree so that a warp's chains
// have one length.  qbits is cleared before; qualifying vertices are ORed in.
__global__ void pull_light_kernel(const LightItem* __restrict__ items, int64_t nl,
                                  const int32_t* __restrict__ col,
                                  const double* __restrict__ sh, Table D, double c, int fmode,
                                  uint32_t* __restrict__ qbits, Counters* C) {
  int64_t nins = 0;  // keys inserted here, counted once per block
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    const LightItem it = items[i];
    const int32_t w = it.w;
    const uint32_t m = 1u << (w & 31);
    const bool present = (D.bits[w >> 5] & m) != 0;
    double acc = present ? D.dval[w] : 0.0;
    bool touched = present;
    for (int k = 0; k < it.d; k++) {
      const double x = sh[col[it.beg + k]];
      if (pull_member(x)) {
        acc = acc + x;
        touched = true;
      }
    }
    if (touched) {
      D.dval[w] = acc;
      if (!present && !(atomicOr(&D.bits[w >> 5], m) & m)) nins++;
      if (pull_qualifies(acc, it.d, c, fmode)) atomicOr(&qbits[w >> 5], m);
    }
  }
  flush_count(nins, &C->inserted);
}

// Heavy vertices are read in batches of 32 * BATCH edges: every lane issues
// the loads of BATCH edges (column, then share) before any of them is used,
// so one batch costs two memory round trips; BATCH is the graph's tuned value
// (kPullBatch until tuned).
constexpr int kPullBatch = 8;

// Writes a heavy vertex's gathered value (lane 0 calls it); 1 if the vertex
// became a key here (the caller counts it).
__device__ inline int pull_finish(const Table& D, int32_t w, int64_t d, double acc, bool touched,
                                  bool present, double c, int fmode, uint32_t* qbits) {
  if (!touched) return 0;
  const uint32_t m = 1u << (w & 31);
  D.dval[w] = acc;
  const int ins = !present && !(atomicOr(&D.bits[w >> 5], m) & m);
  if (pull_qualifies(acc, d, c, fmode)) atomicOr(&qbits[w >> 5], m);
  return ins;
}

// ---------------------------------------------------------------------------
// The ordered fold acc <- RN(acc + s_k) of 256 shares by a warp, without a
// chain of dependent FP64 adds (the segment-parallel fold of long lists
// refolds a segment with it where its composed step does not apply).
//
// While acc stays in one binade it is A * u with the integer A below 2^53,
// and each share is an integer step A -> A + g[A & 1] (fold_step in
// fx128.cuh); steps compose, so a warp scan of the compositions gives every
// partial fold.  The first position whose value reaches 2^53 leaves the
// binade: that one add is done in FP64 (the rounding of the next binade
// applies), and the scan restarts after it with the new binade.  Every
// result equals the sequential fold's bit for bit.
// ---------------------------------------------------------------------------
// Folds the 32 * 8 shares v (lane l holds positions 8l .. 8l+7, in list
// order) into acc, lane-uniformly.
__device__ inline double fold_batch(double acc, const double v[8], int lane) {
  int start = 0;
  while (start < 256) {
    const int bu = fold_binade(acc);
    const int64_t A0 = fold_int(acc);
    FoldStep st[8];
    FoldStep F = {0, 0};
#pragma unroll
    for (int j = 0; j < 8; j++) {
      st[j] = 8 * lane + j >= start ? fold_step(v[j], bu) : FoldStep{0, 0};
      F = fold_compose(F, st[j]);
    }
    // inclusive scan over lanes, then shift to exclusive
    FoldStep P = F;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      FoldStep q;
      q.g0 = __shfl_up_sync(0xffffffffu, P.g0, o);
      q.g1 = __shfl_up_sync(0xffffffffu, P.g1, o);
      if (lane >= o) P = fold_compose(q, P);
    }
    FoldStep E;
    E.g0 = __shfl_up_sync(0xffffffffu, P.g0, 1);
    E.g1 = __shfl_up_sync(0xffffffffu, P.g1, 1);
    if (lane == 0) E = {0, 0};
    int64_t A = fold_apply(E, A0);
    int cj = -1;
    int64_t before = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int64_t nx = fold_apply(st[j], A);
      if (cj < 0 && nx >= kFoldTop) {
        cj = j;
        before = A;
      }
      A = nx;
    }
    const unsigned crossed = __ballot_sync(0xffffffffu, cj >= 0);
    if (!crossed) {
      const int64_t Aend = __shfl_sync(0xffffffffu, A, 31);
      return fold_double(Aend, bu);
    }
    const int lc = __ffs(crossed) - 1;
    double nacc = 0.0;
    if (lane == lc) {
      double sj = 0.0;
#pragma unroll
      for (int j = 0; j < 8; j++)
        if (j == cj) sj = v[j];
      nacc = fold_double(before, bu) + sj;  // the add that leaves the binade
    }
    acc = __shfl_sync(0xffffffffu, nacc, lc);
    start = 8 * lc + __shfl_sync(0xffffffffu, cj, lc) + 1;
  }
  return acc;
}

// Deterministic mode, vertices of degree (kPullLight, kDetBig]: one lane per
// vertex folds its in-frontier shares in adjacency order with FP64 adds --
// the fold's definition, so bit-identical by construction.  The vertices are
// taken longest list first and a warp's lanes have lists of similar length,
// so every add is issued for (nearly) all 32 lanes; each lane loads eight
// columns, then their eight shares, before folding them.
__global__ void __launch_bounds__(kBlock)
    pull_mid_det_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                        const int32_t* __restrict__ mid, int64_t nmid,
                        const double* __restrict__ sh, Table D, double c, int fmode,
                        uint32_t* __restrict__ qbits, Counters* C) {
  int64_t nins = 0;  // keys inserted here, counted once per block
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nmid;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int ins = 0;
    if (i < nmid) {
      const int32_t w = mid[i];
      const int64_t o0 = off[w], d = off[w + 1] - o0;
      const uint32_t m = 1u << (w & 31);
      const bool present = (D.bits[w >> 5] & m) != 0;
      double acc = present ? D.dval[w] : 0.0;
      bool touched = present;
      // software-pipelined: the next batch's shares and the batch after's
      // columns are read before this batch's adds, so a batch costs the
      // larger of one memory trip and its sixteen dependent adds, not both
      int32_t u[16], un[16];
      double x[16];
#pragma unroll
      for (int j = 0; j < 16; j++) u[j] = j < d ? col[o0 + j] : -1;
#pragma unroll
      for (int j = 0; j < 16; j++) un[j] = 16 + j < d ? col[o0 + 16 + j] : -1;
#pragma unroll
      for (int j = 0; j < 16; j++) x[j] = u[j] >= 0 ? sh[u[j]] : 0.0;
      for (int64_t k = 0; k < d; k += 16) {
        double xn[16];
#pragma unroll
        for (int j = 0; j < 16; j++) xn[j] = un[j] >= 0 ? sh[un[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < 16; j++) u[j] = k + 32 + j < d ? col[o0 + k + 32 + j] : -1;
#pragma unroll
        for (int j = 0; j < 16; j++) {
          if (pull_member(x[j])) {  // in order: j ascending is adjacency order
            acc = acc + x[j];
            touched = true;
          }
        }
#pragma unroll
        for (int j = 0; j < 16; j++) {
          x[j] = xn[j];
          un[j] = u[j];
        }
      }
      if (touched) {
        D.dval[w] = acc;
        if (!present && !(atomicOr(&D.bits[w >> 5], m) & m)) ins = 1;
        if (pull_qualifies(acc, d, c, fmode)) atomicOr(&qbits[w >> 5], m);
      }
    }
    nins += ins;
  }
  flush_count(nins, &C->inserted);
}

// ---------------------------------------------------------------------------
// Deterministic mode, vertices of degree > kDetBig: the fold of the whole
// list is split into 256-edge segments that are worked on in parallel.
//  1. det_seg_sum: each segment's plain sum and whether it holds a member.
//  2. det_seg_predict: per vertex, a running sum of the segment sums
//     predicts the binade the fold is in at each segment's start (the fold
//     differs from the exact prefix sum by rounding only, so the prediction
//     misses only next to a power of two).
//  3. det_seg_step: each segment's composed integer step (see fold_step) for
//     its predicted binade.
//  4. det_seg_verify: one warp per vertex walks its segments in order: when
//     the fold's actual binade is the predicted one and the composed step
//     keeps the value below 2^53, the step is the exact fold of the segment
//     (the value only grows, so no intermediate value left the binade);
//     otherwise the segment is folded element by element (fold_batch).
// The result is the sequential fold, bit for bit.
// ---------------------------------------------------------------------------
__global__ void det_seg_sum_kernel(const int32_t* __restrict__ col,
                                   const DetSeg* __restrict__ segs, int64_t nsegs,
                                   const double* __restrict__ sh, double* __restrict__ segsum,
                                   int32_t* __restrict__ segany) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp0; k < nsegs; k += nwarps) {
    const DetSeg S = segs[k];
    int32_t u[8];
#pragma unroll
    for (int j = 0; j < 8; j++) u[j] = 32 * j + lane < S.len ? col[S.beg + 32 * j + lane] : -1;
    double x = 0.0;
    bool mem = false;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const double v = u[j] >= 0 ? sh[u[j]] : 0.0;
      x += v;
      mem = mem || pull_member(v);
    }
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const bool any = __any_sync(0xffffffffu, mem);
    if (lane == 0) {
      segsum[k] = x;
      segany[k] = any ? 1 : 0;
    }
  }
}

__global__ void det_seg_predict_kernel(const int32_t* __restrict__ big_w,
                                       const int64_t* __restrict__ seg0, int64_t nbig, Table D,
                                       const double* __restrict__ segsum,
                                       int32_t* __restrict__ pred) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbig;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = big_w[b];
    const bool present = (D.bits[w >> 5] >> (w & 31)) & 1u;
    double acc = present ? D.dval[w] : 0.0;
    for (int64_t k = seg0[b]; k < seg0[b + 1]; k++) {
      pred[k] = fold_binade(acc);
      acc += segsum[k];
    }
  }
}

__global__ void det_seg_step_kernel(const int32_t* __restrict__ col,
                                    const DetSeg* __restrict__ segs, int64_t nsegs,
                                    const double* __restrict__ sh,
                                    const int32_t* __restrict__ pred,
                                    FoldStep* __restrict__ step) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp0; k < nsegs; k += nwarps) {
    const DetSeg S = segs[k];
    const int bu = pred[k];
    int32_t u[8];
#pragma unroll
    for (int j = 0; j < 8; j++) u[j] = 8 * lane + j < S.len ? col[S.beg + 8 * lane + j] : -1;
    FoldStep F = {0, 0};
#pragma unroll
    for (int j = 0; j < 8; j++)
      F = fold_compose(F, fold_step(u[j] >= 0 ? sh[u[j]] : 0.0, bu));
    // ordered reduction: lane l's steps come before lane l+1's
    for (int o = 1; o < 32; o <<= 1) {
      FoldStep q;
      q.g0 = __shfl_down_sync(0xffffffffu, F.g0, o);
      q.g1 = __shfl_down_sync(0xffffffffu, F.g1, o);
      if ((lane & (2 * o - 1)) == 0) F = fold_compose(F, q);
    }
    if (lane == 0) step[k] = F;
  }
}

__global__ void __launch_bounds__(kBlock)
    det_seg_verify_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                          const DetSeg* __restrict__ segs, const int32_t* __restrict__ big_w,
                          const int64_t* __restrict__ seg0, int64_t nbig,
                          const double* __restrict__ sh, const int32_t* __restrict__ pred,
                          const FoldStep* __restrict__ step, const int32_t* __restrict__ segany,
                          Table D, double c, int fmode, uint32_t* __restrict__ qbits,
                          Counters* C) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t nins = 0;
  for (int64_t b = warp0; b < nbig; b += nwarps) {
    const int32_t w = big_w[b];
    const bool present = (D.bits[w >> 5] >> (w & 31)) & 1u;
    double acc = present ? D.dval[w] : 0.0;  // >= +0, the same in every lane
    bool touched = present;
    const int64_t k1 = seg0[b + 1];
    for (int64_t k0 = seg0[b]; k0 < k1; k0 += 32) {
      // 32 segments' predictions and steps, one per lane, walked in order
      const int64_t kl = k0 + lane;
      const bool ok = kl < k1;
      const int pl = ok ? pred[kl] : 0;
      const FoldStep sl = ok ? step[kl] : FoldStep{0, 0};
      touched = touched || __any_sync(0xffffffffu, ok && segany[kl] != 0);
      const int cnt = (int)min((int64_t)32, k1 - k0);
      for (int j = 0; j < cnt; j++) {
        const int pj = __shfl_sync(0xffffffffu, pl, j);
        FoldStep sj;
        sj.g0 = __shfl_sync(0xffffffffu, sl.g0, j);
        sj.g1 = __shfl_sync(0xffffffffu, sl.g1, j);
        const int bu = fold_binade(acc);
        if (bu == pj) {
          const int64_t A = fold_apply(sj, fold_int(acc));
          if (A < kFoldTop) {
            acc = fold_double(A, bu);
            continue;
          }
        }
        // the prediction missed or the segment leaves the binade: fold it
        // element by element
        const DetSeg S = segs[k0 + j];
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int pos = 8 * lane + q;
          v[q] = pos < S.len ? sh[col[S.beg + pos]] : 0.0;
        }
        acc = fold_batch(acc, v, lane);
      }
    }
    if (lane == 0)
      nins += pull_finish(D, w, off[w + 1] - off[w], acc, touched, present, c, fmode, qbits);
  }
  flush_count(nins, &C->inserted);
}

// ---------------------------------------------------------------------------
// Pull edgeMap, atomic mode.  The order of the adds is free, so the gather
// sums in 128-bit fixed point (fx128.cuh) instead of FP64: per edge one
// 16-byte load and four integer adds, and per vertex one rounding.  The
// round's scale L comes from the range of the frontier's shares:
// range[0] = max over nonzero shares of (2047 - biased exponent),
// range[1] = max biased exponent (both 0 before the round).
// shx[v] = {X, flag} for a frontier vertex v, {0, 0} otherwise.
// ---------------------------------------------------------------------------
// A share's contribution to the range (emin holds 2047 - biased exponent).
__device__ inline void range_take(double x, int& emin, int& emax) {
  const uint64_t b = fx_bits(x) & kFxMask;
  if (b) {
    const int be = fx_bexp(b);
    emin = max(emin, 2047 - be);
    emax = max(emax, be);
  }
}

// The block's range into range[] (every thread of the block calls it).
__device__ inline void range_flush(int emin, int emax, int32_t* __restrict__ range) {
  __shared__ int s_r[2][kBlock / 32];
  // one atomic pair per block: same-address atomics serialise in L2
  emin = __reduce_max_sync(0xffffffffu, emin);
  emax = __reduce_max_sync(0xffffffffu, emax);
  const int wib = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_r[0][wib] = emin;
    s_r[1][wib] = emax;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    emin = threadIdx.x < kBlock / 32 ? s_r[0][threadIdx.x] : 0;
    emax = threadIdx.x < kBlock / 32 ? s_r[1][threadIdx.x] : 0;
    emin = __reduce_max_sync(0xffffffffu, emin);
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (threadIdx.x == 0 && (emin | emax)) {
      atomicMax(&range[0], emin);
      atomicMax(&range[1], emax);
    }
  }
}

__global__ void share_range_kernel(int64_t nf, const double* __restrict__ share,
                                   int32_t* __restrict__ range) {
  int emin = 0, emax = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x)
    range_take(share[i], emin, emax);
  range_flush(emin, emax, range);
}

// HK-PR vertexMap of a pull round gathering 8-byte shares: the step of
// vmap_hkpr_kernel, with the share written straight into the per-vertex
// array the gathers read (pull_scatter_kernel's membership encoding) and, in
// atomic mode (range non-null, zeroed before), the shares' exponent range
// reduced here; a pull round needs no push records.
__global__ void vmap_hkpr_pull_kernel(int64_t nf, const int32_t* __restrict__ fv,
                                      const int32_t* __restrict__ fs, Table S, Table P,
                                      const int32_t* __restrict__ deg, double t, int j, int last,
                                      double* __restrict__ sh, int32_t* __restrict__ range,
                                      Counters* C) {
  int emin = 0, emax = 0;
  int64_t nins = 0;  // counted once per block
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nf;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int ins = 0;
    if (i < nf) {
      const int32_t v = fv[i];
      const double r = fs[i] >= 0 ? *tb_val(S, fs[i]) : 0.0;
      const int64_t d = deg[v];
      const int64_t ps = tb_find_or_insert(P, v, &ins, &C->err);
      if (ps >= 0) *tb_val(P, ps) = *tb_val(P, ps) + r;
      const double x = last ? r / (double)d : (t * r) / ((double)(j + 1) * (double)d);
      sh[v] = pull_member(x) ? x : -0.0;
      range_take(x, emin, emax);
    }
    nins += ins;
  }
  flush_count(nins, &C->aux);
  if (range) range_flush(emin, emax, range);
}

__device__ inline int round_scale(const int32_t* range, int g) {
  return fx_scale(2047 - range[0], range[1], g);
}

// The gathered frontier share as a fixed-point record: either stored so
// (16 bytes per vertex), or stored as the double share with the membership
// encoding of the deterministic pull (+0.0 outside the frontier, -0.0 for a
// zero share) and converted here (8 bytes per vertex, a few integer
// operations per edge).  Same value either way.
__device__ inline Fx to_fx(const Fx& x, int) { return x; }
__device__ inline Fx to_fx(double s, int L) {
  const uint64_t b = fx_bits(s);
  Fx x = fx_from_bits(b, L);  // -0.0 -> 0
  x.hi |= (uint64_t)(b != 0) << 63;
  return x;
}
template <typename SH>
__device__ inline SH no_share();
template <>
__device__ inline Fx no_share<Fx>() {
  return Fx{0, 0};
}
template <>
__device__ inline double no_share<double>() {
  return 0.0;
}

__global__ void pull_scatter_fx_kernel(int64_t nf, const int32_t* __restrict__ fv,
                                       const double* __restrict__ share, Fx* __restrict__ shx,
                                       const int32_t* __restrict__ range, int g, int clear) {
  const int L = clear ? 0 : round_scale(range, g);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    Fx x = {0, 0};
    if (!clear) {
      x = fx_from_double(share[i], L);
      x.hi |= kFxFlag;
    }
    shx[fv[i]] = x;
  }
}

// Autotuning input: every vertex in the frontier with share 1 (X = 1 at
// the scale the range {1023, 1023} gives).
template <typename SH>
__global__ void tune_fill_kernel(SH* __restrict__ shx, int64_t n, int32_t* __restrict__ range,
                                 int g) {
  const int L = fx_scale(1023, 1023, g);
  const Fx one = fx_from_double(1.0, L);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(SH) == sizeof(Fx)) {
      shx[v] = Fx{one.lo, one.hi | kFxFlag};
    } else {
      shx[v] = 1.0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    range[0] = 2047 - 1023;
    range[1] = 1023;
  }
}

// Vertices of degree 1..kPullLight, one thread each, taken from the graph's
// list grouped by degree so that the threads of a warp walk lists of one
// length (in id order most of a warp idled behind its longest list); the
// edges are read four at a time (all column loads, then all share loads).
// The bitmap qbits is cleared before this launch; this kernel and the heavy
// one OR their qualifying vertices in.
template <typename SH>
__device__ inline void pull_light_fx_body(int64_t bid, int64_t nblk,
                                          const LightItem* __restrict__ items, int64_t nl,
                                          const int32_t* __restrict__ col,
                                          const SH* __restrict__ shx,
                                          const int32_t* __restrict__ range, int g, Table D,
                                          double c, int fmode, uint32_t* __restrict__ qbits,
                                          Counters* C) {
  const int L = round_scale(range, g);
  int64_t nins = 0;  // keys inserted here, counted once per block
  for (int64_t i = bid * blockDim.x + threadIdx.x; i < nl; i += nblk * blockDim.x) {
    const LightItem it = items[i];
    const int32_t w = it.w, d = it.d;
    Fx acc = {0, 0};
    uint64_t flag = 0;
    for (int k = 0; k < d; k += 4) {
      int32_t u[4];
#pragma unroll
      for (int j = 0; j < 4; j++) u[j] = k + j < d ? col[it.beg + k + j] : -1;
      SH raw[4];
#pragma unroll
      for (int j = 0; j < 4; j++) raw[j] = u[j] >= 0 ? shx[u[j]] : no_share<SH>();
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const Fx x = to_fx(raw[j], L);
        flag |= x.hi;
        fx_add(acc, x);
      }
    }
    const uint32_t m = 1u << (w & 31);
    const bool present = (D.bits[w >> 5] & m) != 0;
    if (present || (flag & kFxFlag)) {
      const double v = (present ? D.dval[w] : 0.0) + fx_to_double(acc, L);
      D.dval[w] = v;
      if (!present && !(atomicOr(&D.bits[w >> 5], m) & m)) nins++;
      if (pull_qualifies(v, d, c, fmode)) atomicOr(&qbits[w >> 5], m);
    }
  }
  flush_count(nins, &C->inserted);
}

// Heavy vertices: one warp per work item (at most kPullItem edges of one
// heavy vertex); lanes sum strided parts, then a butterfly.  The item's
// record and the vertex's current state are loaded first and the latter is
// not waited for until the end, so an item costs three dependent memory
// trips (record, columns, shares).  A vertex with one item is finished at
// once; otherwise the item's sum is added into hacc[h] (two 64-bit atomic
// adds, the low word's carry taken from its returned old value) and the warp
// that completes the vertex's last item finishes it and resets the
// accumulators for the next round.
// GL lanes (8, 16 or 32) work on one item; a warp's 32 / GL groups take
// consecutive items.  The loop over items runs the same number of times in
// every lane of the warp (a group past the end works on nothing), so the
// group-wide shuffles always find all their lanes.
template <int BATCH, int GL, typename SH>
__device__ inline void pull_heavy_fx_body(int64_t bid, int64_t nblk,
                                          const int64_t* __restrict__ off,
                                          const int32_t* __restrict__ col,
                                          const PullItem* __restrict__ items, int64_t nitems,
                                          const SH* __restrict__ shx,
                                          const int32_t* __restrict__ range, int g, Table D,
                                          double c, int fmode, uint32_t* __restrict__ qbits,
                                          Fx* __restrict__ hacc, int32_t* __restrict__ hcnt,
                                          int32_t* __restrict__ htouch, Counters* C) {
  constexpr int kGroups = 32 / GL;
  const int L = round_scale(range, g);
  int64_t nins = 0;  // vertices that became keys here
  const int lane = threadIdx.x & 31, gl = lane % GL, gid = lane / GL;
  const int64_t warp0 = (bid * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (nblk * blockDim.x) >> 5;
  for (int64_t base = warp0 * kGroups; base < nitems; base += nwarps * kGroups) {
    const int64_t it = base + gid;
    const bool valid = it < nitems;
    PullItem I;
    if (valid) {
      I = items[it];
    } else {
      I.beg = 0;
      I.w = 0;
      I.h = 0;
      I.len = 0;
      I.nparts = 1;
    }
    const int32_t w = I.w;
    // the vertex's state, needed only by the group's first lane at the end
    uint32_t bword = 0;
    double cur = 0.0;
    int64_t d = 0;
    if (gl == 0 && valid) {
      bword = D.bits[w >> 5];
      cur = D.dval[w];
      d = off[w + 1] - off[w];
    }
    Fx part = {0, 0};
    uint64_t flag = 0;
    for (int k0 = 0; k0 < I.len; k0 += GL * BATCH) {
      int32_t u[BATCH];
#pragma unroll
      for (int j = 0; j < BATCH; j++) {
        const int k = k0 + GL * j + gl;
        u[j] = k < I.len ? col[I.beg + k] : -1;
      }
      SH raw[BATCH];
#pragma unroll
      for (int j = 0; j < BATCH; j++) raw[j] = u[j] >= 0 ? shx[u[j]] : no_share<SH>();
#pragma unroll
      for (int j = 0; j < BATCH; j++) {
        const Fx x = to_fx(raw[j], L);
        flag |= x.hi;
        fx_add(part, x);
      }
    }
    uint32_t mem = (flag & kFxFlag) ? 1u : 0u;
    for (int o = GL / 2; o > 0; o >>= 1) {  // within the group
      Fx t;
      t.lo = __shfl_xor_sync(0xffffffffu, part.lo, o);
      t.hi = __shfl_xor_sync(0xffffffffu, part.hi, o);
      fx_add(part, t);
      mem |= __shfl_xor_sync(0xffffffffu, mem, o);
    }
    const bool any = mem != 0;
    if (gl != 0 || !valid) continue;
    const bool present = (bword >> (w & 31)) & 1u;
    if (I.nparts == 1) {
      if (present || any)
        nins += pull_finish(D, w, d, (present ? cur : 0.0) + fx_to_double(part, L), true,
                            present, c, fmode, qbits);
      continue;
    }
    const int32_t h = I.h;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(&hacc[h]);
    if (part.lo | part.hi) {
      const unsigned long long old = atomicAdd(&acc[0], (unsigned long long)part.lo);
      const unsigned long long carry = old + part.lo < old ? 1ull : 0ull;
      atomicAdd(&acc[1], (unsigned long long)part.hi + carry);
    }
    if (any) atomicOr(&htouch[h], 1);
    __threadfence();
    if (atomicAdd(&hcnt[h], 1) == I.nparts - 1) {
      __threadfence();
      Fx total;
      total.lo = atomicAdd(&acc[0], 0ull);
      total.hi = atomicAdd(&acc[1], 0ull);
      if (present || atomicOr(&htouch[h], 0) != 0)
        nins += pull_finish(D, w, d, (present ? cur : 0.0) + fx_to_double(total, L), true,
                            present, c, fmode, qbits);
      acc[0] = 0;
      acc[1] = 0;
      hcnt[h] = 0;
      htouch[h] = 0;
    }
  }
  flush_count(nins, &C->inserted);
}

template <int BATCH, int GL, typename SH>
__global__ void __launch_bounds__(kBlock)
    pull_heavy_fx_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                         const PullItem* __restrict__ items, int64_t nitems,
                         const SH* __restrict__ shx, const int32_t* __restrict__ range, int g,
                         Table D, double c, int fmode, uint32_t* __restrict__ qbits,
                         Fx* __restrict__ hacc, int32_t* __restrict__ hcnt,
                         int32_t* __restrict__ htouch, Counters* C) {
  pull_heavy_fx_body<BATCH, GL, SH>(blockIdx.x, gridDim.x, off, col, items, nitems, shx, range, g,
                                    D, c, fmode, qbits, hacc, hcnt, htouch, C);
}

template <typename SH>
__global__ void pull_light_fx_kernel(const LightItem* __restrict__ items, int64_t nl,
                                     const int32_t* __restrict__ col,
                                     const SH* __restrict__ shx,
                                     const int32_t* __restrict__ range, int g, Table D, double c,
                                     int fmode, uint32_t* __restrict__ qbits, Counters* C) {
  pull_light_fx_body<SH>(blockIdx.x, gridDim.x, items, nl, col, shx, range, g, D, c, fmode,
                         qbits, C);
}

// ---------------------------------------------------------------------------
// edgeMap, deterministic mode.
// ---------------------------------------------------------------------------
// Emits record e of source i: with a self record, local index 0 is
// (v, +0.0) (adding +0.0 to a non-negative value changes nothing) and local
// index q >= 1 is edge q-1; without, local index q is edge q.
__global__ void __launch_bounds__(kBlock)
    emit_records_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ fv,
                        const double* __restrict__ share, const int64_t* __restrict__ epos,
                        const int64_t* __restrict__ foff, int64_t nf, int64_t R, int self_rec,
                        uint32_t* __restrict__ rkey, double* __restrict__ rval) {
  __shared__ int64_t s_epos[kEdgeTile + 1];
  __shared__ int64_t s_off[kEdgeTile];
  __shared__ double s_share[kEdgeTile];
  __shared__ int32_t s_v[kEdgeTile];
  __shared__ int64_t s_i0, s_i1;
  const int64_t ntiles = (R + kEdgeTile - 1) / kEdgeTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kEdgeTile;
    const int64_t e1 = min(R, e0 + kEdgeTile);
    const int cntsrc = stage_sources(epos, nf, R, e0, e1, &s_i0, &s_i1, s_epos);
    const int64_t i0 = s_i0;
    for (int j = threadIdx.x; j < cntsrc; j += kBlock) {
      s_off[j] = foff[i0 + j];
      s_share[j] = share[i0 + j];
      s_v[j] = fv[i0 + j];
    }
    __syncthreads();
    for (int k = 0; k < kEdgeItems; k++) {
      const int64_t e = e0 + k * kBlock + threadIdx.x;
      int64_t q = 0;
      const int j = e < e1 ? find_source(s_epos, cntsrc, e, &q) : -1;
      if (j >= 0) {
        if (self_rec && q == 0) {
          rkey[e] = (uint32_t)s_v[j];
          rval[e] = 0.0;
        } else {
          if (self_rec) q -= 1;
          rkey[e] = (uint32_t)col[s_off[j] + q];
          rval[e] = s_share[j];
        }
      }
    }
    __syncthreads();
  }
}

__global__ void head_flags_kernel(const uint32_t* __restrict__ rkey, int64_t R,
                                  int64_t* __restrict__ flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R;
       e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = (e == 0 || rkey[e] != rkey[e - 1]) ? 1 : 0;
}

// flag[] was scanned (exclusive) into segid[]; heads record their start.
__global__ void head_starts_kernel(const uint32_t* __restrict__ rkey, int64_t R,
                                   const int64_t* __restrict__ segid,
                                   int64_t* __restrict__ segstart) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R;
       e += (int64_t)gridDim.x * blockDim.x)
    if (e == 0 || rkey[e] != rkey[e - 1]) segstart[segid[e]] = e;
}

// One thread per destination run: left fold from the current table value,
// in ascending source order (the order of the run after the stable sort).
// Runs longer than kFoldLong records (a hub destination) are not folded by
// one thread: fold_kernel resolves their slot and lists them, and
// fold_long_kernel folds each with a warp, 256 records at a time, with the
// binade scan of fold_batch (same bits as the sequential fold).
constexpr int64_t kFoldLong = 64;

__global__ void fold_kernel(const uint32_t* __restrict__ rkey, const double* __restrict__ rval,
                            int64_t R, const int64_t* __restrict__ segstart, int64_t nseg,
                            Table D, const int32_t* __restrict__ deg, double c, int fmode,
                            int64_t* __restrict__ qflag, int32_t* __restrict__ segv,
                            int32_t* __restrict__ segslot, int64_t* __restrict__ longs,
                            int32_t* __restrict__ nlong, Counters* C) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nseg;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = base + threadIdx.x;
    int ins = 0;
    bool is_long = false;
    if (sg < nseg) {
      const int64_t b = segstart[sg];
      const int64_t e = sg + 1 < nseg ? segstart[sg + 1] : R;
      const int32_t w = (int32_t)rkey[b];
      const int64_t slot = tb_find_or_insert(D, w, &ins, &C->err);
      int64_t q = 0;
      if (slot >= 0 && e - b > kFoldLong) {
        is_long = true;  // folded by fold_long_kernel, which also sets qflag
      } else if (slot >= 0) {
        double acc = *tb_val(D, slot);
        for (int64_t k = b; k < e; k++) acc = acc + rval[k];
        *tb_val(D, slot) = acc;
        if (fmode == kFmThreshold) q = acc >= c * (double)deg[w] ? 1 : 0;
        else if (fmode == kFmInserted) q = 1;
      }
      if (!is_long) qflag[sg] = q;
      segv[sg] = w;
      segslot[sg] = (int32_t)slot;
    }
    // warp-aggregated append of the long runs
    const unsigned active = __activemask();
    const unsigned m = __ballot_sync(active, is_long);
    if (m) {
      const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
      int at = 0;
      if (lane == leader) at = atomicAdd(nlong, __popc(m));
      at = __shfl_sync(active, at, leader);
      if (is_long) longs[at + __popc(m & ((1u << lane) - 1))] = sg;
    }
    count_inserted(ins, &C->inserted);
  }
}

__global__ void __launch_bounds__(kBlock)
    fold_long_kernel(const double* __restrict__ rval, int64_t R,
                     const int64_t* __restrict__ segstart, int64_t nseg,
                     const int64_t* __restrict__ longs, const int32_t* __restrict__ nlong,
                     Table D, const int32_t* __restrict__ deg, double c, int fmode,
                     int64_t* __restrict__ qflag, const int32_t* __restrict__ segv,
                     const int32_t* __restrict__ segslot) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nl = *nlong;
  for (int64_t i = warp0; i < nl; i += nwarps) {
    const int64_t sg = longs[i];
    const int64_t b = segstart[sg];
    const int64_t e = sg + 1 < nseg ? segstart[sg + 1] : R;
    const int32_t w = segv[sg];
    const int64_t slot = segslot[sg];
    double acc = *tb_val(D, slot);  // the same in every lane
    for (int64_t k0 = b; k0 < e; k0 += 256) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int64_t k = k0 + 8 * lane + j;
        v[j] = k < e ? rval[k] : 0.0;  // +0.0 past the run adds nothing
      }
      acc = fold_batch(acc, v, lane);
    }
    if (lane == 0) {
      *tb_val(D, slot) = acc;
      int64_t q = 0;
      if (fmode == kFmThreshold) q = acc >= c * (double)deg[w] ? 1 : 0;
      else if (fmode == kFmInserted) q = 1;
      qflag[sg] = q;
    }
  }
}

// Order-preserving compaction of the qualifying runs into the next frontier.
__global__ void compact_frontier_kernel(const int64_t* __restrict__ qflag,
                                        const int64_t* __restrict__ qpos, int64_t nseg,
                                        const int32_t* __restrict__ segv,
                                        const int32_t* __restrict__ segslot,
                                        const int32_t* __restrict__ deg, int32_t* nfv,
                                        int32_t* nfs, int32_t ncap, Counters* C) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nseg;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = base + threadIdx.x;
    int64_t d = 0;
    if (sg < nseg && qflag[sg]) {
      const int64_t pos = qpos[sg];
      if (pos < ncap) {
        nfv[pos] = segv[sg];
        nfs[pos] = segslot[sg];
      } else {
        atomicOr(&C->err, kErrFrontierOverflow);
      }
      d = deg[segv[sg]];
    }
    // integer sum of degrees: order-independent
    const unsigned active = __activemask();
    unsigned long long lo = __reduce_add_sync(active, (unsigned)(d & 0xFFFF));
    unsigned long long hi = __reduce_add_sync(active, (unsigned)(d >> 16));
    if ((threadIdx.x & 31) == __ffs(active) - 1 && (lo | hi))
      atomicAdd((unsigned long long*)&C->next_edges, lo + (hi << 16));
  }
}

__global__ void set_counter_size_kernel(Counters* C, const int64_t* total) {
  C->next_size = (int32_t)*total;
}

__global__ void init_seed_kernel(Table T, int32_t x, double r0, int32_t* fv, int32_t* fs,
                                 Counters* C) {
  int ins = 0;
  int64_t s = tb_find_or_insert(T, x, &ins, &C->err);
  if (s >= 0) *tb_val(T, s) = r0;
  fv[0] = x;
  fs[0] = (int32_t)s;
}

// Seed set: seeds (ascending, distinct) with their initial residuals.
__global__ void init_seeds_kernel(Table T, const int32_t* __restrict__ x,
                                  const double* __restrict__ r0, int64_t k, int32_t* fv,
                                  int32_t* fs, Counters* C) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    int ins = 0;
    const int64_t s = tb_find_or_insert(T, x[i], &ins, &C->err);
    if (s >= 0) *tb_val(T, s) = r0[i];
    fv[i] = x[i];
    fs[i] = (int32_t)s;
  }
}

// beta-fraction rounds: order the frontier by r/d descending, ties by
// ascending id (sort by id, then stably by the key 0x7FF...F - bits(r/d)).
__global__ void sel_ids_kernel(const int32_t* __restrict__ fv, int64_t nf,
                               uint32_t* __restrict__ key, int32_t* __restrict__ pos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    key[i] = (uint32_t)fv[i];
    pos[i] = (int32_t)i;
  }
}

__global__ void sel_keys_kernel(const int32_t* __restrict__ fv, const int32_t* __restrict__ fs,
                                const int32_t* __restrict__ pos, int64_t nf, Table T,
                                const int32_t* __restrict__ deg, uint64_t* __restrict__ key) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = pos[i];
    const double r = fs[j] >= 0 ? *tb_val(T, fs[j]) : 0.0;
    const double kv = r / (double)deg[fv[j]];
    key[i] = 0x7FFFFFFFFFFFFFFFull - ((uint64_t)__double_as_longlong(kv) & 0x7FFFFFFFFFFFFFFFull);
  }
}

// The first m in the order push (written with their ids as keys, to be
// sorted ascending), the rest stay (rv/rs).
__global__ void sel_split_kernel(const int32_t* __restrict__ fv, const int32_t* __restrict__ fs,
                                 const int32_t* __restrict__ pos, int64_t nf, int64_t m,
                                 uint32_t* __restrict__ sv, int32_t* __restrict__ ss,
                                 int32_t* __restrict__ rv, int32_t* __restrict__ rs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = pos[i];
    if (i < m) {
      sv[i] = (uint32_t)fv[j];
      ss[i] = fs[j];
    } else {
      rv[i - m] = fv[j];
      rs[i - m] = fs[j];
    }
  }
}

__global__ void copy_frontier_kernel(const uint32_t* __restrict__ sv,
                                     const int32_t* __restrict__ ss, int64_t m,
                                     const int32_t* __restrict__ deg, int32_t* fv, int32_t* fs,
                                     unsigned long long* edges) {
  unsigned long long e = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    fv[i] = (int32_t)sv[i];
    fs[i] = ss[i];
    e += (unsigned long long)deg[sv[i]];
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e) atomicAdd(edges, e);
}

// Next frontier = the round's qualifying vertices together with the
// candidates that did not push and still have r >= eps d (a seed is on the
// first frontier whatever its residual; afterwards only the threshold
// counts): concatenated, sorted by id, duplicates dropped (a waiting
// candidate that was pushed to may be in both).  A dropped one gets the key
// 0xFFFFFFFF (no vertex id), which sorts last.
__global__ void cat_frontier_kernel(const int32_t* __restrict__ av, const int32_t* __restrict__ as,
                                    int64_t na, const int32_t* __restrict__ bv,
                                    const int32_t* __restrict__ bs, int64_t nb, Table T,
                                    const int32_t* __restrict__ deg, double eps,
                                    uint32_t* __restrict__ kv, int32_t* __restrict__ ks) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < na) {
      kv[i] = (uint32_t)av[i];
      ks[i] = as[i];
    } else {
      const int32_t v = bv[i - na], s = bs[i - na];
      const bool keep = s >= 0 && *tb_val(T, s) >= eps * (double)deg[v];
      kv[i] = keep ? (uint32_t)v : 0xFFFFFFFFu;
      ks[i] = s;
    }
  }
}

__global__ void uniq_flags_kernel(const uint32_t* __restrict__ kv, int64_t n,
                                  int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (kv[i] != 0xFFFFFFFFu && (i == 0 || kv[i] != kv[i - 1])) ? 1 : 0;
}

__global__ void uniq_write_kernel(const uint32_t* __restrict__ kv, const int32_t* __restrict__ ks,
                                  const int64_t* __restrict__ flag, const int64_t* __restrict__ pos,
                                  int64_t n, const int32_t* __restrict__ deg, int32_t* fv,
                                  int32_t* fs, unsigned long long* edges) {
  unsigned long long e = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    fv[pos[i]] = (int32_t)kv[i];
    fs[pos[i]] = ks[i];
    e += (unsigned long long)deg[kv[i]];
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e) atomicAdd(edges, e);
}

}  // namespace

template <typename SH>
using HeavyKernel = void (*)(const int64_t*, const int32_t*, const PullItem*, int64_t, const SH*,
                             const int32_t*, int, Table, double, int, uint32_t*, Fx*, int32_t*,
                             int32_t*, Counters*);

// The heavy-vertex gather compiled for a (batch depth, lanes per item) shape.
template <typename SH>
HeavyKernel<SH> heavy_kernel(int batch, int group) {
  if (group == 8)
    return batch == 16 ? pull_heavy_fx_kernel<16, 8, SH> : pull_heavy_fx_kernel<8, 8, SH>;
  if (group == 16)
    return batch == 16 ? pull_heavy_fx_kernel<16, 16, SH> : pull_heavy_fx_kernel<8, 16, SH>;
  return batch == 16 ? pull_heavy_fx_kernel<16, 32, SH>
         : batch == 4 ? pull_heavy_fx_kernel<4, 32, SH>
                      : pull_heavy_fx_kernel<kPullBatch, 32, SH>;
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
namespace {

struct Frontier {
  DBuf<int32_t> v, s;
  int64_t size = 0, edges = 0;
  void release(lgc_ctx* ctx) {
    v.release(ctx);
    s.release(ctx);
  }
};

struct PushWork {
  lgc_ctx* ctx;
  lgc_graph* g;
  Frontier F, G;
  DBuf<double> share;
  DBuf<int64_t> cnt, epos, foff;
  DBuf<uint32_t> rk, rk2;
  DBuf<double> rv, rv2;
  DBuf<int64_t> flag, segid, segstart, qflag, qpos;
  DBuf<int32_t> segv, segslot;
  DBuf<int64_t> longs;  // runs folded by a warp
  DBuf<int32_t> nlong;
  DBuf<int64_t> total;  // one device int64
  // pull rounds: per-vertex frontier share (membership encoded), qualify bitmap
  DBuf<double> psh;
  DBuf<uint32_t> pq;
  DBuf<Fx> pshx;                   // atomic mode: per-vertex fixed-point shares
  DBuf<int32_t> prange;            // atomic mode: exponent range of the shares
  DBuf<Fx> phacc;                  // per heavy vertex: partial sums of its items
  DBuf<int32_t> phcnt, phtouch;    // per heavy vertex: items done, any frontier neighbour
  // deterministic pull of big vertices: per segment sum, member flag,
  // predicted binade, composed step
  DBuf<double> dsum;
  DBuf<int32_t> dany, dpred;
  DBuf<FoldStep> dstep;
  bool pull_ready = false;
  // beta-fraction rounds: the candidates that did not push, sort scratch
  Frontier U;
  DBuf<uint64_t> selk, selk2;
  DBuf<uint32_t> selv, selv2;
  DBuf<int32_t> seli, seli2;
  DBuf<unsigned long long> selcnt;
  // device-driven rounds: two frontier buffers, block sums, counters, state
  Frontier X[2];
  DBuf<int64_t> xbsum;
  DBuf<Counters> xcn;
  DBuf<RoundsState> xst;
  lgc_stats st{};
  explicit PushWork(lgc_ctx* c, lgc_graph* gr) : ctx(c), g(gr) {}
  ~PushWork() {
    F.release(ctx);
    G.release(ctx);
    X[0].release(ctx);
    X[1].release(ctx);
    U.release(ctx);
    selk.release(ctx);
    selk2.release(ctx);
    selv.release(ctx);
    selv2.release(ctx);
    seli.release(ctx);
    seli2.release(ctx);
    selcnt.release(ctx);
    dsum.release(ctx);
    dany.release(ctx);
    dpred.release(ctx);
    dstep.release(ctx);
    xbsum.release(ctx);
    xcn.release(ctx);
    xst.release(ctx);
    share.release(ctx);
    cnt.release(ctx);
    epos.release(ctx);
    foff.release(ctx);
    rk.release(ctx);
    rk2.release(ctx);
    rv.release(ctx);
    rv2.release(ctx);
    flag.release(ctx);
    segid.release(ctx);
    segstart.release(ctx);
    qflag.release(ctx);
    qpos.release(ctx);
    segv.release(ctx);
    segslot.release(ctx);
    longs.release(ctx);
    nlong.release(ctx);
    total.release(ctx);
    psh.release(ctx);
    pshx.release(ctx);
    prange.release(ctx);
    pq.release(ctx);
    phacc.release(ctx);
    phcnt.release(ctx);
    phtouch.release(ctx);
  }

  int reset_counters() {
    LGC_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(Counters), ctx->stream));
    return LGC_OK;
  }
  int read_counters(Counters* out) {
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_counters, ctx->d_counters, sizeof(Counters),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    LGC_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    LGC_TRY(sort_check(ctx));
    *out = *ctx->h_counters;
    if (out->err & kErrTableFull) return LGC_ETABLEFULL;
    if (out->err & kErrFrontierOverflow) return LGC_ETABLEFULL;
    return LGC_OK;
  }
  int reserve_frontier_scratch(int64_t nf) {
    LGC_TRY(share.reserve(ctx, nf));
    LGC_TRY(cnt.reserve(ctx, nf));
    LGC_TRY(epos.reserve(ctx, nf));
    LGC_TRY(foff.reserve(ctx, nf));
    LGC_TRY(total.reserve(ctx, 1));
    return LGC_OK;
  }
  int reserve_next(int64_t cap) {
    LGC_TRY(G.v.reserve(ctx, cap));
    LGC_TRY(G.s.reserve(ctx, cap));
    return LGC_OK;
  }
  void record_trace() {
    if (!ctx->trace) return;
    size_t at = ctx->trace_ids.size();
    ctx->trace_ids.resize(at + F.size);
    if (F.size)
      cudaMemcpyAsync(ctx->trace_ids.data() + at, F.v.ptr, 4 * F.size, cudaMemcpyDeviceToHost,
                      ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    ctx->trace_sizes.push_back(F.size);
  }

  // edgeMap + filter into table D.  Records per source are cnt[] (scanned
  // into epos by the caller's vertexMap step).  Returns the counters.
  int edge_phase(const Table& D, double c, int fmode, bool det, bool self_rec, int64_t nrec,
                 Counters* out, bool bulk = false) {
    cudaStream_t s = ctx->stream;
    const int64_t nf = F.size;
    const int32_t ncap = (int32_t)G.v.cap;
    // algorithmic bytes: 24 per pushed edge (col 4, key 4, value read-modify-write 16),
    // 24 per frontier source staged (epos, off, share), 8 per next-frontier entry
    const double alg_bytes = 24.0 * (double)(nrec - (self_rec && det ? nf : 0)) + 24.0 * nf;
    if (bulk) {
      if (nrec > 0) {
        int64_t tiles = ceil_div(nrec, kEdgeTile);
        int grid = (int)(tiles < (ctx->sms * 16) ? tiles : (ctx->sms * 16));
        // a dense destination's inserted keys: population after - before
        const int64_t words = (g->n + 31) / 32;
        const int pg = std::min(grid_for(words), ctx->sms * 8);
        if (D.dense) {
          bits_pop_kernel<<<pg, kBlock, 0, s>>>(D.bits, words, -1, &ctx->d_counters->inserted);
          LGC_COUNT_LAUNCH(ctx);
        }
        {
          ProfScope ps(ctx, LGC_PROF_EDGEMAP, alg_bytes);
          emap_red_kernel<<<grid, kBlock, 0, s>>>(g->col, share.ptr, epos.ptr, foff.ptr, nf, nrec,
                                                   total.ptr, D, ctx->d_counters);
          LGC_COUNT_LAUNCH(ctx);
        }
        if (D.dense) {
          bits_pop_kernel<<<pg, kBlock, 0, s>>>(D.bits, words, 1, &ctx->d_counters->inserted);
          LGC_COUNT_LAUNCH(ctx);
        }
        LGC_CUDA_TRY(cudaGetLastError());
      }
      if (fmode != kFmNone) {  // the qualifying keys in ascending id, with their degrees
        const int64_t words = (g->n + 31) / 32;
        const int64_t ntiles = ceil_div(words, kCmpTileWords);
        uint32_t epoch;
        unsigned long long *ticket, t0;
        LGC_TRY(lb_begin(ctx, ntiles, &epoch, &ticket, &t0));
        compact_words_kernel<DenseQualWord><<<(unsigned)ntiles, kBlock, 0, s>>>(
            DenseQualWord{D, g->deg, g->n, c, fmode}, words, ntiles, g->deg, G.v.ptr, G.s.ptr,
            ncap, ticket, t0, ctx->sort_status, epoch, ctx->d_sort_err, ctx->d_counters);
        LGC_COUNT_LAUNCH(ctx);
        LGC_CUDA_TRY(cudaGetLastError());
        lb_commit(ctx, ntiles);
      }
      int st = read_counters(out);
      if (ctx->profile && nrec > 0 && !ctx->prof_pending.empty())
        ctx->prof_pending.back().bytes += 8.0 * out->next_size;
      return st;
    }
    if (!det) {
      if (nrec > 0) {
        int64_t tiles = ceil_div(nrec, kEdgeTile);
        int grid = (int)(tiles < (ctx->sms * 16) ? tiles : (ctx->sms * 16));
        ProfScope ps(ctx, LGC_PROF_EDGEMAP, alg_bytes);
        emap_atomic_kernel<<<grid, kBlock, 0, s>>>(g->col, g->deg, share.ptr, epos.ptr, foff.ptr,
                                                    nf, nrec, total.ptr, D, c, fmode, G.v.ptr,
                                                    G.s.ptr, ncap, ctx->d_counters);
        LGC_COUNT_LAUNCH(ctx);
        LGC_CUDA_TRY(cudaGetLastError());
      }
      int st = read_counters(out);
      if (ctx->profile && nrec > 0 && !ctx->prof_pending.empty())
        ctx->prof_pending.back().bytes += 8.0 * out->next_size;
      return st;
    }
    // deterministic: emit, stable sort by destination, fold, compact
    LGC_TRY(rk.reserve(ctx, nrec));
    LGC_TRY(rk2.reserve(ctx, nrec));
    LGC_TRY(rv.reserve(ctx, nrec));
    LGC_TRY(rv2.reserve(ctx, nrec));
    LGC_TRY(flag.reserve(ctx, nrec));
    LGC_TRY(segid.reserve(ctx, nrec));
    if (nrec > 0) {
      int64_t tiles = ceil_div(nrec, kEdgeTile);
      int grid = (int)(tiles < (ctx->sms * 16) ? tiles : (ctx->sms * 16));
      ProfScope ps(ctx, LGC_PROF_DET_EDGE, alg_bytes);
      emit_records_kernel<<<grid, kBlock, 0, s>>>(g->col, F.v.ptr, share.ptr, epos.ptr, foff.ptr,
                                                   nf, nrec, self_rec ? 1 : 0, rk.ptr, rv.ptr);
      LGC_COUNT_LAUNCH(ctx);
      LGC_CUDA_TRY(cudaGetLastError());
      LGC_TRY(radix_sort_u32_f64(ctx, rk.ptr, rv.ptr, rk2.ptr, rv2.ptr, nrec, bits_for(g->n)));
      head_flags_kernel<<<grid_for(nrec), kBlock, 0, s>>>(rk.ptr, nrec, flag.ptr);
      LGC_COUNT_LAUNCH(ctx);
      LGC_TRY(scan_i64(ctx, flag.ptr, segid.ptr, nrec, false, total.ptr));
    }
    int64_t nseg = 0;
    if (nrec > 0) {
      LGC_CUDA_TRY(cudaMemcpyAsync(&ctx->h_counters->aux, total.ptr, 8, cudaMemcpyDeviceToHost, s));
      LGC_CUDA_TRY(cudaStreamSynchronize(s));
      nseg = ctx->h_counters->aux;
    }
    LGC_TRY(segstart.reserve(ctx, nseg));
    LGC_TRY(qflag.reserve(ctx, nseg));
    LGC_TRY(qpos.reserve(ctx, nseg));
    LGC_TRY(segv.reserve(ctx, nseg));
    LGC_TRY(segslot.reserve(ctx, nseg));
    if (nseg > 0) {
      ProfScope ps(ctx, LGC_PROF_DET_EDGE, 0.0);
      head_starts_kernel<<<grid_for(nrec), kBlock, 0, s>>>(rk.ptr, nrec, segid.ptr, segstart.ptr);
      LGC_COUNT_LAUNCH(ctx);
      LGC_TRY(longs.reserve(ctx, nseg));
      LGC_TRY(nlong.reserve(ctx, 1));
      LGC_CUDA_TRY(cudaMemsetAsync(nlong.ptr, 0, 4, s));
      fold_kernel<<<grid_for(nseg), kBlock, 0, s>>>(rk.ptr, rv.ptr, nrec, segstart.ptr, nseg, D,
                                                     g->deg, c, fmode, qflag.ptr, segv.ptr,
                                                     segslot.ptr, longs.ptr, nlong.ptr,
                                                     ctx->d_counters);
      LGC_COUNT_LAUNCH(ctx);
      fold_long_kernel<<<ctx->sms * 4, kBlock, 0, s>>>(rv.ptr, nrec, segstart.ptr, nseg,
                                                        longs.ptr, nlong.ptr, D, g->deg, c, fmode,
                                                        qflag.ptr, segv.ptr, segslot.ptr);
      LGC_COUNT_LAUNCH(ctx);
      LGC_CUDA_TRY(cudaGetLastError());
      if (fmode != kFmNone) {
        LGC_TRY(scan_i64(ctx, qflag.ptr, qpos.ptr, nseg, false, total.ptr));
        compact_frontier_kernel<<<grid_for(nseg), kBlock, 0, s>>>(
            qflag.ptr, qpos.ptr, nseg, segv.ptr, segslot.ptr, g->deg, G.v.ptr, G.s.ptr, ncap,
            ctx->d_counters);
        LGC_COUNT_LAUNCH(ctx);
        set_counter_size_kernel<<<1, 1, 0, s>>>(ctx->d_counters, total.ptr);
        LGC_COUNT_LAUNCH(ctx);
        LGC_CUDA_TRY(cudaGetLastError());
      }
    }
    return read_counters(out);
  }

  // The bytes per gathered share of a pull round: atomic mode gathers 16-byte
  // fixed-point records or 8-byte doubles (the graph's tuned choice);
  // deterministic mode always doubles.
  int pull_share_bytes(bool det) const {
    return det ? 8 : (ctx->pull_share ? ctx->pull_share : g->pull_share);
  }

  // The pull rounds' per-vertex arrays (zeroed at first use; every round
  // leaves them zeroed again).
  int pull_reserve(bool det) {
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n, words = (n + 31) / 32;
    if (!pull_ready) {
      LGC_TRY(pq.reserve(ctx, words));
      pull_ready = true;
    }
    const int sb = pull_share_bytes(det);
    if (sb == 8 && !psh.ptr) {
      LGC_TRY(psh.reserve(ctx, n));
      LGC_CUDA_TRY(cudaMemsetAsync(psh.ptr, 0, 8 * n, s));
    }
    if (!det && sb == 16 && !pshx.ptr) {
      LGC_TRY(pshx.reserve(ctx, n));
      LGC_CUDA_TRY(cudaMemsetAsync(pshx.ptr, 0, sizeof(Fx) * n, s));
    }
    if (!det && !prange.ptr) {
      LGC_TRY(prange.reserve(ctx, 2));
      LGC_TRY(phacc.reserve(ctx, g->nheavy + 1));
      LGC_TRY(phcnt.reserve(ctx, g->nheavy + 1));
      LGC_TRY(phtouch.reserve(ctx, g->nheavy + 1));
      LGC_CUDA_TRY(cudaMemsetAsync(phacc.ptr, 0, sizeof(Fx) * (g->nheavy + 1), s));
      LGC_CUDA_TRY(cudaMemsetAsync(phcnt.ptr, 0, 4 * (g->nheavy + 1), s));
      LGC_CUDA_TRY(cudaMemsetAsync(phtouch.ptr, 0, 4 * (g->nheavy + 1), s));
    }
    return LGC_OK;
  }

  // Pull round into the dense table D.  The frontier's shares (share[], from
  // the vertexMap) are scattered into the per-vertex array -- unless the
  // vertexMap wrote them there itself (scattered: 8-byte shares, with the
  // range in atomic mode) --, every vertex gathers (in adjacency order in
  // deterministic mode, heavy vertices by a tree reduction in atomic mode),
  // the qualifying vertices are compacted in ascending id, and the
  // per-vertex array is cleared again (O(|F|)).
  int pull_phase(const Table& D, double c, int fmode, Counters* out, bool det,
                 bool scattered = false) {
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n, words = (n + 31) / 32, nf = F.size;
    LGC_TRY(pull_reserve(det));
    const int sb = pull_share_bytes(det);
    const int32_t ncap = (int32_t)G.v.cap;
    // sums of at most max_deg terms: max_deg < 2^gb
    int gb = 1;
    while (gb < 62 && (int64_t{1} << gb) <= g->max_deg) gb++;
    if (!scattered && det) {
      pull_scatter_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, F.v.ptr, share.ptr, psh.ptr, 0);
      LGC_COUNT_LAUNCH(ctx);
    } else if (!scattered) {
      LGC_CUDA_TRY(cudaMemsetAsync(prange.ptr, 0, 8, s));
      const int64_t rb = ceil_div(nf, kBlock);
      const int rg = (int)std::max<int64_t>(1, std::min<int64_t>(rb, ctx->sms * 4));
      share_range_kernel<<<rg, kBlock, 0, s>>>(nf, share.ptr, prange.ptr);
      LGC_COUNT_LAUNCH(ctx);
      if (sb == 8) {
        pull_scatter_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, F.v.ptr, share.ptr, psh.ptr, 0);
      } else {
        pull_scatter_fx_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, F.v.ptr, share.ptr, pshx.ptr,
                                                                prange.ptr, gb, 0);
      }
      LGC_COUNT_LAUNCH(ctx);
    }
    {
      ProfScope ps(ctx, det ? LGC_PROF_DET_EDGE : LGC_PROF_PULL,
                   24.0 * (double)F.edges + 24.0 * nf);
      if (det) {
        // every gather ORs its qualifying vertices into the cleared bitmap
        LGC_CUDA_TRY(cudaMemsetAsync(pq.ptr, 0, 4 * words, s));
        if (g->nlight_det > 0) {
          const int lgl =
              (int)std::min<int64_t>(ceil_div(g->nlight_det, kBlock), (ctx->sms * 32));
          pull_light_kernel<<<lgl, kBlock, 0, s>>>(g->light_det, g->nlight_det, g->col, psh.ptr,
                                                   D, c, fmode, pq.ptr, ctx->d_counters);
          LGC_COUNT_LAUNCH(ctx);
        }
        if (g->ndet_mid > 0) {
          const int mg = (int)std::min<int64_t>(ceil_div(g->ndet_mid, kBlock), (ctx->sms * 32));
          pull_mid_det_kernel<<<mg, kBlock, 0, s>>>(g->off, g->col, g->det_mid, g->ndet_mid,
                                                    psh.ptr, D, c, fmode, pq.ptr,
                                                    ctx->d_counters);
          LGC_COUNT_LAUNCH(ctx);
        }
        if (g->nbig > 0) {  // lists longer than kDetBig, folded segment-parallel
          LGC_TRY(dsum.reserve(ctx, g->nsegs));
          LGC_TRY(dany.reserve(ctx, g->nsegs));
          LGC_TRY(dpred.reserve(ctx, g->nsegs));
          LGC_TRY(dstep.reserve(ctx, g->nsegs));
          const int sg = (int)std::min<int64_t>(ceil_div(g->nsegs, kBlock / 32), (ctx->sms * 16));
          det_seg_sum_kernel<<<sg, kBlock, 0, s>>>(g->col, g->segs, g->nsegs, psh.ptr, dsum.ptr,
                                                   dany.ptr);
          LGC_COUNT_LAUNCH(ctx);
          det_seg_predict_kernel<<<grid_for(g->nbig), kBlock, 0, s>>>(
              g->big_w, g->big_seg0, g->nbig, D, dsum.ptr, dpred.ptr);
          LGC_COUNT_LAUNCH(ctx);
          det_seg_step_kernel<<<sg, kBlock, 0, s>>>(g->col, g->segs, g->nsegs, psh.ptr, dpred.ptr,
                                                    dstep.ptr);
          LGC_COUNT_LAUNCH(ctx);
          const int vg = (int)std::min<int64_t>(ceil_div(g->nbig, kBlock / 32), (ctx->sms * 16));
          det_seg_verify_kernel<<<vg, kBlock, 0, s>>>(g->off, g->col, g->segs, g->big_w,
                                                      g->big_seg0, g->nbig, psh.ptr, dpred.ptr,
                                                      dstep.ptr, dany.ptr, D, c, fmode, pq.ptr,
                                                      ctx->d_counters);
          LGC_COUNT_LAUNCH(ctx);
        }
      } else {
        // light vertices (writing every bitmap word), then the heavy items
        // (ORing their vertices in); the two in one grid measured slower
        auto gather = [&](auto* shv) {
          using SH = std::remove_const_t<std::remove_pointer_t<decltype(shv)>>;
          if (g->nlight > 0) {
            const int lgl = (int)std::min<int64_t>(ceil_div(g->nlight, kBlock), (ctx->sms * 32));
            pull_light_fx_kernel<SH><<<lgl, kBlock, 0, s>>>(g->light, g->nlight, g->col, shv,
                                                             prange.ptr, gb, D, c, fmode, pq.ptr,
                                                             ctx->d_counters);
            LGC_COUNT_LAUNCH(ctx);
          }
          if (g->nitems > 0) {
            const int gw = ctx->pull_group ? ctx->pull_group : g->pull_group;
            const int64_t hb = ceil_div(g->nitems, (kBlock / 32) * (32 / gw));
            const int hg = (int)(hb < (ctx->sms * 16) ? hb : (ctx->sms * 16));
            const int batch = ctx->pull_batch ? ctx->pull_batch : g->pull_batch;
            HeavyKernel<SH> heavy = heavy_kernel<SH>(batch, gw);
            heavy<<<hg, kBlock, 0, s>>>(g->off, g->col, g->items, g->nitems, shv, prange.ptr, gb,
                                        D, c, fmode, pq.ptr, phacc.ptr, phcnt.ptr, phtouch.ptr,
                                        ctx->d_counters);
            LGC_COUNT_LAUNCH(ctx);
          }
        };
        // both gathers OR their qualifying vertices into the cleared bitmap
        LGC_CUDA_TRY(cudaMemsetAsync(pq.ptr, 0, 4 * words, s));
        if (sb == 8) gather(psh.ptr);
        else gather(pshx.ptr);
      }
    }
    if (fmode != kFmNone)  // the qualifying vertices, in ascending id, with their degrees
      LGC_TRY(bits_compact(ctx, pq.ptr, words, g->deg, G.v.ptr, G.s.ptr, ncap, ctx->d_counters));
    if (sb == 8) {
      pull_scatter_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, F.v.ptr, share.ptr, psh.ptr, 1);
    } else {
      pull_scatter_fx_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, F.v.ptr, share.ptr, pshx.ptr,
                                                              prange.ptr, gb, 1);
    }
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    return read_counters(out);
  }

  // Consecutive small rounds of atomic PR-Nibble on the device (see
  // rounds_prnibble_kernel).  Runs at least one round when small_round()
  // holds for the current one; afterwards F, T's key count and st describe
  // the state reached, and the host continues from there.
  static constexpr int64_t kRoundsEmax = int64_t{1} << 20;
  static constexpr int64_t kRoundsPerLaunch = 1024;
  int64_t rounds_emax() const { return std::min<int64_t>(kRoundsEmax, g->nnz / 16); }
  int64_t rounds_fcap() const { return std::min<int64_t>(g->n, 2 * kRoundsEmax); }
  static int64_t key_limit(const Table& T) { return T.dense ? INT64_MAX : T.cap / 2; }
  bool small_round_nibble() const {
    return ctx->device_rounds && !ctx->trace && F.size > 0 && F.edges <= rounds_emax() &&
           F.size + F.edges <= rounds_fcap();
  }
  bool small_round(const Table& T, int64_t count) const {
    return ctx->device_rounds && !ctx->trace && F.size > 0 && F.edges <= rounds_emax() &&
           F.size + F.edges <= rounds_fcap() && count + F.edges <= key_limit(T);
  }
  int device_rounds_prnibble(Table& T, int64_t* count, double alpha, double cs, double cn,
                             double eps, int rule, int64_t rounds_left) {
    cudaStream_t s = ctx->stream;
    static int blocks_per_sm = -1;  // the same for every device of this build
    if (blocks_per_sm < 0) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rounds_prnibble_kernel, kBlock, 0) !=
          cudaSuccess)
        nb = 0;
      blocks_per_sm = nb;
    }
    int sms = 0;
    LGC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    // one block per SM: the rounds are small, and fewer blocks wait at each
    // grid barrier (two per SM measured 0.3% slower on the bench step)
    const int G = sms * std::min(blocks_per_sm, 1);
    if (G < 1) {  // no co-resident grid possible: rounds stay on the host
      ctx->device_rounds = false;
      return LGC_OK;
    }
    const int64_t fcap = rounds_fcap();
    for (int k = 0; k < 2; k++) {
      LGC_TRY(X[k].v.reserve(ctx, fcap));
      LGC_TRY(X[k].s.reserve(ctx, fcap));
    }
    LGC_TRY(reserve_frontier_scratch(fcap));
    LGC_TRY(xbsum.reserve(ctx, G));
    LGC_TRY(xcn.reserve(ctx, 2));
    LGC_TRY(xst.reserve(ctx, 1));
    LGC_TRY(total.reserve(ctx, 8));
    LGC_CUDA_TRY(cudaMemcpyAsync(X[0].v.ptr, F.v.ptr, 4 * F.size, cudaMemcpyDeviceToDevice, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(X[0].s.ptr, F.s.ptr, 4 * F.size, cudaMemcpyDeviceToDevice, s));
    rounds_init_kernel<<<1, 1, 0, s>>>(xcn.ptr, xst.ptr, F.size, F.edges, *count);
    LGC_COUNT_LAUNCH(ctx);
    int32_t fc = (int32_t)fcap;
    // at most kRoundsPerLaunch rounds per launch: the host regains control
    // at least that often
    int64_t mr = std::min<int64_t>(rounds_left, kRoundsPerLaunch), em = rounds_emax(),
            kl = key_limit(T);
    void* args[] = {&T, &g->off, &g->col, &g->deg, &alpha, &cs, &cn, &eps, &rule,
                    &X[0].v.ptr, &X[0].s.ptr, &X[1].v.ptr, &X[1].s.ptr, &fc, &share.ptr, &cnt.ptr,
                    &epos.ptr, &foff.ptr, &xbsum.ptr, &xcn.ptr, &xst.ptr, &mr, &em, &kl};
    {
      ProfScope ps(ctx, LGC_PROF_EDGEMAP, 0.0);
      LGC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)rounds_prnibble_kernel, G, kBlock,
                                               args, 0, s));
      LGC_COUNT_LAUNCH(ctx);
    }
    rounds_pack_kernel<<<1, 1, 0, s>>>(xcn.ptr, xst.ptr, total.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, total.ptr, 64, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t* o = ctx->h_scratch;
    const int64_t cur = o[1], nf = o[2], E = o[3], rounds = o[5];
    if (ctx->profile && !ctx->prof_pending.empty())
      ctx->prof_pending.back().bytes += 24.0 * (double)o[7] + 88.0 * (double)o[6];
    if ((o[0] >> 8) != 0) return LGC_ETABLEFULL;
    if (rounds < 1) return LGC_ECUDA;  // the host checked that the first round is small
    LGC_TRY(F.v.reserve(ctx, std::max<int64_t>(nf, 1024)));
    LGC_TRY(F.s.reserve(ctx, std::max<int64_t>(nf, 1024)));
    LGC_CUDA_TRY(cudaMemcpyAsync(F.v.ptr, X[cur].v.ptr, 4 * nf, cudaMemcpyDeviceToDevice, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(F.s.ptr, X[cur].s.ptr, 4 * nf, cudaMemcpyDeviceToDevice, s));
    F.size = nf;
    F.edges = E;
    *count = o[4];
    st.rounds += rounds;
    st.pushes += o[6];
    st.pushed_edges += o[7];
    return LGC_OK;
  }

  // Nibble's rounds on the device (rounds_nibble_kernel) from the host's p
  // table P and frontier F, at most rounds_left of them.  Afterwards P holds
  // p (a table of the kernel's, or the same one), Pn is a spare, F and the
  // counters are the host's again, *done counts the rounds run and *over is
  // set when a round's frontier came out empty (the run is over).
  int device_rounds_nibble(Table& P, Table& Pn, int64_t* count, double eps, int fmode,
                           int64_t rounds_left, int64_t* done, bool* over) {
    cudaStream_t s = ctx->stream;
    *done = 0;
    *over = false;
    static int blocks_per_sm = -1;  // the same for every device of this build
    if (blocks_per_sm < 0) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rounds_nibble_kernel, kBlock, 0) !=
          cudaSuccess)
        nb = 0;
      blocks_per_sm = nb;
    }
    int sms = 0;
    LGC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    // one block per SM: the rounds are small, and fewer blocks wait at each
    // grid barrier (two per SM measured 0.3% slower on the bench step)
    const int G = sms * std::min(blocks_per_sm, 1);
    if (G < 1) {  // no co-resident grid possible: rounds stay on the host
      ctx->device_rounds = false;
      return LGC_OK;
    }
    const int64_t fcap = rounds_fcap();
    // p' tables with room for 8 times this round's keys (a round that
    // would not fit returns to the host, which comes back with bigger ones)
    const int64_t keys8 = std::min<int64_t>(g->n, 8 * (F.size + F.edges));
    const int64_t cap = pow2_at_least(2 * std::max<int64_t>(1024, keys8));
    Table A, B;
    int st_ = table_create(ctx, &A, cap, false);
    if (st_ == LGC_OK) st_ = table_create(ctx, &B, cap, false);
    if (st_ != LGC_OK) {
      table_destroy(ctx, &A);
      table_destroy(ctx, &B);
      return st_;
    }
    auto fail = [&](int code) {
      table_destroy(ctx, &A);
      table_destroy(ctx, &B);
      return code;
    };
    for (int k = 0; k < 2; k++) {
      if (X[k].v.reserve(ctx, fcap) || X[k].s.reserve(ctx, fcap)) return fail(LGC_ENOMEM);
    }
    if (reserve_frontier_scratch(fcap) || xbsum.reserve(ctx, G) || xcn.reserve(ctx, 2) ||
        xst.reserve(ctx, 1) || total.reserve(ctx, 8))
      return fail(LGC_ENOMEM);
    if (cudaMemcpyAsync(X[0].v.ptr, F.v.ptr, 4 * F.size, cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(X[0].s.ptr, F.s.ptr, 4 * F.size, cudaMemcpyDeviceToDevice, s))
      return fail(LGC_ECUDA);
    rounds_init_kernel<<<1, 1, 0, s>>>(xcn.ptr, xst.ptr, F.size, F.edges, *count);
    LGC_COUNT_LAUNCH(ctx);
    int32_t fc = (int32_t)fcap;
    int64_t mr = std::min<int64_t>(rounds_left, kRoundsPerLaunch), em = rounds_emax(),
            kl = cap / 2;
    void* args[] = {&P, &A, &B, &g->off, &g->col, &g->deg, &eps, &fmode, &X[0].v.ptr,
                    &X[0].s.ptr, &X[1].v.ptr, &X[1].s.ptr, &fc, &share.ptr, &cnt.ptr, &epos.ptr,
                    &foff.ptr, &xbsum.ptr, &xcn.ptr, &xst.ptr, &mr, &em, &kl};
    {
      ProfScope ps(ctx, LGC_PROF_EDGEMAP, 0.0);
      if (cudaLaunchCooperativeKernel((const void*)rounds_nibble_kernel, G, kBlock, args, 0, s))
        return fail(LGC_ECUDA);
      LGC_COUNT_LAUNCH(ctx);
    }
    rounds_pack_kernel<<<1, 1, 0, s>>>(xcn.ptr, xst.ptr, total.ptr);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaMemcpyAsync(ctx->h_scratch, total.ptr, 64, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return fail(LGC_ECUDA);
    const int64_t* o = ctx->h_scratch;
    const int64_t stop = o[0] & 0xff, err = (o[0] >> 8) & 0xff, ptab = (o[0] >> 16) & 0xff;
    const int64_t cur = o[1], nf = o[2], E = o[3], rounds = o[5];
    if (ctx->profile && !ctx->prof_pending.empty())
      ctx->prof_pending.back().bytes += 24.0 * (double)o[7] + 88.0 * (double)o[6];
    if (err != 0) return fail(LGC_ETABLEFULL);
    if (rounds < 1) return fail(LGC_ECUDA);  // the host checked that the first round is small
    st.rounds += rounds;
    st.pushes += o[6];
    st.pushed_edges += o[7];
    *done = rounds;
    // p: where the kernel left it; the other tables are spares or freed
    if (ptab != 0) {
      table_destroy(ctx, &P);
      table_destroy(ctx, &Pn);
      P = ptab == 1 ? A : B;
      Pn = ptab == 1 ? B : A;
    } else {
      table_destroy(ctx, &A);
      table_destroy(ctx, &B);
    }
    if (stop == 1) {
      *over = true;
      return LGC_OK;
    }
    LGC_TRY(F.v.reserve(ctx, std::max<int64_t>(nf, 1024)));
    LGC_TRY(F.s.reserve(ctx, std::max<int64_t>(nf, 1024)));
    LGC_CUDA_TRY(cudaMemcpyAsync(F.v.ptr, X[cur].v.ptr, 4 * nf, cudaMemcpyDeviceToDevice, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(F.s.ptr, X[cur].s.ptr, 4 * nf, cudaMemcpyDeviceToDevice, s));
    F.size = nf;
    F.edges = E;
    *count = o[4];
    return LGC_OK;
  }

  // beta-fraction rounds: keeps in F the first m candidates by r/d
  // descending (ties by ascending id), in ascending id, and moves the others
  // to U (they stay candidates).
  int select_top(const Table& T, int64_t m) {
    cudaStream_t s = ctx->stream;
    const int64_t nf = F.size, E0 = F.edges;
    const int vb = bits_for(g->n);
    LGC_TRY(selv.reserve(ctx, nf));
    LGC_TRY(selv2.reserve(ctx, nf));
    LGC_TRY(seli.reserve(ctx, nf));
    LGC_TRY(seli2.reserve(ctx, nf));
    LGC_TRY(selk.reserve(ctx, nf));
    LGC_TRY(selk2.reserve(ctx, nf));
    LGC_TRY(selcnt.reserve(ctx, 2));
    LGC_TRY(U.v.reserve(ctx, nf));
    LGC_TRY(U.s.reserve(ctx, nf));
    sel_ids_kernel<<<grid_for(nf), kBlock, 0, s>>>(F.v.ptr, nf, selv.ptr, seli.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(radix_sort_u32_i32(ctx, selv.ptr, seli.ptr, selv2.ptr, seli2.ptr, nf, vb));
    sel_keys_kernel<<<grid_for(nf), kBlock, 0, s>>>(F.v.ptr, F.s.ptr, seli.ptr, nf, T, g->deg,
                                                     selk.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(radix_sort_u64_i32(ctx, selk.ptr, seli.ptr, selk2.ptr, seli2.ptr, nf, 64));
    sel_split_kernel<<<grid_for(nf), kBlock, 0, s>>>(F.v.ptr, F.s.ptr, seli.ptr, nf, m, selv.ptr,
                                                      seli2.ptr, U.v.ptr, U.s.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(radix_sort_u32_i32(ctx, selv.ptr, seli2.ptr, selv2.ptr, seli.ptr, m, vb));
    LGC_CUDA_TRY(cudaMemsetAsync(selcnt.ptr, 0, 8, s));
    copy_frontier_kernel<<<grid_for(m), kBlock, 0, s>>>(selv.ptr, seli2.ptr, m, g->deg, F.v.ptr,
                                                         F.s.ptr, selcnt.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, selcnt.ptr, 8, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    F.size = m;
    F.edges = ctx->h_scratch[0];
    U.size = nf - m;
    U.edges = E0 - F.edges;
    return LGC_OK;
  }

  // G (the round's next frontier) united with U: sorted by id, duplicates
  // dropped.
  int merge_rest(const Table& T, double eps) {
    if (U.size == 0) return LGC_OK;
    cudaStream_t s = ctx->stream;
    const int64_t na = G.size, nb = U.size, tot = na + nb;
    LGC_TRY(selv.reserve(ctx, tot));
    LGC_TRY(selv2.reserve(ctx, tot));
    LGC_TRY(seli.reserve(ctx, tot));
    LGC_TRY(seli2.reserve(ctx, tot));
    LGC_TRY(flag.reserve(ctx, tot));
    LGC_TRY(qpos.reserve(ctx, tot));
    LGC_TRY(selcnt.reserve(ctx, 2));
    cat_frontier_kernel<<<grid_for(tot), kBlock, 0, s>>>(G.v.ptr, G.s.ptr, na, U.v.ptr, U.s.ptr,
                                                          nb, T, g->deg, eps, selv.ptr, seli.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(radix_sort_u32_i32(ctx, selv.ptr, seli.ptr, selv2.ptr, seli2.ptr, tot, 32));
    uniq_flags_kernel<<<grid_for(tot), kBlock, 0, s>>>(selv.ptr, tot, flag.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(scan_i64(ctx, flag.ptr, qpos.ptr, tot, false, (int64_t*)selcnt.ptr + 1));
    // G's entries are in selv/seli now: its buffers may be replaced
    LGC_TRY(G.v.reserve(ctx, tot));
    LGC_TRY(G.s.reserve(ctx, tot));
    LGC_CUDA_TRY(cudaMemsetAsync(selcnt.ptr, 0, 8, s));
    uniq_write_kernel<<<grid_for(tot), kBlock, 0, s>>>(selv.ptr, seli.ptr, flag.ptr, qpos.ptr, tot,
                                                        g->deg, G.v.ptr, G.s.ptr, selcnt.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, selcnt.ptr, 16, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    G.edges = ctx->h_scratch[0];
    G.size = ctx->h_scratch[1];
    U.size = 0;
    U.edges = 0;
    return LGC_OK;
  }


  void swap_frontiers() {
    std::swap(F.v, G.v);
    std::swap(F.s, G.s);
    F.size = G.size;
    F.edges = G.edges;
    G.size = 0;
    G.edges = 0;
  }
};

int vgrid(const lgc_ctx* ctx, int64_t nf) {
  int64_t g = ceil_div(nf, kBlock);
  if (g > (ctx->sms * 32)) g = (ctx->sms * 32);
  return (int)(g < 1 ? 1 : g);
}

int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Bulk rounds (atomic mode): the destination is dense and the round pushes at
// least n/32 edges, so a filter pass over the n-bit presence bitmap costs no
// more than a constant times the round's own work.
bool use_bulk(bool det, const Table& D, int64_t round_edges, int64_t n) {
  return !det && D.dense && round_edges >= n / 32;
}

// Pull rounds: when the frontier's edges are at least 1/16 of the graph's,
// gathering over every vertex costs no more than a constant times the push
// it replaces, and it needs neither atomics nor (deterministic mode) records
// and a sort.  The destination must be (made) dense.
bool use_pull(const lgc_ctx* ctx, const lgc_graph* g, int64_t round_edges) {
  if (ctx->table_form == 1 || ctx->pull_policy == 1) return false;
  if (ctx->pull_policy == 2) return true;
  return g->n >= 1024 && round_edges >= g->nnz / 16;
}

// An empty dense table over n vertices (reusing the allocation if it is one).
int fresh_dense(lgc_ctx* ctx, Table* T, int64_t n) {
  if (T->dense && T->cap == n && !T->p) return table_clear(ctx, T);
  table_destroy(ctx, T);
  return table_create_dense(ctx, T, n, false);
}

// An empty dense table for a pull round's destination: only the presence
// bitmap is cleared, since the gathers set a vertex's value when they make it
// a key and never read the value of a non-key, and the table's later readers
// read keys only.
int fresh_dense_keys(lgc_ctx* ctx, Table* T, int64_t n) {
  if (T->dense && T->cap == n && !T->p) {
    LGC_CUDA_TRY(cudaMemsetAsync(T->bits, 0, sizeof(uint32_t) * ((n + 31) / 32), ctx->stream));
    return LGC_OK;
  }
  table_destroy(ctx, T);
  return table_create_dense(ctx, T, n, false);
}

// Before a round that may add up to `add` keys to a persistent table holding
// `count`: switch to the dense form once it may reach n/8 keys, else grow the
// hashed form to stay at most half full.  Frontier slots are re-resolved.
int ensure_capacity(lgc_ctx* ctx, Table* T, int64_t count, int64_t add, int64_t n,
                    const int32_t* fv, int32_t* fs, int64_t nf) {
  if (T->dense) return LGC_OK;
  const int64_t need = min64(count + add, n);
  if (want_dense(ctx, need, n)) return table_to_dense(ctx, T, n, fv, fs, nf);
  if (2 * need > T->cap) return table_grow(ctx, T, 2 * need, fv, fs, nf);
  return LGC_OK;
}

int finish_svec(lgc_ctx* ctx, lgc_graph* g, const Table& T, const double* vals, lgc_svec** p,
                lgc_stats* st_out, lgc_stats& st) {
  int32_t* d_idx = nullptr;
  double* d_val = nullptr;
  int64_t nnz = 0;
  LGC_TRY(table_extract_sorted(ctx, T, vals, g->n, &d_idx, &d_val, &nnz));
  int s = make_svec(ctx, d_idx, d_val, nnz, ctx->result_on_device, p);
  dfree(ctx, d_idx);
  dfree(ctx, d_val);
  st.table_capacity = T.cap;
  if (st_out) *st_out = st;
  return s;
}

}  // namespace

// Picks the degree bins and the shape of the atomic pull gather for this
// graph: for each light threshold L (vertices of degree <= L one thread each,
// the rest in work items), the lists are rebuilt and every heavy-gather shape
// (edges per lane per batch, lanes per work item, bytes per gathered share)
// gathers a frontier of all vertices into a scratch dense set three times
// after one untimed launch; the light gather of the same share width is
// timed the same way, and the fastest sum of the two medians wins.  The
// gathered sums are exact, so every candidate gives the same values.
int autotune_pull(lgc_ctx* ctx, lgc_graph* g) {
  if (g->n == 0 || g->nnz == 0) return LGC_OK;
  cudaStream_t s = ctx->stream;
  const int64_t n = g->n, words = (n + 31) / 32;
  Table D;
  Fx *shx = nullptr, *hacc = nullptr;
  double* shd = nullptr;
  int32_t *range = nullptr, *hcnt = nullptr, *htouch = nullptr;
  uint32_t* q = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = LGC_OK;
  int gb = 1;
  while (gb < 62 && (int64_t{1} << gb) <= g->max_deg) gb++;
  do {
    if ((st = table_create_dense(ctx, &D, n, false)) || (st = dalloc_t(ctx, &shx, n)) ||
        (st = dalloc_t(ctx, &shd, n)) || (st = dalloc_t(ctx, &range, 2)) ||
        (st = dalloc_t(ctx, &q, words)))
      break;
    if (cudaMemsetAsync(q, 0, 4 * words, s) || cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
      st = LGC_ECUDA;
      break;
    }
    tune_fill_kernel<Fx><<<grid_for(n), kBlock, 0, s>>>(shx, n, range, gb);
    LGC_COUNT_LAUNCH(ctx);
    tune_fill_kernel<double><<<grid_for(n), kBlock, 0, s>>>(shd, n, range, gb);
    LGC_COUNT_LAUNCH(ctx);
    // median of three timed launches after an untimed one
    auto timed = [&](auto&& launch, float* med) {
      float t[3] = {0.f, 0.f, 0.f};
      for (int r = -1; r < 3 && st == LGC_OK; r++) {
        if (cudaEventRecord(e0, s)) st = LGC_ECUDA;
        launch();
        LGC_COUNT_LAUNCH(ctx);
        if (cudaEventRecord(e1, s) || cudaEventSynchronize(e1)) st = LGC_ECUDA;
        if (st == LGC_OK && r >= 0 && cudaEventElapsedTime(&t[r], e0, e1)) st = LGC_ECUDA;
      }
      std::sort(t, t + 3);
      *med = t[1];
    };
    // (batch depth, lanes per item) x (16- or 8-byte shares) x light threshold
    const int cand[7][2] = {{4, 32}, {8, 32}, {16, 32}, {8, 16}, {16, 16}, {8, 8}, {16, 8}};
    const int lights[4] = {32, 64, 128, 256};
    float best_ms = 0.f;
    int best = kPullBatch, best_group = 32, best_share = 16, best_light = g->pull_light;
    bool first = true;
    for (int li = 0; li < 4 && st == LGC_OK; li++) {
      if (g->pull_light != lights[li] && (st = rebuild_pull_lists(ctx, g, lights[li])) != LGC_OK)
        break;
      dfree(ctx, hacc);
      dfree(ctx, hcnt);
      dfree(ctx, htouch);
      hacc = nullptr;
      hcnt = nullptr;
      htouch = nullptr;
      if ((st = dalloc_t(ctx, &hacc, g->nheavy + 1)) ||
          (st = dalloc_t(ctx, &hcnt, g->nheavy + 1)) ||
          (st = dalloc_t(ctx, &htouch, g->nheavy + 1)))
        break;
      if (cudaMemsetAsync(hacc, 0, sizeof(Fx) * (g->nheavy + 1), s) ||
          cudaMemsetAsync(hcnt, 0, 4 * (g->nheavy + 1), s) ||
          cudaMemsetAsync(htouch, 0, 4 * (g->nheavy + 1), s)) {
        st = LGC_ECUDA;
        break;
      }
      for (int sb : {16, 8}) {
        float light_ms = 0.f;
        auto light_of = [&](auto* shv) {
          using SH = std::remove_pointer_t<decltype(shv)>;
          const int lgl = (int)std::max<int64_t>(
              1, std::min<int64_t>(ceil_div(g->nlight, kBlock), (ctx->sms * 32)));
          timed([&] {
            pull_light_fx_kernel<SH><<<lgl, kBlock, 0, s>>>(g->light, g->nlight, g->col, shv,
                                                           range, gb, D, 1.0, kFmThreshold, q,
                                                           ctx->d_counters);
          }, &light_ms);
        };
        if (g->nlight > 0) {
          if (sb == 16) light_of(shx);
          else light_of(shd);
        }
        if (st == LGC_OK && g->nitems == 0 && (first || light_ms < best_ms)) {
          first = false;  // every vertex is light at this threshold
          best_ms = light_ms;
          best_share = sb;
          best_light = lights[li];
        }
        for (int ci = 0; ci < 7 && st == LGC_OK && g->nitems > 0; ci++) {
          const int cb = cand[ci][0], cg = cand[ci][1];
          float med = 0.f;
          auto heavy_of = [&](auto* shv) {
            using SH = std::remove_pointer_t<decltype(shv)>;
            HeavyKernel<SH> heavy = heavy_kernel<SH>(cb, cg);
            const int64_t hb = ceil_div(g->nitems, (kBlock / 32) * (32 / cg));
            const int hg = (int)(hb < (ctx->sms * 16) ? hb : (ctx->sms * 16));
            timed([&] {
              heavy<<<hg, kBlock, 0, s>>>(g->off, g->col, g->items, g->nitems, shv, range, gb, D,
                                          1.0, kFmThreshold, q, hacc, hcnt, htouch,
                                          ctx->d_counters);
            }, &med);
          };
          if (sb == 16) heavy_of(shx);
          else heavy_of(shd);
          if (st != LGC_OK) break;
          if (first || light_ms + med < best_ms) {
            first = false;
            best_ms = light_ms + med;
            best = cb;
            best_group = cg;
            best_share = sb;
            best_light = lights[li];
          }
        }
      }
    }
    if (st == LGC_OK && g->pull_light != best_light)
      st = rebuild_pull_lists(ctx, g, best_light);
    if (st == LGC_OK && !first) {
      g->pull_batch = best;
      g->pull_group = best_group;
      g->pull_share = best_share;
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  table_destroy(ctx, &D);
  for (void* p : {(void*)shx, (void*)shd, (void*)range, (void*)q, (void*)hacc, (void*)hcnt,
                  (void*)htouch})
    dfree(ctx, p);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(Counters), s);
  if (cudaGetLastError() != cudaSuccess && st == LGC_OK) st = LGC_ECUDA;
  return st;
}

namespace {

// The synchronous PR-Nibble rounds (Sec. 3.3) from the state in W.F, T and
// count until the frontier is empty, or LGC_EMAXROUNDS once max_rounds
// rounds have run in all (W.st.rounds holds the rounds already run).
int prnibble_rounds(lgc_ctx* ctx, lgc_graph* g, PushWork& W, Table& T, int64_t& count,
                    const lgc_prnibble_params* prm, double beta) {
  const double alpha = prm->alpha, eps = prm->eps;
  const bool det = prm->mode == LGC_MODE_DET;
  const double cs = (2.0 * alpha) / (1.0 + alpha);
  const double cn = (1.0 - alpha) / (1.0 + alpha);
  const int64_t max_rounds = prm->max_rounds > 0 ? prm->max_rounds : INT64_MAX;
  int status = LGC_OK;
  lgc_stats& st = W.st;
  while (W.F.size > 0) {
    if (st.rounds >= max_rounds) return LGC_EMAXROUNDS;
    if (!det && beta >= 1.0 && W.small_round(T, count)) {
      status = W.device_rounds_prnibble(T, &count, alpha, cs, cn, eps, prm->rule,
                                        max_rounds - st.rounds);
      if (status != LGC_OK) return status;
      continue;
    }
    // room for the round's new keys (at most the frontier's edges)
    if ((status = ensure_capacity(ctx, &T, count, W.F.edges, g->n, W.F.v.ptr, W.F.s.ptr,
                                  W.F.size)) != LGC_OK)
      return status;
    const bool pull = use_pull(ctx, g, W.F.edges);
    if (pull && !T.dense &&
        (status = table_to_dense(ctx, &T, g->n, W.F.v.ptr, W.F.s.ptr, W.F.size)) != LGC_OK)
      return status;
    const bool bulk = use_bulk(det, T, W.F.edges, g->n);
    // beta-fraction rounds: the top ceil(beta |F|) candidates push, the
    // others wait in W.U (after every change of the table's slots)
    if (beta < 1.0 && W.F.size > 1) {
      int64_t m = (int64_t)std::ceil(beta * (double)W.F.size);
      m = std::max<int64_t>(1, std::min<int64_t>(m, W.F.size));
      if (m < W.F.size && (status = W.select_top(T, m)) != LGC_OK) return status;
    }
    W.record_trace();
    const int64_t nf = W.F.size;
    if ((status = W.reserve_frontier_scratch(nf)) != LGC_OK) return status;
    if ((status = W.reserve_next(min64(g->n, count + W.F.edges + nf))) != LGC_OK) return status;
    if ((status = W.reset_counters()) != LGC_OK) return status;
    {
      ProfScope ps(ctx, LGC_PROF_VERTEXMAP, 64.0 * nf);
      vmap_prnibble_kernel<<<vgrid(ctx, nf), kBlock, 0, ctx->stream>>>(
          nf, W.F.v.ptr, W.F.s.ptr, T, g->off, alpha, cs, cn, eps, prm->rule, det ? 1 : 0,
          (!det && !bulk && !pull) ? 1 : 0, W.share.ptr, W.cnt.ptr, W.foff.ptr, W.G.v.ptr,
          W.G.s.ptr, (int32_t)W.G.v.cap, ctx->d_counters);
      LGC_COUNT_LAUNCH(ctx);
    }
    if (cudaGetLastError() != cudaSuccess) {
      return LGC_ECUDA;
    }
    Counters C;
    if (pull) {
      status = W.pull_phase(T, eps, kFmThreshold, &C, det);
    } else {
      int64_t nrec = W.F.edges;
      if (det) {
        // one record per edge and one self record per frontier vertex
        // (cnt[i] = d + 1): the total is known without reading it back
        nrec = W.F.edges + nf;
        if ((status = scan_i64(ctx, W.cnt.ptr, W.epos.ptr, nf, false, W.total.ptr)) != LGC_OK)
          return status;
      } else {
        if ((status = scan_i64(ctx, W.cnt.ptr, W.epos.ptr, nf, false, W.total.ptr)) != LGC_OK)
          return status;
      }
      status = W.edge_phase(T, eps, kFmThreshold, det, true, nrec, &C, bulk);
    }
    if (status != LGC_OK) return status;
    st.rounds++;
    st.pushes += nf;
    st.pushed_edges += W.F.edges;
    count += C.inserted;
    W.G.size = C.next_size;
    W.G.edges = C.next_edges;
    if ((status = W.merge_rest(T, eps)) != LGC_OK) return status;  // candidates that waited
    W.swap_frontiers();
  }
  return status;
}

}  // namespace

// PR-Nibble from the seed set seeds[0..k) with weights (null: all 1) and
// beta-fraction rounds (beta = 1: every candidate pushes).  One seed of
// weight 1 with beta = 1 is Fig. alg:pr-nibble2 / alg:pr-nibble exactly.
int run_prnibble_set(lgc_ctx* ctx, lgc_graph* g, int64_t k, const int32_t* seeds,
                     const double* weights, double beta, const lgc_prnibble_params* prm,
                     lgc_svec** p, lgc_stats* st_out, lgc_svec** r_out) {
  if (!g || k < 1 || !seeds || !prm || !(beta > 0.0 && beta <= 1.0)) return LGC_EINVAL;
  const double alpha = prm->alpha, eps = prm->eps;
  if (!(alpha > 0.0 && alpha < 1.0) || !(eps > 0.0) || (prm->rule != 0 && prm->rule != 1) ||
      (prm->mode != 0 && prm->mode != 1))
    return LGC_EINVAL;
  // r starts as w_i / W (W summed left to right), the seeds in ascending id
  std::vector<std::pair<int32_t, double>> init((size_t)k);
  double Wsum = 0.0;
  int64_t dsum = 0;
  for (int64_t i = 0; i < k; i++) {
    int64_t dx = 0;
    LGC_TRY(validate_seed(ctx, g, seeds[i], &dx));
    const double w = weights ? weights[i] : 1.0;
    if (!(w > 0.0) || !std::isfinite(w)) return LGC_EINVAL;
    Wsum = Wsum + w;
    dsum += dx;
    init[i] = {seeds[i], w};
  }
  for (auto& e : init) e.second = e.second / Wsum;
  std::sort(init.begin(), init.end(),
            [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
              return a.first < b.first;
            });
  for (int64_t i = 1; i < k; i++)
    if (init[i].first == init[i - 1].first) return LGC_EINVAL;  // seeds must be distinct
  ctx->trace_ids.clear();
  ctx->trace_sizes.clear();

  PushWork W(ctx, g);
  Table T;
  LGC_TRY(table_create(ctx, &T, 2 * (k + dsum), true));
  int64_t count = k;  // keys in T
  int status = LGC_OK;
  int32_t* d_x = nullptr;
  double* d_r = nullptr;
  do {
    if ((status = W.F.v.reserve(ctx, std::max<int64_t>(k, 1024))) != LGC_OK) break;
    if ((status = W.F.s.reserve(ctx, std::max<int64_t>(k, 1024))) != LGC_OK) break;
    if ((status = W.reset_counters()) != LGC_OK) break;
    if (k == 1) {
      init_seed_kernel<<<1, 1, 0, ctx->stream>>>(T, init[0].first, init[0].second, W.F.v.ptr,
                                                  W.F.s.ptr, ctx->d_counters);
    } else {
      std::vector<int32_t> xs((size_t)k);
      std::vector<double> rs((size_t)k);
      for (int64_t i = 0; i < k; i++) {
        xs[i] = init[i].first;
        rs[i] = init[i].second;
      }
      if ((status = dalloc_t(ctx, &d_x, k)) != LGC_OK) break;
      if ((status = dalloc_t(ctx, &d_r, k)) != LGC_OK) break;
      if (cudaMemcpyAsync(d_x, xs.data(), 4 * k, cudaMemcpyHostToDevice, ctx->stream) ||
          cudaMemcpyAsync(d_r, rs.data(), 8 * k, cudaMemcpyHostToDevice, ctx->stream) ||
          cudaStreamSynchronize(ctx->stream)) {  // xs, rs go out of scope
        status = LGC_ECUDA;
        break;
      }
      init_seeds_kernel<<<grid_for(k), kBlock, 0, ctx->stream>>>(T, d_x, d_r, k, W.F.v.ptr,
                                                                  W.F.s.ptr, ctx->d_counters);
    }
    LGC_COUNT_LAUNCH(ctx);
    W.F.size = k;
    W.F.edges = dsum;
    status = prnibble_rounds(ctx, g, W, T, count, prm, beta);
    W.st.touched = count;
  } while (0);
  if (status == LGC_OK || status == LGC_EMAXROUNDS) {
    int s2 = finish_svec(ctx, g, T, T.p, p, st_out, W.st);
    if (s2 == LGC_OK && r_out) {
      // residual of every key (including zeros), for tests
      int32_t* d_idx = nullptr;
      double* d_val = nullptr;
      int64_t nnz = 0;
      s2 = table_extract_sorted(ctx, T, nullptr, g->n, &d_idx, &d_val, &nnz, false);
      if (s2 == LGC_OK) s2 = make_svec(ctx, d_idx, d_val, nnz, false, r_out);
      dfree(ctx, d_idx);
      dfree(ctx, d_val);
    }
    if (s2 != LGC_OK) status = s2;
  }
  table_destroy(ctx, &T);
  dfree(ctx, d_x);
  dfree(ctx, d_r);
  return status;
}

int run_prnibble(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_prnibble_params* prm,
                 lgc_svec** p, lgc_stats* st_out, lgc_svec** r_out) {
  return run_prnibble_set(ctx, g, 1, &x, nullptr, 1.0, prm, p, st_out, r_out);
}

int run_prnibble_from(lgc_ctx* ctx, lgc_graph* g, const Table& src, const int32_t* d_fv,
                      const int32_t* d_fs, int64_t nf, int64_t E, int64_t count,
                      const lgc_prnibble_params* prm, const lgc_stats& so_far, lgc_svec** p,
                      lgc_stats* st_out) {
  if (!src.p || (!src.dense && src.cap < 64) || (src.dense && src.cap != g->n) || nf < 1)
    return LGC_EINVAL;
  cudaStream_t s = ctx->stream;
  PushWork W(ctx, g);
  Table T;
  // the same form and capacity: the same slots
  if (src.dense) LGC_TRY(table_create_dense(ctx, &T, g->n, true));
  else LGC_TRY(table_create(ctx, &T, src.cap, true));
  int status = LGC_OK;
  do {
    const bool copy_ok =
        src.dense
            ? T.dense && cudaMemcpyAsync(T.dval, src.dval, 8 * src.cap, cudaMemcpyDeviceToDevice,
                                         s) == cudaSuccess &&
                  cudaMemcpyAsync(T.bits, src.bits, 4 * ((src.cap + 31) / 32),
                                  cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                  cudaMemcpyAsync(T.p, src.p, 8 * src.cap, cudaMemcpyDeviceToDevice, s) ==
                      cudaSuccess
            : T.cap == src.cap &&
                  cudaMemcpyAsync(T.s, src.s, sizeof(Slot) * src.cap, cudaMemcpyDeviceToDevice,
                                  s) == cudaSuccess &&
                  cudaMemcpyAsync(T.p, src.p, 8 * src.cap, cudaMemcpyDeviceToDevice, s) ==
                      cudaSuccess;
    if (!copy_ok) {
      status = LGC_ECUDA;
      break;
    }
    if ((status = W.F.v.reserve(ctx, std::max<int64_t>(nf, 1024))) != LGC_OK) break;
    if ((status = W.F.s.reserve(ctx, std::max<int64_t>(nf, 1024))) != LGC_OK) break;
    if (cudaMemcpyAsync(W.F.v.ptr, d_fv, 4 * nf, cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(W.F.s.ptr, d_fs, 4 * nf, cudaMemcpyDeviceToDevice, s)) {
      status = LGC_ECUDA;
      break;
    }
    W.F.size = nf;
    W.F.edges = E;
    W.st.rounds = so_far.rounds;
    W.st.pushes = so_far.pushes;
    W.st.pushed_edges = so_far.pushed_edges;
    status = prnibble_rounds(ctx, g, W, T, count, prm, 1.0);
    W.st.touched = count;
  } while (0);
  if (status == LGC_OK || status == LGC_EMAXROUNDS) {
    const int s2 = finish_svec(ctx, g, T, T.p, p, st_out, W.st);
    if (s2 != LGC_OK) status = s2;
    else if (st_out && status == LGC_EMAXROUNDS) st_out->status_detail = LGC_EMAXROUNDS;
  }
  table_destroy(ctx, &T);
  return status == LGC_EMAXROUNDS ? LGC_OK : status;
}

int run_nibble(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_nibble_params* prm, lgc_svec** p,
               lgc_stats* st_out) {
  int64_t dx = 0;
  LGC_TRY(validate_seed(ctx, g, x, &dx));
  const double eps = prm->eps;
  if (prm->T < 0 || !(eps >= 0.0) || (prm->mode != 0 && prm->mode != 1)) return LGC_EINVAL;
  const bool det = prm->mode == LGC_MODE_DET;
  const int fmode = eps > 0.0 ? kFmThreshold : kFmInserted;
  ctx->trace_ids.clear();
  ctx->trace_sizes.clear();

  PushWork W(ctx, g);
  Table Pc, Pn;  // p and p'
  LGC_TRY(table_create(ctx, &Pc, 64, false));
  int64_t count = 1;
  int status = LGC_OK;
  do {
    if ((status = W.F.v.reserve(ctx, 1024)) != LGC_OK) break;
    if ((status = W.F.s.reserve(ctx, 1024)) != LGC_OK) break;
    if ((status = W.reset_counters()) != LGC_OK) break;
    init_seed_kernel<<<1, 1, 0, ctx->stream>>>(Pc, x, 1.0, W.F.v.ptr, W.F.s.ptr, ctx->d_counters);
    LGC_COUNT_LAUNCH(ctx);
    W.F.size = 1;
    W.F.edges = dx;
    lgc_stats& st = W.st;
    for (int t = 1; t <= prm->T; t++) {
      if (!det && W.small_round_nibble()) {
        int64_t done = 0;
        bool over = false;
        status = W.device_rounds_nibble(Pc, Pn, &count, eps, fmode, prm->T - t + 1, &done, &over);
        if (status != LGC_OK || over) break;
        t += (int)done - 1;  // the loop adds the last one
        continue;
      }
      W.record_trace();
      const int64_t nf = W.F.size;
      const int64_t need = min64(g->n, nf + W.F.edges);
      const bool pull = use_pull(ctx, g, W.F.edges);
      status = pull ? fresh_dense(ctx, &Pn, g->n) : table_fresh(ctx, &Pn, need, g->n, false);
      if (status != LGC_OK) break;  // p' = {}
      const bool bulk = use_bulk(det, Pn, W.F.edges, g->n);
      if ((status = W.reserve_frontier_scratch(nf)) != LGC_OK) break;
      if ((status = W.reserve_next(need)) != LGC_OK) break;
      if ((status = W.reset_counters()) != LGC_OK) break;
      {
        ProfScope ps(ctx, LGC_PROF_VERTEXMAP, 64.0 * nf);
        vmap_nibble_kernel<<<vgrid(ctx, nf), kBlock, 0, ctx->stream>>>(
            nf, W.F.v.ptr, W.F.s.ptr, Pc, Pn, g->off, eps, fmode, det ? 1 : 0,
            (!det && !bulk && !pull) ? 1 : 0, W.share.ptr,
            W.cnt.ptr, W.foff.ptr, W.G.v.ptr, W.G.s.ptr, (int32_t)W.G.v.cap, ctx->d_counters);
        LGC_COUNT_LAUNCH(ctx);
      }
      if (cudaGetLastError() != cudaSuccess) {
        status = LGC_ECUDA;
        break;
      }
      Counters C;
      if (pull) {
        status = W.pull_phase(Pn, eps, fmode, &C, det);
      } else {
        int64_t nrec = W.F.edges;
        if (det) {
          // one record per edge and one self record per frontier vertex
          // (cnt[i] = d + 1): the total is known without reading it back
          nrec = W.F.edges + nf;
          if ((status = scan_i64(ctx, W.cnt.ptr, W.epos.ptr, nf, false, W.total.ptr)) != LGC_OK)
            break;
        } else {
          if ((status = scan_i64(ctx, W.cnt.ptr, W.epos.ptr, nf, false, W.total.ptr)) != LGC_OK)
            break;
        }
        status = W.edge_phase(Pn, eps, fmode, det, true, nrec, &C, bulk);
      }
      if (status != LGC_OK) break;
      st.rounds++;
      st.pushes += nf;
      st.pushed_edges += W.F.edges;
      W.G.size = C.next_size;
      W.G.edges = C.next_edges;
      if (W.G.size == 0) break;  // return the previous p
      std::swap(Pc, Pn);         // p = p'
      count = C.aux + C.inserted;
      W.swap_frontiers();
    }
    st.touched = count;
  } while (0);
  if (status == LGC_OK) status = finish_svec(ctx, g, Pc, nullptr, p, st_out, W.st);
  table_destroy(ctx, &Pc);
  table_destroy(ctx, &Pn);
  return status;
}

int run_hkpr(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_hkpr_params* prm, lgc_svec** p,
             lgc_stats* st_out) {
  int64_t dx = 0;
  LGC_TRY(validate_seed(ctx, g, x, &dx));
  const double t = prm->t, eps = prm->eps;
  const int N = prm->N;
  if (N < 1 || !(t > 0.0) || !(eps >= 0.0) || (prm->mode != 0 && prm->mode != 1))
    return LGC_EINVAL;
  const bool det = prm->mode == LGC_MODE_DET;
  // psi_N = 1, psi_k = 1 + (t/(k+1)) psi_{k+1}; c_j = e^t eps / (2 N psi_j)
  // (the parallel figure's sign of the exponent; LGC_OPT_HK_THRESHOLD_SIGN
  // -1 takes the sequential description's e^-t instead, for comparison)
  std::vector<double> psi(N + 1), c(N + 1);
  psi[N] = 1.0;
  for (int k = N - 1; k >= 0; k--) psi[k] = 1.0 + (t / (double)(k + 1)) * psi[k + 1];
  const double et = ctx->hk_threshold_sign < 0 ? exp(-t) : exp(t);
  for (int j = 0; j <= N; j++) c[j] = (et * eps) / (2.0 * (double)N * psi[j]);
  ctx->trace_ids.clear();
  ctx->trace_sizes.clear();

  PushWork W(ctx, g);
  Table P, Rc, Rn;
  LGC_TRY(table_create(ctx, &P, 2 * (1 + dx), false));
  int status = table_create(ctx, &Rc, 64, false);
  int64_t pcount = 0;
  do {
    if (status != LGC_OK) break;
    if ((status = W.F.v.reserve(ctx, 1024)) != LGC_OK) break;
    if ((status = W.F.s.reserve(ctx, 1024)) != LGC_OK) break;
    if ((status = W.reset_counters()) != LGC_OK) break;
    init_seed_kernel<<<1, 1, 0, ctx->stream>>>(Rc, x, 1.0, W.F.v.ptr, W.F.s.ptr, ctx->d_counters);
    LGC_COUNT_LAUNCH(ctx);
    W.F.size = 1;
    W.F.edges = dx;
    lgc_stats& st = W.st;
    int j = 0;
    while (W.F.size > 0) {
      W.record_trace();
      const int64_t nf = W.F.size;
      const bool last = j + 1 >= N;
      // p takes the frontier (and, on the last level, its neighbours)
      if ((status = ensure_capacity(ctx, &P, pcount, nf + (last ? W.F.edges : 0), g->n, nullptr,
                                    nullptr, 0)) != LGC_OK)
        break;
      const bool pull = use_pull(ctx, g, W.F.edges);
      if (pull && last && !P.dense &&
          (status = table_to_dense(ctx, &P, g->n, nullptr, nullptr, 0)) != LGC_OK)
        break;
      if ((status = W.reserve_frontier_scratch(nf)) != LGC_OK) break;
      if ((status = W.reset_counters()) != LGC_OK) break;
      // a pull round of 8-byte shares takes them straight from the vertexMap
      const bool scattered = pull && W.pull_share_bytes(det) == 8;
      if (scattered) {
        if ((status = W.pull_reserve(det)) != LGC_OK) break;
        if (!det && cudaMemsetAsync(W.prange.ptr, 0, 8, ctx->stream) != cudaSuccess) {
          status = LGC_ECUDA;
          break;
        }
        // per vertex: fv, fs 8, r 8, degree 4, p read-modify-write 16, share 8
        ProfScope ps(ctx, LGC_PROF_VERTEXMAP, 44.0 * nf);
        vmap_hkpr_pull_kernel<<<vgrid(ctx, nf), kBlock, 0, ctx->stream>>>(
            nf, W.F.v.ptr, W.F.s.ptr, Rc, P, g->deg, t, j, last ? 1 : 0, W.psh.ptr,
            det ? nullptr : W.prange.ptr, ctx->d_counters);
        LGC_COUNT_LAUNCH(ctx);
      } else {
        ProfScope ps(ctx, LGC_PROF_VERTEXMAP, 64.0 * nf);
        vmap_hkpr_kernel<<<vgrid(ctx, nf), kBlock, 0, ctx->stream>>>(
            nf, W.F.v.ptr, W.F.s.ptr, Rc, P, g->off, t, j, last ? 1 : 0, W.share.ptr, W.cnt.ptr,
            W.foff.ptr, ctx->d_counters);
        LGC_COUNT_LAUNCH(ctx);
      }
      if (cudaGetLastError() != cudaSuccess) {
        status = LGC_ECUDA;
        break;
      }
      if (!pull &&
          (status = scan_i64(ctx, W.cnt.ptr, W.epos.ptr, nf, false, W.total.ptr)) != LGC_OK)
        break;
      Counters C;
      if (!last) {
        const int64_t need = min64(g->n, W.F.edges);
        status = pull ? fresh_dense_keys(ctx, &Rn, g->n)
                      : table_fresh(ctx, &Rn, need, g->n, false);
        if (status != LGC_OK) break;  // r' = {}
        if ((status = W.reserve_next(need)) != LGC_OK) break;
        const double cj = c[j + 1];
        const int fm = cj > 0.0 ? kFmThreshold : kFmInserted;
        if (pull)
          status = W.pull_phase(Rn, cj, fm, &C, det, scattered);
        else
          status = W.edge_phase(Rn, cj, fm, det, false, W.F.edges, &C,
                                use_bulk(det, Rn, W.F.edges, g->n));
        if (status != LGC_OK) break;
        pcount += C.aux;
        st.rounds++;
        st.pushes += nf;
        st.pushed_edges += W.F.edges;
        std::swap(Rc, Rn);  // r = r'
        W.G.size = C.next_size;
        W.G.edges = C.next_edges;
        W.swap_frontiers();
        j++;
      } else {
        if ((status = W.reserve_next(1)) != LGC_OK) break;
        // no frontier after the last level: fire-and-forget adds in either form
        if (pull)
          status = W.pull_phase(P, 0.0, kFmNone, &C, det, scattered);
        else
          status = W.edge_phase(P, 0.0, kFmNone, det, false, W.F.edges, &C, !det);
        if (status != LGC_OK) break;
        pcount += C.aux + C.inserted;
        st.rounds++;
        st.pushes += nf;
        st.pushed_edges += W.F.edges;
        break;
      }
    }
    st.touched = pcount;
  } while (0);
  if (status == LGC_OK) status = finish_svec(ctx, g, P, nullptr, p, st_out, W.st);
  table_destroy(ctx, &P);
  table_destroy(ctx, &Rc);
  table_destroy(ctx, &Rn);
  return status;
}

}  // namespace lgc

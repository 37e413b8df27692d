// Batched PR-Nibble: B seeds advance together, one launch per kernel per
// round for all of them.  Every seed keeps its own hashed sparse set (r in
// the slot value, p alongside) and its own parameters, and runs exactly the
// synchronous rounds of Sec. 3.3 (Fig. alg:pr-nibble / alg:pr-nibble2): a
// seed's round reads only its own residuals from the start of the round, so
// sharing launches changes nothing in its arithmetic.
//
// The frontiers of all seeds form one list of (seed, vertex, slot) entries,
// grouped by seed.  The vertexMap runs over that list, the edgeMap is
// edge-balanced over the concatenation of all their adjacency lists, and
// the next frontier is appended with per-seed counters (entries, their
// degrees, keys inserted) that the host reads once per round for the whole
// batch to grow each seed's table before its next round.
//
// Deterministic mode emits (seed, destination, share) records, sorts them by
// (seed, destination) stably and folds each run in ascending source order,
// as the single-seed deterministic mode does per seed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "prim.cuh"

namespace lgc {
namespace {

constexpr int kItemsB = 4;
constexpr int kTileB = kBlock * kItemsB;

// Appends (seed, v, slot) to the next frontier: warp-aggregated position,
// per-seed counters by atomics.  Every lane of the calling group must call it.
__device__ inline void batch_append(bool pred, int32_t seed, int32_t v, int32_t slot, int64_t d,
                                    int32_t* nseed, int32_t* nfv, int32_t* nfs, int32_t ncap,
                                    int32_t* gsize, int32_t* gerr, SeedCount* sc) {
  const unsigned active = __activemask();
  const unsigned mask = __ballot_sync(active, pred);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(gsize, __popc(mask));
  base = __shfl_sync(active, base, leader);
  if (pred) {
    const int32_t pos = base + __popc(mask & ((1u << lane) - 1));
    if (pos < ncap) {
      nseed[pos] = seed;
      nfv[pos] = v;
      nfs[pos] = slot;
    } else {
      atomicOr(gerr, kErrFrontierOverflow);
    }
    atomicAdd(&sc[seed].next_size, 1);
    atomicAdd((unsigned long long*)&sc[seed].next_edges, (unsigned long long)d);
  }
}

// Seeds k of this admission: table slots[k] gets r = {seed: 1}, and the
// frontier entry at + k is (slots[k], seed, its table slot).
__global__ void batch_init_kernel(int64_t k, const int32_t* __restrict__ seeds,
                                  const int32_t* __restrict__ slots,
                                  const Table* __restrict__ tabs, int64_t at, int32_t* fseed,
                                  int32_t* fv, int32_t* fs, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = slots[i];
    const Table T = tabs[b];
    int ins = 0;
    const int64_t s = ht_find_or_insert(T, seeds[i], &ins, err);
    if (s >= 0) T.s[s].val = 1.0;
    fseed[at + i] = b;
    fv[at + i] = seeds[i];
    fs[at + i] = (int32_t)s;
  }
}

// vertexMap of every seed's frontier (same arithmetic as the single-seed
// kernel, with the seed's own parameters and table).
__global__ void batch_vmap_kernel(int64_t nf, const int32_t* __restrict__ fseed,
                                  const int32_t* __restrict__ fv, const int32_t* __restrict__ fs,
                                  const Table* __restrict__ tabs,
                                  const SeedParam* __restrict__ prm,
                                  const int64_t* __restrict__ off, int det,
                                  double* __restrict__ share, int64_t* __restrict__ cnt,
                                  int64_t* __restrict__ foff, int32_t* nseed, int32_t* nfv,
                                  int32_t* nfs, int32_t ncap, int32_t* gsize, int32_t* gerr,
                                  SeedCount* sc) {
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nf;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool pred = false;
    int32_t seed = 0, v = 0, slot = 0;
    int64_t d = 0;
    if (i < nf) {
      seed = fseed[i];
      v = fv[i];
      slot = fs[i];
      const Table T = tabs[seed];
      const SeedParam P = prm[seed];
      const bool ok = slot >= 0;
      const double r = ok ? *tb_val(T, slot) : 0.0;
      const int64_t o0 = off[v];
      d = off[v + 1] - o0;
      double sh, rbase;
      if (P.rule == 0) {
        if (ok) T.p[slot] = T.p[slot] + P.cs * r;
        rbase = 0.0;
        sh = (P.cn * r) / (double)d;
      } else {
        if (ok) T.p[slot] = T.p[slot] + P.alpha * r;
        rbase = ((1.0 - P.alpha) * r) / 2.0;
        sh = ((1.0 - P.alpha) * r) / (2.0 * (double)d);
      }
      if (ok) *tb_val(T, slot) = rbase;
      share[i] = sh;
      cnt[i] = d + (det ? 1 : 0);
      foff[i] = o0;
      pred = ok && !det && P.rule == 1 && rbase >= P.eps * (double)d;
    }
    batch_append(pred, seed, v, slot, d, nseed, nfv, nfs, ncap, gsize, gerr, sc);
  }
}

__device__ inline int64_t ub_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Stages the sources owning records [e0, e1) (see the single-seed edgeMap).
__device__ inline int batch_stage(const int64_t* __restrict__ epos, int64_t nf, int64_t total,
                                  int64_t e0, int64_t e1, int64_t* s_i0, int64_t* s_i1,
                                  int64_t* s_epos) {
  if (threadIdx.x == 0) *s_i0 = ub_i64(epos, nf, e0) - 1;
  if (threadIdx.x == 32) *s_i1 = ub_i64(epos, nf, e1 - 1) - 1;
  __syncthreads();
  const int64_t i0 = *s_i0;
  int64_t c = *s_i1 - i0 + 1;
  if (i0 < 0 || c < 0) c = 0;
  if (c > kTileB) c = kTileB;
  for (int j = threadIdx.x; j <= (int)c; j += kBlock)
    s_epos[j] = (i0 + j < nf) ? epos[i0 + j] : total;
  __syncthreads();
  return (int)c;
}

__device__ inline int batch_find(const int64_t* s_epos, int cnt, int64_t e, int64_t* q) {
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

// edgeMap (atomic mode) over all seeds' edges.  Each thread takes kItemsB
// edges and runs them through the phases side by side, as the single-seed
// push does: every item's column, then every item's first probe, then the
// slots, then all the adds, so that a thread keeps kItemsB independent
// memory trips in flight instead of walking one edge's chain after another.
// Keys inserted are counted once per (warp, seed).
__global__ void __launch_bounds__(kBlock)
    batch_emap_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ deg,
                      const double* __restrict__ share, const int64_t* __restrict__ epos,
                      const int64_t* __restrict__ foff, const int32_t* __restrict__ fseed,
                      int64_t nf, int64_t E_host, const int64_t* __restrict__ E_dev,
                      const Table* __restrict__ tabs, const SeedParam* __restrict__ prm,
                      int32_t* nseed, int32_t* nfv, int32_t* nfs, int32_t ncap, int32_t* gsize,
                      int32_t* gerr, SeedCount* sc) {
  __shared__ int64_t s_epos[kTileB + 1];
  __shared__ int64_t s_off[kTileB];
  __shared__ double s_share[kTileB];
  __shared__ int32_t s_seed[kTileB];
  __shared__ int64_t s_i0, s_i1;
  const int lane = threadIdx.x & 31;
  const int64_t E = min(E_host, *E_dev);
  const int64_t ntiles = (E + kTileB - 1) / kTileB;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTileB, e1 = min(E, e0 + kTileB);
    const int cntsrc = batch_stage(epos, nf, E, e0, e1, &s_i0, &s_i1, s_epos);
    const int64_t i0 = s_i0;
    for (int j = threadIdx.x; j < cntsrc; j += kBlock) {
      s_off[j] = foff[i0 + j];
      s_share[j] = share[i0 + j];
      s_seed[j] = fseed[i0 + j];
    }
    __syncthreads();
    int32_t seed[kItemsB], w[kItemsB];
    double sh[kItemsB];
#pragma unroll
    for (int k = 0; k < kItemsB; k++) {
      const int64_t e = e0 + k * kBlock + threadIdx.x;
      int64_t q = 0;
      const int j = e < e1 ? batch_find(s_epos, cntsrc, e, &q) : -1;
      seed[k] = -1;
      w[k] = -1;
      sh[k] = 0.0;
      if (j >= 0) {
        seed[k] = s_seed[j];
        w[k] = col[s_off[j] + q];
        sh[k] = s_share[j];
      }
    }
    // the item's table: a dense one is the value array and the presence
    // bitmap (slot = vertex), a hashed one its slots and hash shift
    const Table* tp[kItemsB];
    int32_t probe[kItemsB];
#pragma unroll
    for (int k = 0; k < kItemsB; k++) {
      probe[k] = 0;
      tp[k] = nullptr;
      if (w[k] >= 0) {
        tp[k] = &tabs[seed[k]];
        probe[k] = tp[k]->dense ? (int32_t)__ldcg(&tp[k]->bits[w[k] >> 5])
                                : __ldcg(&tp[k]->s[hash_slot(w[k], tp[k]->shift)].key);
      }
    }
    int32_t slot[kItemsB];
    int ins[kItemsB];
#pragma unroll
    for (int k = 0; k < kItemsB; k++) {
      slot[k] = -1;
      ins[k] = 0;
      if (w[k] < 0) continue;
      if (tp[k]->dense) {
        slot[k] = w[k];
        const uint32_t m = 1u << (w[k] & 31);
        if (!((uint32_t)probe[k] & m) && !(atomicOr(&tp[k]->bits[w[k] >> 5], m) & m)) ins[k] = 1;
      } else if (probe[k] == w[k] + 1) {
        slot[k] = (int32_t)hash_slot(w[k], tp[k]->shift);
      } else {
        slot[k] = (int32_t)ht_find_or_insert(*tp[k], w[k], &ins[k], &sc[seed[k]].err);
      }
    }
    double old[kItemsB];
#pragma unroll
    for (int k = 0; k < kItemsB; k++)
      old[k] = slot[k] >= 0 ? atomicAdd(tb_val(*tp[k], slot[k]), sh[k]) : 0.0;
#pragma unroll
    for (int k = 0; k < kItemsB; k++) {
      bool pred = false;
      int64_t dw = 0;
      if (slot[k] >= 0) {
        const double nv = old[k] + sh[k];
        const double eps = prm[seed[k]].eps;
        if (nv >= eps) {  // eps*d(w) >= eps for d(w) >= 1: cheap pre-test
          dw = deg[w[k]];
          const double thr = eps * (double)dw;
          pred = old[k] < thr && nv >= thr;
        }
      }
      // inserted keys, one atomic per (warp, seed)
      const unsigned im = __ballot_sync(0xffffffffu, ins[k] != 0);
      if (im) {
        const unsigned peers = __match_any_sync(0xffffffffu, seed[k]);
        if (seed[k] >= 0 && lane == __ffs(peers) - 1 && (im & peers))
          atomicAdd((unsigned long long*)&sc[seed[k]].inserted,
                    (unsigned long long)__popc(im & peers));
      }
      batch_append(pred, seed[k], w[k], slot[k], dw, nseed, nfv, nfs, ncap, gsize, gerr, sc);
    }
    __syncthreads();
  }
}

// Deterministic mode: records keyed (seed << vbits) | destination.
__global__ void __launch_bounds__(kBlock)
    batch_emit_kernel(const int32_t* __restrict__ col, const int32_t* __restrict__ fv,
                      const int32_t* __restrict__ fseed, const double* __restrict__ share,
                      const int64_t* __restrict__ epos, const int64_t* __restrict__ foff,
                      int64_t nf, int64_t R, int vbits, uint64_t* __restrict__ rkey,
                      double* __restrict__ rval) {
  __shared__ int64_t s_epos[kTileB + 1];
  __shared__ int64_t s_off[kTileB];
  __shared__ double s_share[kTileB];
  __shared__ int32_t s_v[kTileB];
  __shared__ int32_t s_seed[kTileB];
  __shared__ int64_t s_i0, s_i1;
  const int64_t ntiles = (R + kTileB - 1) / kTileB;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTileB, e1 = min(R, e0 + kTileB);
    const int cntsrc = batch_stage(epos, nf, R, e0, e1, &s_i0, &s_i1, s_epos);
    const int64_t i0 = s_i0;
    for (int j = threadIdx.x; j < cntsrc; j += kBlock) {
      s_off[j] = foff[i0 + j];
      s_share[j] = share[i0 + j];
      s_v[j] = fv[i0 + j];
      s_seed[j] = fseed[i0 + j];
    }
    __syncthreads();
    for (int k = 0; k < kItemsB; k++) {
      const int64_t e = e0 + k * kBlock + threadIdx.x;
      int64_t q = 0;
      const int j = e < e1 ? batch_find(s_epos, cntsrc, e, &q) : -1;
      if (j < 0) continue;
      const uint64_t hi = (uint64_t)s_seed[j] << vbits;
      if (q == 0) {  // self record (+0.0) keeps the frontier vertex a candidate
        rkey[e] = hi | (uint64_t)s_v[j];
        rval[e] = 0.0;
      } else {
        rkey[e] = hi | (uint64_t)col[s_off[j] + q - 1];
        rval[e] = s_share[j];
      }
    }
    __syncthreads();
  }
}

__global__ void batch_heads_kernel(const uint64_t* __restrict__ rkey, int64_t R,
                                   int64_t* __restrict__ flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R;
       e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = (e == 0 || rkey[e] != rkey[e - 1]) ? 1 : 0;
}

__global__ void batch_starts_kernel(const uint64_t* __restrict__ rkey, int64_t R,
                                    const int64_t* __restrict__ segid,
                                    int64_t* __restrict__ segstart) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < R;
       e += (int64_t)gridDim.x * blockDim.x)
    if (e == 0 || rkey[e] != rkey[e - 1]) segstart[segid[e]] = e;
}

// One thread per (seed, destination) run: left fold from the current value.
__global__ void batch_fold_kernel(const uint64_t* __restrict__ rkey,
                                  const double* __restrict__ rval, int64_t R,
                                  const int64_t* __restrict__ segstart, int64_t nseg, int vbits,
                                  const Table* __restrict__ tabs,
                                  const SeedParam* __restrict__ prm,
                                  const int32_t* __restrict__ deg, int64_t* __restrict__ qflag,
                                  int32_t* __restrict__ segseed, int32_t* __restrict__ segv,
                                  int32_t* __restrict__ segslot, SeedCount* sc) {
  for (int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sg < nseg;
       sg += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = segstart[sg];
    const int64_t e = sg + 1 < nseg ? segstart[sg + 1] : R;
    const int32_t seed = (int32_t)(rkey[b] >> vbits);
    const int32_t w = (int32_t)(rkey[b] & ((1ull << vbits) - 1));
    const Table T = tabs[seed];
    int ins = 0;
    const int64_t slot = tb_find_or_insert(T, w, &ins, &sc[seed].err);
    if (ins) atomicAdd((unsigned long long*)&sc[seed].inserted, 1ull);
    int64_t q = 0;
    if (slot >= 0) {
      double* vp = tb_val(T, slot);
      double acc = *vp;
      for (int64_t k = b; k < e; k++) acc = acc + rval[k];
      *vp = acc;
      q = acc >= prm[seed].eps * (double)deg[w] ? 1 : 0;
    }
    qflag[sg] = q;
    segseed[sg] = seed;
    segv[sg] = w;
    segslot[sg] = (int32_t)slot;
  }
}

__global__ void batch_compact_kernel(const int64_t* __restrict__ qflag,
                                     const int64_t* __restrict__ qpos, int64_t nseg,
                                     const int32_t* __restrict__ segseed,
                                     const int32_t* __restrict__ segv,
                                     const int32_t* __restrict__ segslot,
                                     const int32_t* __restrict__ deg, int32_t* nseed, int32_t* nfv,
                                     int32_t* nfs, int32_t ncap, int32_t* gerr, SeedCount* sc) {
  for (int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sg < nseg;
       sg += (int64_t)gridDim.x * blockDim.x) {
    if (!qflag[sg]) continue;
    const int64_t pos = qpos[sg];
    const int32_t seed = segseed[sg], v = segv[sg];
    if (pos < ncap) {
      nseed[pos] = seed;
      nfv[pos] = v;
      nfs[pos] = segslot[sg];
    } else {
      atomicOr(gerr, kErrFrontierOverflow);
    }
    atomicAdd(&sc[seed].next_size, 1);
    atomicAdd((unsigned long long*)&sc[seed].next_edges, (unsigned long long)deg[v]);
  }
}

// Groups the next frontier by seed: entry i goes to the next free position
// of its seed's range (cursor[b] starts at the range's first position), so
// that the next round's edge tiles are seed-major and the tables written at
// one time are those of a few seeds.  Order inside a seed is arbitrary,
// which the atomic mode does not depend on.
__global__ void batch_group_kernel(int64_t nf, const int32_t* __restrict__ gs,
                                   const int32_t* __restrict__ gv,
                                   const int32_t* __restrict__ gslot, int32_t* cursor,
                                   int32_t* __restrict__ fs, int32_t* __restrict__ fv,
                                   int32_t* __restrict__ fslot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = gs[i];
    const int32_t pos = atomicAdd(&cursor[b], 1);
    fs[pos] = b;
    fv[pos] = gv[i];
    fslot[pos] = gslot[i];
  }
}

// Frontier slots of seeds whose table was rebuilt are looked up again.
__global__ void batch_reresolve_kernel(int64_t nf, const int32_t* __restrict__ fseed,
                                       const int32_t* __restrict__ fv, int32_t* __restrict__ fs,
                                       const Table* __restrict__ tabs,
                                       const int32_t* __restrict__ grown) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x)
    if (grown[fseed[i]]) fs[i] = (int32_t)tb_find(tabs[fseed[i]], fv[i]);
}

// Keeps the frontier entries of seeds that are still running (order kept).
__global__ void batch_keep_flags_kernel(int64_t nf, const int32_t* __restrict__ fseed,
                                        const int32_t* __restrict__ alive,
                                        int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = alive[fseed[i]] ? 1 : 0;
}

__global__ void batch_seed_flags_kernel(int64_t nf, const int32_t* __restrict__ fseed,
                                        int32_t b, int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = fseed[i] == b ? 1 : 0;
}

__global__ void batch_keep_write_kernel(int64_t nf, const int64_t* __restrict__ flag,
                                        const int64_t* __restrict__ pos,
                                        const int32_t* __restrict__ a,
                                        const int32_t* __restrict__ b,
                                        const int32_t* __restrict__ c, int32_t* oa, int32_t* ob,
                                        int32_t* oc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      oa[pos[i]] = a[i];
      ob[pos[i]] = b[i];
      oc[pos[i]] = c[i];
    }
}


}  // namespace

// ---------------------------------------------------------------------------
// Table storage for the batch: the tables created or grown in one step share
// one device allocation (a slab), cleared by one memset; a slab is freed when
// none of its tables is in use any more.  Growing many seeds' tables is one
// rehash launch over all their old slots; the results of all seeds are
// extracted, sorted and copied out together.
// ---------------------------------------------------------------------------
int64_t table_bytes(int64_t cap) { return ceil_div(cap * (int64_t)(sizeof(Slot) + 8), 256) * 256; }

// A dense table over n vertices: values, p, presence bits (each part
// 256-aligned).
int64_t dense_bytes(int64_t n) {
  return 2 * ceil_div(8 * n, 256) * 256 + ceil_div(4 * ceil_div(n, 32), 256) * 256;
}

int64_t pow2_cap(int64_t min_cap) { return pow2_at_least(min_cap < 64 ? 64 : min_cap); }

// Tables for seeds `which`, carved from one new cleared slab: hashed ones
// (slots + p) of the given capacities (powers of two >= 64), or dense ones
// over all n vertices where caps[k] == -1.
int carve_tables(lgc_ctx* ctx, Slabs* S, const std::vector<int64_t>& which,
                 const std::vector<int64_t>& caps, int64_t n, std::vector<Table>* tabs,
                 std::vector<int>* slab_of) {
  if (which.empty()) return LGC_OK;
  int64_t bytes = 0;
  for (int64_t c : caps) {
    if (c > (int64_t{1} << 31)) return LGC_EINVAL;  // 32-bit slot hashes
    bytes += c < 0 ? dense_bytes(n) : table_bytes(c);
  }
  char* base = nullptr;
  LGC_TRY(dalloc_t(ctx, &base, (size_t)bytes));
  LGC_CUDA_TRY(cudaMemsetAsync(base, 0, (size_t)bytes, ctx->stream));
  S->ptr.push_back(base);
  S->refs.push_back((int64_t)which.size());
  const int id = (int)S->ptr.size() - 1;
  int64_t at = 0;
  for (size_t k = 0; k < which.size(); k++) {
    const int64_t cap = caps[k];
    if (cap < 0) {
      Table T;
      T.dense = 1;
      T.cap = n;
      T.dval = reinterpret_cast<double*>(base + at);
      T.p = reinterpret_cast<double*>(base + at + ceil_div(8 * n, 256) * 256);
      T.bits = reinterpret_cast<uint32_t*>(base + at + 2 * ceil_div(8 * n, 256) * 256);
      at += dense_bytes(n);
      (*tabs)[which[k]] = T;
      (*slab_of)[which[k]] = id;
      continue;
    }
    int lg = 0;
    while (((int64_t)1 << lg) < cap) lg++;
    Table T;
    T.cap = cap;
    T.shift = 32 - lg;
    T.s = reinterpret_cast<Slot*>(base + at);
    T.p = reinterpret_cast<double*>(base + at + cap * (int64_t)sizeof(Slot));
    at += table_bytes(cap);
    (*tabs)[which[k]] = T;
    (*slab_of)[which[k]] = id;
  }
  return LGC_OK;
}

// Re-inserts every key of the old tables rg[k].from into rg[k].to; old slot
// i of table k is virtual slot beg[k] + i.
__global__ void batch_rehash_kernel(const Regrow* __restrict__ rg,
                                    const int64_t* __restrict__ beg, int64_t ng, int64_t total,
                                    int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = ub_i64(beg, ng, i) - 1;
    const Table from = rg[k].from, to = rg[k].to;
    const int64_t j = i - beg[k];
    const Slot s = from.s[j];
    if (s.key == 0) continue;
    const int32_t v = s.key - 1;
    if (to.dense) {  // distinct keys: plain writes
      atomicOr(&to.bits[v >> 5], 1u << (v & 31));
      to.dval[v] = s.val;
      to.p[v] = from.p[j];
      continue;
    }
    int ins = 0;
    const int64_t q = ht_find_or_insert(to, v, &ins, err);
    if (q < 0) continue;
    to.s[q].aux = s.aux;
    to.s[q].val = s.val;
    to.p[q] = from.p[j];
  }
}

// Result extraction works on chunks of kChunk slots: chunk c belongs to the
// table b with choff[b] <= c < choff[b + 1] (found once per chunk), so the
// cost is one pass over the tables' slots, with no per-slot search and no
// array as long as all the slots together.
constexpr int kChunk = 4096;

__device__ inline int chunk_table(const int64_t* __restrict__ choff, int64_t B, int64_t c,
                                  int* s_b) {
  if (threadIdx.x == 0) *s_b = (int)(ub_i64(choff, B, c) - 1);
  __syncthreads();
  const int b = *s_b;
  __syncthreads();
  return b;
}

// Slot j of T holds a key with p > 0 (dense: slot = vertex).
__device__ inline bool kept_entry(const Table& T, int64_t j) {
  if (T.dense) return ((T.bits[j >> 5] >> (j & 31)) & 1u) && T.p[j] > 0.0;
  return T.s[j].key != 0 && T.p[j] > 0.0;
}

// Per table, the number of kept entries (keys with p > 0).
__global__ void batch_count_kernel(const Table* __restrict__ tabs,
                                   const int64_t* __restrict__ choff, int64_t B,
                                   int64_t nchunks, unsigned long long* __restrict__ kept) {
  __shared__ int s_b;
  __shared__ unsigned s_cnt;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int b = chunk_table(choff, B, c, &s_b);
    const Table T = tabs[b];
    const int64_t j0 = (c - choff[b]) * kChunk;
    const int64_t j1 = min(T.cap, j0 + kChunk);
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    unsigned k = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x)
      k += kept_entry(T, j) ? 1u : 0u;
    k = __reduce_add_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(&s_cnt, k);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(&kept[b], (unsigned long long)s_cnt);
  }
}

// Writes every kept entry of table b at the next free position of b's
// output range (cursor[b] starts at the range's first position) as the key
// (b << vbits) | vertex and p; the order within a range is fixed afterwards
// by the sort.
__global__ void batch_gather_kernel(const Table* __restrict__ tabs,
                                    const int64_t* __restrict__ choff, int64_t B,
                                    int64_t nchunks, unsigned long long* cursor, int vbits,
                                    uint64_t* __restrict__ key, double* __restrict__ val) {
  __shared__ int s_b;
  const int lane = threadIdx.x & 31;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int b = chunk_table(choff, B, c, &s_b);
    const Table T = tabs[b];
    const int64_t j0 = (c - choff[b]) * kChunk;
    const int64_t j1 = min(T.cap, j0 + kChunk);
    // whole warps iterate together (the chunk is a multiple of the block)
    for (int64_t jb = j0; jb < j1; jb += blockDim.x) {
      const int64_t j = jb + threadIdx.x;
      const bool keep = j < j1 && kept_entry(T, j);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (!m) continue;
      unsigned long long base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(&cursor[b], (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (keep) {
        const unsigned long long at = base + __popc(m & ((1u << lane) - 1u));
        key[at] = ((uint64_t)b << vbits) | (uint64_t)(T.dense ? j : T.s[j].key - 1);
        val[at] = T.p[j];
      }
    }
  }
}

__global__ void batch_ids_kernel(const uint64_t* __restrict__ key, int64_t m, int vbits,
                                 int32_t* __restrict__ idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    idx[i] = (int32_t)(key[i] & ((1ull << vbits) - 1));
}

int extract_all(lgc_ctx* ctx, int64_t B, int64_t n, int vbits, const std::vector<Table>& tabs,
                lgc_svec** p_out) {
  (void)n;
  cudaStream_t s = ctx->stream;
  // chunks per table (a table with capacity 0 -- its seed finished outside
  // the batch -- has none)
  std::vector<int64_t> choff(B + 1, 0);
  for (int64_t b = 0; b < B; b++) choff[b + 1] = choff[b] + ceil_div(tabs[b].cap, kChunk);
  const int64_t nchunks = choff[B];
  const int kbits = vbits + bits_for(B);
  Table* d_tabs = nullptr;
  int64_t* d_choff = nullptr;
  unsigned long long* d_cnt = nullptr;
  uint64_t *key = nullptr, *key2 = nullptr;
  double *val = nullptr, *val2 = nullptr;
  int32_t* idx = nullptr;
  std::vector<int64_t> hstart(B + 1, 0);
  std::vector<unsigned long long> hcnt(B, 0);
  int32_t* hidx = nullptr;
  double* hval = nullptr;
  int st = LGC_OK;
  do {
    if ((st = dalloc_t(ctx, &d_tabs, B)) || (st = dalloc_t(ctx, &d_choff, B + 1)) ||
        (st = dalloc_t(ctx, &d_cnt, B)))
      break;
    if (cudaMemcpyAsync(d_tabs, tabs.data(), sizeof(Table) * B, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_choff, choff.data(), 8 * (B + 1), cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(d_cnt, 0, 8 * B, s)) {
      st = LGC_ECUDA;
      break;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nchunks, (ctx->sms * 16)));
    if (nchunks > 0) {
      batch_count_kernel<<<grid, kBlock, 0, s>>>(d_tabs, d_choff, B, nchunks, d_cnt);
      LGC_COUNT_LAUNCH(ctx);
    }
    if (cudaMemcpyAsync(hcnt.data(), d_cnt, 8 * B, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s)) {
      st = LGC_ECUDA;
      break;
    }
    for (int64_t b = 0; b < B; b++) {
      if ((int64_t)hcnt[b] > tabs[b].cap) st = LGC_ECUDA;  // never size anything from it
      hstart[b + 1] = hstart[b] + (int64_t)hcnt[b];
    }
    if (st != LGC_OK) break;
    const int64_t m = hstart[B];
    if ((st = dalloc_t(ctx, &key, m)) || (st = dalloc_t(ctx, &key2, m)) ||
        (st = dalloc_t(ctx, &val, m)) || (st = dalloc_t(ctx, &val2, m)) ||
        (st = dalloc_t(ctx, &idx, m)))
      break;
    if (nchunks > 0) {
      // the counters become the cursors: each starts at its range
      if (cudaMemcpyAsync(d_cnt, hstart.data(), 8 * B, cudaMemcpyHostToDevice, s)) {
        st = LGC_ECUDA;
        break;
      }
      batch_gather_kernel<<<grid, kBlock, 0, s>>>(d_tabs, d_choff, B, nchunks, d_cnt, vbits,
                                                   key, val);
      LGC_COUNT_LAUNCH(ctx);
    }
    if ((st = radix_sort_u64_f64(ctx, key, val, key2, val2, m, kbits)) != LGC_OK) break;
    batch_ids_kernel<<<grid_for(m), kBlock, 0, s>>>(key, m, vbits, idx);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaGetLastError() != cudaSuccess) {
      st = LGC_ECUDA;
      break;
    }
    if (ctx->result_on_device) {
      for (int64_t b = 0; b < B && st == LGC_OK; b++)
        st = make_svec(ctx, idx + hstart[b], val + hstart[b], hstart[b + 1] - hstart[b], true,
                       &p_out[b]);
      break;
    }
    // page-locked staging: the copies run at the link's speed
    hidx = (int32_t*)host_alloc(4 * (m ? m : 1));
    hval = (double*)host_alloc(8 * (m ? m : 1));
    if (!hidx || !hval) {
      st = LGC_ENOMEM;
      break;
    }
    if ((m && (cudaMemcpyAsync(hidx, idx, 4 * m, cudaMemcpyDeviceToHost, s) ||
               cudaMemcpyAsync(hval, val, 8 * m, cudaMemcpyDeviceToHost, s))) ||
        cudaStreamSynchronize(s)) {
      st = LGC_ECUDA;
      break;
    }
    for (int64_t b = 0; b < B && st == LGC_OK; b++) {
      const int64_t a = hstart[b], k = hstart[b + 1] - a;
      SvecBox* box = new (std::nothrow) SvecBox();
      if (!box) {
        st = LGC_ENOMEM;
        break;
      }
      box->ctx = ctx;
      box->pub.nnz = k;
      box->pub.on_device = 0;
      box->pub.idx = (int32_t*)host_alloc(4 * (k ? k : 1));
      box->pub.val = (double*)host_alloc(8 * (k ? k : 1));
      if (!box->pub.idx || !box->pub.val) {
        host_free(box->pub.idx);
        host_free(box->pub.val);
        delete box;
        st = LGC_ENOMEM;
        break;
      }
      memcpy(box->pub.idx, hidx + a, 4 * k);
      memcpy(box->pub.val, hval + a, 8 * k);
      p_out[b] = &box->pub;
    }
  } while (0);
  for (void* q : {(void*)d_tabs, (void*)d_choff, (void*)d_cnt, (void*)key, (void*)key2,
                  (void*)val, (void*)val2, (void*)idx})
    dfree(ctx, q);
  host_free(hidx);
  host_free(hval);
  return st;
}

// ---------------------------------------------------------------------------
// The batch engine: seeds occupy slots; seeds can be added between rounds
// (they start with their first round at the next one), and a slot whose
// seed has finished is extracted and reused.  lgc_prnibble_batch adds all
// its seeds at once and runs rounds until none has a frontier; the request
// loop adds PR-Nibble requests as they are admitted (continuous batching).
// A seed's rounds are the same whatever else shares them.
// ---------------------------------------------------------------------------
int BatchEngine::init(lgc_ctx* c, lgc_graph* gr, int m) {
  ctx = c;
  g = gr;
  mode = m;
  det = m == LGC_MODE_DET;
  n = g->n;
  vbits = bits_for(n);
  handoff_edges = ctx->batch_handoff != 0 ? (ctx->batch_handoff > 0 ? ctx->batch_handoff
                                                                     : INT64_MAX)
                                           : batch_handoff_of(g);
  LGC_TRY(dalloc_t(ctx, &gsize, 4));  // frontier size, overflow, rehash error, init error
  LGC_CUDA_TRY(cudaMemsetAsync(gsize, 0, 16, ctx->stream));
  return LGC_OK;
}

int BatchEngine::reserve_slots(int64_t want) {
  if (want <= cap) return LGC_OK;
  int64_t nc = std::max<int64_t>(cap ? cap : 64, 64);
  while (nc < want) nc *= 2;
  if (nc > (int64_t{1} << 24)) return LGC_EINVAL;
  auto grow = [&](auto& v, auto fill) { v.resize(nc, fill); };
  grow(seed_of, 0);
  grow(dseed, 0);
  grow(count, 0);
  grow(nfs, 0);
  grow(edges, 0);
  grow(rounds, 0);
  grow(pushes, 0);
  grow(pushed, 0);
  grow(max_rounds, 0);
  grow(sp, SeedParam{});
  grow(prm, lgc_prnibble_params{});
  grow(tabs, Table{});
  grow(slab_of, -1);
  grow(grown, 0);
  grow(alive, 0);
  grow(state, kFree);
  grow(alone, 0);
  grow(p_alone, (lgc_svec*)nullptr);
  grow(st_alone, lgc_stats{});
  grow(sc_h, SeedCount{});
  grow(cursor_h, 0);
  grow(fin_status, 0);
  for (int64_t b = nc - 1; b >= cap; b--) free_slots.push_back(b);
  cap = nc;
  if (det && vbits + bits_for(cap) > 64) return LGC_EINVAL;
  LGC_TRY(d_tabs.reserve(ctx, cap));
  LGC_TRY(d_prm.reserve(ctx, cap));
  LGC_TRY(d_sc.reserve(ctx, cap));
  LGC_TRY(d_grown.reserve(ctx, cap));
  LGC_TRY(d_alive.reserve(ctx, cap));
  tabs_dirty = prm_dirty = true;
  return LGC_OK;
}

int BatchEngine::add(int64_t k, const int32_t* seeds, const lgc_prnibble_params* P,
                     int64_t* slots_out) {
  if (k < 1) return LGC_EINVAL;
  for (int64_t i = 0; i < k; i++) {
    const lgc_prnibble_params& q = P[i];
    if (!(q.alpha > 0.0 && q.alpha < 1.0) || !(q.eps > 0.0) || (q.rule != 0 && q.rule != 1) ||
        q.mode != mode)
      return LGC_EINVAL;
    if (seeds[i] < 0 || seeds[i] >= n || g->hdeg[seeds[i]] < 1) return LGC_EINVAL;
  }
  if ((int64_t)free_slots.size() < k) LGC_TRY(reserve_slots(cap + k));
  std::vector<int64_t> which(k), caps(k);
  std::vector<int32_t> slot32(k);
  for (int64_t i = 0; i < k; i++) {
    const int64_t b = free_slots.back();
    free_slots.pop_back();
    which[i] = b;
    slot32[i] = (int32_t)b;
    if (slots_out) slots_out[i] = b;
    const lgc_prnibble_params& q = P[i];
    seed_of[b] = seeds[i];
    dseed[b] = g->hdeg[seeds[i]];
    count[b] = 1;
    nfs[b] = 1;
    edges[b] = dseed[b];
    rounds[b] = pushes[b] = pushed[b] = 0;
    max_rounds[b] = q.max_rounds > 0 ? q.max_rounds : INT64_MAX;
    prm[b] = q;
    sp[b].alpha = q.alpha;
    sp[b].eps = q.eps;
    sp[b].cs = (2.0 * q.alpha) / (1.0 + q.alpha);
    sp[b].cn = (1.0 - q.alpha) / (1.0 + q.alpha);
    sp[b].rule = q.rule;
    sp[b].pad = 0;
    alive[b] = 1;
    alone[b] = 0;
    state[b] = kRunning;
    fin_status[b] = 0;
    caps[i] = pow2_cap(2 * (1 + dseed[b]));
  }
  LGC_TRY(carve_tables(ctx, &slabs, which, caps, n, &tabs, &slab_of));
  tabs_dirty = prm_dirty = true;
  LGC_TRY(upload());
  cudaStream_t s = ctx->stream;
  // the new seeds' entries go after the running ones (each seed's own
  // entries stay in ascending id, which the deterministic order needs)
  LGC_TRY(Fs.reserve_keep(ctx, nf + k, nf));
  LGC_TRY(Fv.reserve_keep(ctx, nf + k, nf));
  LGC_TRY(Fslot.reserve_keep(ctx, nf + k, nf));
  LGC_TRY(d_new.reserve(ctx, 2 * k));
  LGC_CUDA_TRY(cudaMemcpyAsync(d_new.ptr, seeds, 4 * k, cudaMemcpyHostToDevice, s));
  LGC_CUDA_TRY(cudaMemcpyAsync(d_new.ptr + k, slot32.data(), 4 * k, cudaMemcpyHostToDevice, s));
  batch_init_kernel<<<grid_for(k), kBlock, 0, s>>>(k, d_new.ptr, d_new.ptr + k, d_tabs.ptr, nf,
                                                    Fs.ptr, Fv.ptr, Fslot.ptr, gsize + 3);
  LGC_COUNT_LAUNCH(ctx);
  LGC_CUDA_TRY(cudaGetLastError());
  // the host arrays above go out of scope: the copies must have been made
  LGC_CUDA_TRY(cudaStreamSynchronize(s));
  nf += k;
  running += k;
  return LGC_OK;
}

int BatchEngine::upload() {
  cudaStream_t s = ctx->stream;
  if (tabs_dirty)
    LGC_CUDA_TRY(cudaMemcpyAsync(d_tabs.ptr, tabs.data(), sizeof(Table) * cap,
                                 cudaMemcpyHostToDevice, s));
  if (prm_dirty)
    LGC_CUDA_TRY(cudaMemcpyAsync(d_prm.ptr, sp.data(), sizeof(SeedParam) * cap,
                                 cudaMemcpyHostToDevice, s));
  tabs_dirty = prm_dirty = false;
  return LGC_OK;
}

// Keeps the frontier entries of the seeds still alive (order kept).
int BatchEngine::compact_alive() {
  cudaStream_t s = ctx->stream;
  LGC_CUDA_TRY(cudaMemcpyAsync(d_alive.ptr, alive.data(), 4 * cap, cudaMemcpyHostToDevice, s));
  LGC_TRY(flag.reserve(ctx, nf));
  LGC_TRY(qpos.reserve(ctx, nf));
  LGC_TRY(Gs.reserve(ctx, nf));
  LGC_TRY(Gv.reserve(ctx, nf));
  LGC_TRY(Gslot.reserve(ctx, nf));
  batch_keep_flags_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, Fs.ptr, d_alive.ptr, flag.ptr);
  LGC_COUNT_LAUNCH(ctx);
  LGC_TRY(scan_i64(ctx, flag.ptr, qpos.ptr, nf, false, total.ptr));
  batch_keep_write_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, flag.ptr, qpos.ptr, Fs.ptr, Fv.ptr,
                                                           Fslot.ptr, Gs.ptr, Gv.ptr, Gslot.ptr);
  LGC_COUNT_LAUNCH(ctx);
  std::swap(Fs, Gs);
  std::swap(Fv, Gv);
  std::swap(Fslot, Gslot);
  int64_t k = 0;
  for (int64_t b = 0; b < cap; b++) {
    if (!alive[b]) nfs[b] = 0;
    k += nfs[b];
  }
  nf = k;
  return LGC_OK;
}

void BatchEngine::finish(int64_t b, int status) {
  alive[b] = 0;
  state[b] = kDone;
  fin_status[b] = status;
  running--;
  done.push_back(b);
}

int BatchEngine::round() {
  cudaStream_t s = ctx->stream;
  if (nf == 0) return LGC_OK;
  bool drop = false;
  // seeds with a big frontier continue alone from their state
  for (int64_t b = 0; b < cap; b++) {
    if (state[b] != kRunning || !alive[b] || nfs[b] == 0 || edges[b] < handoff_edges ||
        (!tabs[b].dense && tabs[b].cap < 64))
      continue;
    LGC_TRY(flag.reserve(ctx, nf));
    LGC_TRY(qpos.reserve(ctx, nf));
    LGC_TRY(Gs.reserve(ctx, nf));
    LGC_TRY(Gv.reserve(ctx, nf));
    LGC_TRY(Gslot.reserve(ctx, nf));
    batch_seed_flags_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, Fs.ptr, (int32_t)b, flag.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(scan_i64(ctx, flag.ptr, qpos.ptr, nf, false, total.ptr));
    batch_keep_write_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, flag.ptr, qpos.ptr, Fs.ptr,
                                                             Fv.ptr, Fslot.ptr, Gs.ptr, Gv.ptr,
                                                             Gslot.ptr);
    LGC_COUNT_LAUNCH(ctx);
    lgc_stats so_far{};
    so_far.rounds = rounds[b];
    so_far.pushes = pushes[b];
    so_far.pushed_edges = pushed[b];
    const int st = run_prnibble_from(ctx, g, tabs[b], Gv.ptr, Gslot.ptr, nfs[b], edges[b],
                                     count[b], &prm[b], so_far, &p_alone[b], &st_alone[b]);
    if (st != LGC_OK && st != LGC_EMAXROUNDS) return st;
    alone[b] = 1;
    finish(b, st);
    drop = true;
  }
  if (drop) {
    LGC_TRY(compact_alive());
    if (nf == 0) return LGC_OK;
  }
  // grow the tables of the seeds whose round's new keys would not fit at
  // load 1/2: one slab for all new tables, one rehash launch for all
  // (a table that would take more memory hashed than dense becomes dense)
  std::vector<int64_t> gw, gcap;
  int64_t next_cap = 0, E = 0;
  for (int64_t b = 0; b < cap; b++) {
    grown[b] = 0;
    if (nfs[b] == 0) continue;
    const int64_t need = std::min<int64_t>(count[b] + edges[b], n);
    if (!tabs[b].dense && 2 * need > tabs[b].cap) {
      gw.push_back(b);
      const int64_t hc = pow2_cap(2 * need);
      gcap.push_back(ctx->table_form != 1 && table_bytes(hc) > dense_bytes(n) ? -1 : hc);
      grown[b] = 1;
    }
    next_cap += std::min<int64_t>(n, count[b] + edges[b] + nfs[b]);
    E += edges[b];
  }
  if (!gw.empty()) {
    std::vector<Regrow> rg(gw.size());
    std::vector<int64_t> rgbeg(gw.size() + 1, 0);
    std::vector<int> old_slab(gw.size());
    for (size_t k = 0; k < gw.size(); k++) {
      rg[k].from = tabs[gw[k]];
      old_slab[k] = slab_of[gw[k]];
      rgbeg[k + 1] = rgbeg[k] + tabs[gw[k]].cap;
    }
    LGC_TRY(carve_tables(ctx, &slabs, gw, gcap, n, &tabs, &slab_of));
    for (size_t k = 0; k < gw.size(); k++) rg[k].to = tabs[gw[k]];
    LGC_TRY(d_rg.reserve(ctx, gw.size()));
    LGC_TRY(d_rgbeg.reserve(ctx, gw.size() + 1));
    LGC_CUDA_TRY(cudaMemcpyAsync(d_rg.ptr, rg.data(), sizeof(Regrow) * gw.size(),
                                 cudaMemcpyHostToDevice, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(d_rgbeg.ptr, rgbeg.data(), 8 * (gw.size() + 1),
                                 cudaMemcpyHostToDevice, s));
    const int64_t tot = rgbeg[gw.size()];
    batch_rehash_kernel<<<(int)std::min<int64_t>(ceil_div(tot, kBlock), (ctx->sms * 16)), kBlock,
                          0, s>>>(d_rg.ptr, d_rgbeg.ptr, (int64_t)gw.size(), tot, gsize + 2);
    LGC_COUNT_LAUNCH(ctx);
    // the old tables are released in stream order, after the rehash
    for (size_t k = 0; k < gw.size(); k++) slabs.release(ctx, old_slab[k]);
    tabs_dirty = true;
    LGC_TRY(upload());
    LGC_CUDA_TRY(cudaMemcpyAsync(d_grown.ptr, grown.data(), 4 * cap, cudaMemcpyHostToDevice, s));
    batch_reresolve_kernel<<<grid_for(nf), kBlock, 0, s>>>(nf, Fs.ptr, Fv.ptr, Fslot.ptr,
                                                            d_tabs.ptr, d_grown.ptr);
    LGC_COUNT_LAUNCH(ctx);
  }
  LGC_TRY(share.reserve(ctx, nf));
  LGC_TRY(cnt.reserve(ctx, nf));
  LGC_TRY(epos.reserve(ctx, nf));
  LGC_TRY(foff.reserve(ctx, nf));
  LGC_TRY(total.reserve(ctx, 1));
  LGC_TRY(Gs.reserve(ctx, next_cap));
  LGC_TRY(Gv.reserve(ctx, next_cap));
  LGC_TRY(Gslot.reserve(ctx, next_cap));
  const int32_t ncap = (int32_t)std::min<size_t>(Gv.cap, INT32_MAX);
  LGC_CUDA_TRY(cudaMemsetAsync(d_sc.ptr, 0, sizeof(SeedCount) * cap, s));
  LGC_CUDA_TRY(cudaMemsetAsync(gsize, 0, 8, s));
  {
    ProfScope ps(ctx, LGC_PROF_VERTEXMAP, 64.0 * nf);
    batch_vmap_kernel<<<std::min(grid_for(nf), (ctx->sms * 32)), kBlock, 0, s>>>(
        nf, Fs.ptr, Fv.ptr, Fslot.ptr, d_tabs.ptr, d_prm.ptr, g->off, det ? 1 : 0, share.ptr,
        cnt.ptr, foff.ptr, Gs.ptr, Gv.ptr, Gslot.ptr, ncap, gsize, gsize + 1, d_sc.ptr);
    LGC_COUNT_LAUNCH(ctx);
  }
  LGC_TRY(scan_i64(ctx, cnt.ptr, epos.ptr, nf, false, total.ptr));
  if (!det) {
    if (E > 0) {
      const int64_t tiles = ceil_div(E, kTileB);
      ProfScope ps(ctx, LGC_PROF_EDGEMAP, 24.0 * (double)E + 28.0 * nf);
      batch_emap_kernel<<<(int)std::min<int64_t>(tiles, (ctx->sms * 16)), kBlock, 0, s>>>(
          g->col, g->deg, share.ptr, epos.ptr, foff.ptr, Fs.ptr, nf, E, total.ptr, d_tabs.ptr,
          d_prm.ptr, Gs.ptr, Gv.ptr, Gslot.ptr, ncap, gsize, gsize + 1, d_sc.ptr);
      LGC_COUNT_LAUNCH(ctx);
    }
  } else {
    const int64_t R = E + nf;  // one self record per frontier entry
    LGC_TRY(rk.reserve(ctx, R));
    LGC_TRY(rk2.reserve(ctx, R));
    LGC_TRY(rv.reserve(ctx, R));
    LGC_TRY(rv2.reserve(ctx, R));
    LGC_TRY(flag.reserve(ctx, R));
    LGC_TRY(segid.reserve(ctx, R));
    {
      const int64_t tiles = ceil_div(R, kTileB);
      ProfScope ps(ctx, LGC_PROF_DET_EDGE, 24.0 * (double)E + 28.0 * nf);
      batch_emit_kernel<<<(int)std::min<int64_t>(tiles, (ctx->sms * 16)), kBlock, 0, s>>>(
          g->col, Fv.ptr, Fs.ptr, share.ptr, epos.ptr, foff.ptr, nf, R, vbits, rk.ptr, rv.ptr);
      LGC_COUNT_LAUNCH(ctx);
      LGC_TRY(radix_sort_u64_f64(ctx, rk.ptr, rv.ptr, rk2.ptr, rv2.ptr, R, vbits + bits_for(cap)));
      batch_heads_kernel<<<grid_for(R), kBlock, 0, s>>>(rk.ptr, R, flag.ptr);
      LGC_COUNT_LAUNCH(ctx);
      LGC_TRY(scan_i64(ctx, flag.ptr, segid.ptr, R, false, total.ptr));
    }
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, total.ptr, 8, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nseg = ctx->h_scratch[0];
    LGC_TRY(segstart.reserve(ctx, nseg));
    LGC_TRY(qflag.reserve(ctx, nseg));
    LGC_TRY(qpos.reserve(ctx, nseg));
    LGC_TRY(segseed.reserve(ctx, nseg));
    LGC_TRY(segv.reserve(ctx, nseg));
    LGC_TRY(segslot.reserve(ctx, nseg));
    ProfScope ps(ctx, LGC_PROF_DET_EDGE, 0.0);
    batch_starts_kernel<<<grid_for(R), kBlock, 0, s>>>(rk.ptr, R, segid.ptr, segstart.ptr);
    LGC_COUNT_LAUNCH(ctx);
    batch_fold_kernel<<<grid_for(nseg), kBlock, 0, s>>>(rk.ptr, rv.ptr, R, segstart.ptr, nseg,
                                                         vbits, d_tabs.ptr, d_prm.ptr, g->deg,
                                                         qflag.ptr, segseed.ptr, segv.ptr,
                                                         segslot.ptr, d_sc.ptr);
    LGC_COUNT_LAUNCH(ctx);
    LGC_TRY(scan_i64(ctx, qflag.ptr, qpos.ptr, nseg, false, total.ptr));
    batch_compact_kernel<<<grid_for(nseg), kBlock, 0, s>>>(
        qflag.ptr, qpos.ptr, nseg, segseed.ptr, segv.ptr, segslot.ptr, g->deg, Gs.ptr, Gv.ptr,
        Gslot.ptr, ncap, gsize + 1, d_sc.ptr);
    LGC_COUNT_LAUNCH(ctx);
  }
  LGC_CUDA_TRY(cudaGetLastError());
  // one read-back per round for the whole batch
  LGC_CUDA_TRY(cudaMemcpyAsync(sc_h.data(), d_sc.ptr, sizeof(SeedCount) * cap,
                               cudaMemcpyDeviceToHost, s));
  LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, gsize, 16, cudaMemcpyDeviceToHost, s));
  LGC_CUDA_TRY(cudaStreamSynchronize(s));
  LGC_TRY(sort_check(ctx));
  const int32_t* gs = (const int32_t*)ctx->h_scratch;
  if (gs[1] != 0 || gs[2] != 0 || gs[3] != 0) return LGC_ETABLEFULL;
  int64_t next = 0;
  for (int64_t b = 0; b < cap; b++) {
    if (state[b] != kRunning) continue;
    if (sc_h[b].err) return LGC_ETABLEFULL;
    if (nfs[b] > 0) {
      rounds[b]++;
      pushes[b] += nfs[b];
      pushed[b] += edges[b];
    }
    count[b] += sc_h[b].inserted;
    nfs[b] = sc_h[b].next_size;
    edges[b] = sc_h[b].next_edges;
    next += nfs[b];
  }
  if (!det && next > 0) {
    // the atomic next frontier arrives in no order: group it by seed
    int64_t at = 0;
    for (int64_t b = 0; b < cap; b++) {
      cursor_h[b] = (int32_t)at;
      at += state[b] == kRunning ? nfs[b] : 0;
    }
    if (at != next) return LGC_ECUDA;  // counters disagree with the sizes
    LGC_TRY(Fs.reserve(ctx, next));
    LGC_TRY(Fv.reserve(ctx, next));
    LGC_TRY(Fslot.reserve(ctx, next));
    LGC_TRY(d_cursor.reserve(ctx, cap));
    LGC_CUDA_TRY(cudaMemcpyAsync(d_cursor.ptr, cursor_h.data(), 4 * cap, cudaMemcpyHostToDevice,
                                 s));
    batch_group_kernel<<<std::min(grid_for(next), (ctx->sms * 32)), kBlock, 0, s>>>(
        next, Gs.ptr, Gv.ptr, Gslot.ptr, d_cursor.ptr, Fs.ptr, Fv.ptr, Fslot.ptr);
    LGC_COUNT_LAUNCH(ctx);
  } else {
    // the deterministic next frontier is in (seed, vertex) order already
    std::swap(Fs, Gs);
    std::swap(Fv, Gv);
    std::swap(Fslot, Gslot);
  }
  nf = next;
  // seeds whose frontier is empty are done; seeds at their round limit
  // leave with what they have
  drop = false;
  for (int64_t b = 0; b < cap; b++) {
    if (state[b] != kRunning) continue;
    if (nfs[b] == 0) {
      finish(b, LGC_OK);
    } else if (rounds[b] >= max_rounds[b]) {
      finish(b, LGC_EMAXROUNDS);
      drop = true;
    }
  }
  if (drop && nf > 0) LGC_TRY(compact_alive());
  return LGC_OK;
}

int BatchEngine::extract(const std::vector<int64_t>& which, lgc_svec** outs, lgc_stats* sts) {
  for (size_t i = 0; i < which.size(); i++) outs[i] = nullptr;
  if (which.empty()) return LGC_OK;
  // the chosen slots' tables in a list of their own (seeds that finished
  // alone have theirs already)
  std::vector<Table> tx(which.size());
  for (size_t i = 0; i < which.size(); i++) {
    const int64_t b = which[i];
    if (state[b] != kDone) return LGC_EINVAL;
    tx[i] = alone[b] ? Table{} : tabs[b];
  }
  std::vector<lgc_svec*> got(which.size(), nullptr);
  LGC_TRY(extract_all(ctx, (int64_t)which.size(), n, vbits, tx, got.data()));
  for (size_t i = 0; i < which.size(); i++) {
    const int64_t b = which[i];
    if (alone[b]) {
      lgc_svec_free(got[i]);
      got[i] = p_alone[b];
      p_alone[b] = nullptr;
    }
    outs[i] = got[i];
    if (sts) {
      if (alone[b]) {
        sts[i] = st_alone[b];
      } else {
        sts[i] = lgc_stats{};
        sts[i].rounds = rounds[b];
        sts[i].pushes = pushes[b];
        sts[i].pushed_edges = pushed[b];
        sts[i].touched = count[b];
        sts[i].table_capacity = tabs[b].cap;
        sts[i].status_detail = fin_status[b] == LGC_EMAXROUNDS ? LGC_EMAXROUNDS : 0;
      }
    }
  }
  return LGC_OK;
}

void BatchEngine::release(int64_t b) {
  if (b < 0 || b >= cap || state[b] == kFree) return;
  slabs.release(ctx, slab_of[b]);
  slab_of[b] = -1;
  tabs[b] = Table{};
  tabs_dirty = true;
  lgc_svec_free(p_alone[b]);
  p_alone[b] = nullptr;
  if (state[b] == kRunning) running--;
  state[b] = kFree;
  alive[b] = 0;
  nfs[b] = 0;
  free_slots.push_back(b);
}

int64_t BatchEngine::table_bytes_live() const {
  int64_t t = 0;
  for (int64_t b = 0; b < cap; b++)
    if (state[b] != kFree) t += tabs[b].dense ? dense_bytes(n) : table_bytes(tabs[b].cap);
  return t;
}

void BatchEngine::fini() {
  slabs.release_all(ctx);
  for (int64_t b = 0; b < cap; b++) lgc_svec_free(p_alone[b]);
  p_alone.clear();
  for (auto* d : {&Fs, &Fv, &Fslot, &Gs, &Gv, &Gslot, &segseed, &segv, &segslot, &d_cursor,
                  &d_new, &d_grown, &d_alive})
    d->release(ctx);
  for (auto* d : {&share, &rv, &rv2}) d->release(ctx);
  for (auto* d : {&cnt, &epos, &foff, &total, &flag, &segid, &segstart, &qflag, &qpos})
    d->release(ctx);
  rk.release(ctx);
  rk2.release(ctx);
  d_rg.release(ctx);
  d_rgbeg.release(ctx);
  d_tabs.release(ctx);
  d_prm.release(ctx);
  d_sc.release(ctx);
  dfree(ctx, gsize);
  gsize = nullptr;
}

int64_t batch_handoff_of(const lgc_graph* g) {
  return g->batch_handoff ? g->batch_handoff
                          : std::max<int64_t>(int64_t{1} << 20, g->nnz / 64);
}

// Times one batch of 256 seeds (degree >= 2, drawn by a fixed SplitMix64
// stream; eps log-uniform in [1e-7, 1e-5]; alpha 0.01; atomic) at each
// candidate hand-off threshold -- 2m/64, 2m/16, 2m/4, never -- after one
// untimed run, and keeps the fastest for the graph.
int autotune_batch(lgc_ctx* ctx, lgc_graph* g) {
  if (g->nnz == 0) return LGC_OK;
  std::vector<int32_t> seeds;
  std::vector<lgc_prnibble_params> prm;
  uint64_t k = 0;
  auto mix = [](uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  while ((int)seeds.size() < 256 && k < 64 * (uint64_t)g->n + 4096) {
    const uint64_t w = mix(k++);
    const int32_t v = (int32_t)(w % (uint64_t)g->n);
    if (g->hdeg[v] < 2) continue;
    const double u = (double)(mix(w) >> 11) * 0x1.0p-53;
    lgc_prnibble_params p{};
    p.alpha = 0.01;
    p.eps = pow(10.0, -7.0 + 2.0 * u);
    p.rule = LGC_RULE_OPT;
    p.mode = LGC_MODE_ATOMIC;
    seeds.push_back(v);
    prm.push_back(p);
  }
  const int64_t B = (int64_t)seeds.size();
  if (B == 0) return LGC_OK;
  const bool dev = ctx->result_on_device;
  const int64_t user = ctx->batch_handoff;
  ctx->result_on_device = true;
  ctx->batch_handoff = 0;  // the graph's value decides below
  const int64_t cand[4] = {std::max<int64_t>(int64_t{1} << 20, g->nnz / 64),
                           std::max<int64_t>(int64_t{1} << 20, g->nnz / 16),
                           std::max<int64_t>(int64_t{1} << 20, g->nnz / 4), INT64_MAX};
  std::vector<lgc_svec*> out(B, nullptr);
  int st = LGC_OK;
  double best_s = 0.0;
  int64_t best = cand[0];
  for (int c = -1; c < 4 && st == LGC_OK; c++) {
    g->batch_handoff = cand[c < 0 ? 0 : c];
    const double t0 = now_seconds();
    st = run_prnibble_batch(ctx, g, B, seeds.data(), prm.data(), out.data(), nullptr);
    if (st == LGC_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = LGC_ECUDA;
    const double dt = now_seconds() - t0;
    for (int64_t b = 0; b < B; b++) {
      lgc_svec_free(out[b]);
      out[b] = nullptr;
    }
    if (st == LGC_OK && c >= 0 && (c == 0 || dt < best_s)) {
      best_s = dt;
      best = cand[c];
    }
  }
  g->batch_handoff = st == LGC_OK ? best : 0;
  ctx->result_on_device = dev;
  ctx->batch_handoff = user;
  return st;
}

int run_prnibble_batch(lgc_ctx* ctx, lgc_graph* g, int64_t B, const int32_t* seeds_h,
                       const lgc_prnibble_params* prm_h, lgc_svec** p_out, lgc_stats* st_out) {
  if (!g || B < 1 || B > (1 << 24) || !seeds_h || !prm_h || !p_out) return LGC_EINVAL;
  const int mode = prm_h[0].mode;
  if (mode != 0 && mode != 1) return LGC_EINVAL;
  for (int64_t b = 0; b < B; b++) p_out[b] = nullptr;
  BatchEngine E;
  int status = E.init(ctx, g, mode);
  std::vector<int64_t> slot(B);
  if (status == LGC_OK) status = E.reserve_slots(B);
  if (status == LGC_OK) status = E.add(B, seeds_h, prm_h, slot.data());
  while (status == LGC_OK && E.nf > 0) status = E.round();
  if (status == LGC_OK) status = E.extract(slot, p_out, st_out);
  E.fini();
  if (status != LGC_OK) {
    for (int64_t b = 0; b < B; b++) {
      lgc_svec_free(p_out[b]);
      p_out[b] = nullptr;
    }
  }
  return status;
}

}  // namespace lgc

extern "C" int lgc_prnibble_batch(lgc_graph* g, int64_t B, const int32_t* seeds,
                                  const lgc_prnibble_params* prm, lgc_svec** p_out,
                                  lgc_stats* st) {
  if (!g) return LGC_EINVAL;
  return lgc::run_prnibble_batch(g->ctx, g, B, seeds, prm, p_out, st);
}

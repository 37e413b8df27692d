// Parallel sweep cut (Sec. 3.1, Theorem thm:sweep).
//
//  S1  key_i = p[v_i]/d(v_i) for the entries with p > 0
//  S2  stable LSD radix sort on (0x7FFF...F - bits(key)), so keys come out
//      non-increasing; the input is in ascending id, so ties stay in
//      ascending id
//  S3  rank table: hash table v -> i (1-based) over the sorted vertices;
//      vertices outside S_N have rank N+1
//  S4  vol_i = inclusive prefix sum of d(v_i)
//  S5  delta_i = d(v_i) - 2 #{w in N(v_i) : rank(w) < i}: adding v_i to S
//      turns its edges to S_{i-1} from boundary into interior and the rest
//      into boundary.  This is the per-rank sum of the paper's Z pairs, read
//      off without materialising and sorting Z.  Edge-balanced over vol(S_N);
//      for a support of at least n/32 vertices, vertex-centric over the
//      graph's degree-binned lists instead (the swept vertices' lists read in
//      CSR order, as a pull round reads them)
//  S6  cut_i = inclusive prefix sum of delta
//  S7  argmin of cut_i / min(vol_i, 2m - vol_i), compared exactly as
//      cut_i * den_j < cut_j * den_i on 128-bit products, first index on
//      ties, zero denominators skipped
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "prim.cuh"

namespace lgc {

namespace {

constexpr int kTileItems = 4;
constexpr int kTile = kBlock * kTileItems;

// Also flags (bad != 0) entries that are not vertices of degree >= 1.
__global__ void sweep_keys_kernel(const int32_t* __restrict__ idx, const double* __restrict__ val,
                                  int64_t n0, const int32_t* __restrict__ deg, int64_t n,
                                  uint64_t* __restrict__ key, int32_t* __restrict__ id,
                                  unsigned long long* npos, int* bad) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n0;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = idx[i];
    double pv = val[i];
    if (v < 0 || v >= n || deg[v] < 1) {
      atomicOr(bad, 1);
      v = 0;
      pv = 0.0;
    }
    uint64_t k = ~0ull;
    if (pv > 0.0) {
      const double r = pv / (double)deg[v];
      k = 0x7FFFFFFFFFFFFFFFull - (uint64_t)__double_as_longlong(r);
      c++;
    }
    key[i] = k;
    id[i] = v;
  }
  // one atomic per block: same-address atomics from every warp queue in L2
  __shared__ unsigned long long s_c[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_c[k];
    if (t) atomicAdd(npos, t);
  }
}

// The rank set: a dense int32 array indexed by vertex id (0 = not in S_N)
// when the support is a sizeable part of the graph, else a hash table.
// Entries n0 > i >= N (not in the support, sorted last) get d_i = 0, so the
// prefix sums over all n0 entries equal those over the N swept ones.
__global__ void rank_insert_kernel(const int32_t* __restrict__ order, int64_t n0,
                                   const unsigned long long* __restrict__ dN, Table T,
                                   int32_t* __restrict__ dense_rank,
                                   const int32_t* __restrict__ deg, int64_t* __restrict__ d_i,
                                   int* err, int* bad) {
  const int64_t N = (int64_t)*dN;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n0;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= N) {
      d_i[i] = 0;
      continue;
    }
    const int32_t v = order[i];
    if (dense_rank) {
      if (atomicExch(&dense_rank[v], (int32_t)(i + 1)) != 0) atomicOr(bad, 1);  // named twice
    } else {
      int ins = 0;
      const int64_t s = ht_find_or_insert(T, v, &ins, err);
      if (s >= 0) {
        T.s[s].aux = (int32_t)(i + 1);
        if (!ins) atomicOr(bad, 1);  // named twice
      }
    }
    d_i[i] = deg[v];
  }
}

__device__ inline int64_t rank_of(const Table& T, const int32_t* dense_rank, int32_t w,
                                  int64_t N) {
  if (dense_rank) {
    const int32_t r = dense_rank[w];
    return r ? r : N + 1;
  }
  const int64_t s = ht_find(T, w);
  return s >= 0 ? T.s[s].aux : N + 1;
}

// The first sorted vertex of every kTile-edge tile of the vol(S_N) edges:
// vertex i's edges are [vol[i-1], vol[i]), and the tiles starting in that
// range get i (every swept vertex has d >= 1, so each tile start has exactly
// one writer).  N from dN when it is given, else the argument.
// At most cap tiles are written (more only for an invalid input, which ORs
// flag into *bad).
__global__ void tile_first_kernel(const int64_t* __restrict__ vol,
                                  const unsigned long long* __restrict__ dN, int64_t n_arg,
                                  int32_t* __restrict__ tile0, int64_t cap, int* bad, int flag) {
  const int64_t N = dN ? (int64_t)*dN : n_arg;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i > 0 ? vol[i - 1] : 0, b = vol[i];
    for (int64_t t = (a + kTile - 1) / kTile; t * kTile < b; t++) {
      if (t >= cap) {
        atomicOr(bad, flag);
        break;
      }
      tile0[t] = (int32_t)i;
    }
  }
}

// A tile's sorted vertices: from its first one through the next tile's first
// (or the last vertex), at most kTile of them.
__device__ inline int tile_sources(const int32_t* tile0, int64_t tile, int64_t ntiles, int64_t N,
                                   int64_t* i0) {
  *i0 = tile0[tile];
  const int64_t last = tile + 1 < ntiles ? tile0[tile + 1] : N - 1;
  const int64_t cnt = last - *i0 + 1;
  return (int)(cnt < kTile ? cnt : kTile);
}

// Edge-balanced over the vol(S_N) edges of the sorted vertices; counts, per
// vertex v_i, the neighbours ranked before it.
__global__ void __launch_bounds__(kBlock)
    sweep_cross_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                       const int32_t* __restrict__ order, const int64_t* __restrict__ vol,
                       const unsigned long long* __restrict__ dN,
                       const int64_t* __restrict__ dV, const int32_t* __restrict__ tile0,
                       int64_t cap, Table T, const int32_t* __restrict__ dense_rank,
                       int32_t* __restrict__ before) {
  __shared__ int64_t s_vol[kTile];  // inclusive vol of the tile's sources
  __shared__ int64_t s_off[kTile];
  __shared__ int32_t s_cnt[kTile];
  const int64_t N = (int64_t)*dN, V = *dV;
  const int64_t ntiles = min((V + kTile - 1) / kTile, cap);  // cap: invalid input, flagged
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTile, e1 = min(V, e0 + kTile);
    int64_t i0;
    const int cnt = tile_sources(tile0, tile, ntiles, N, &i0);
    for (int j = threadIdx.x; j < cnt; j += kBlock) {
      s_vol[j] = vol[i0 + j];
      s_off[j] = off[order[i0 + j]];
      s_cnt[j] = 0;
    }
    __syncthreads();
    for (int k = 0; k < kTileItems; k++) {
      const int64_t e = e0 + (int64_t)k * kBlock + threadIdx.x;
      if (e < e1) {
        int lo = 0, hi = cnt;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (s_vol[mid] <= e) lo = mid + 1;
          else hi = mid;
        }
        const int j = lo;  // source index within the tile
        if (j >= cnt) continue;
        const int64_t first = j > 0 ? s_vol[j - 1] : (i0 > 0 ? vol[i0 - 1] : 0);
        const int32_t w = col[s_off[j] + (e - first)];
        if (rank_of(T, dense_rank, w, N) < i0 + j + 1) atomicAdd(&s_cnt[j], 1);
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kBlock)
      if (s_cnt[j]) atomicAdd(&before[i0 + j], s_cnt[j]);
    __syncthreads();
  }
}

// S5 vertex-centric: the vertex of rank r (1-based; 0 = not swept) counts
// its neighbours of rank 1..r-1 into before[r-1].  ru - 1 < r - 1 unsigned
// holds exactly for 1 <= ru < r.
__device__ inline int ranked_before(uint32_t ru, uint32_t r) { return ru - 1u < r - 1u; }

// Vertices of degree 1..light, one thread each, from the graph's list
// grouped by degree; four edges' loads in flight.
__global__ void sweep_cross_light_kernel(const LightItem* __restrict__ items, int64_t nl,
                                         const int32_t* __restrict__ col,
                                         const int32_t* __restrict__ drank,
                                         int32_t* __restrict__ before) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    const LightItem it = items[i];
    const uint32_t r = (uint32_t)drank[it.w];
    if (r == 0) continue;
    int cnt = 0;
    for (int k = 0; k < it.d; k += 4) {
      int32_t u[4];
#pragma unroll
      for (int j = 0; j < 4; j++) u[j] = k + j < it.d ? col[it.beg + k + j] : -1;
      uint32_t ru[4];
#pragma unroll
      for (int j = 0; j < 4; j++) ru[j] = u[j] >= 0 ? (uint32_t)drank[u[j]] : 0u;
#pragma unroll
      for (int j = 0; j < 4; j++) cnt += ranked_before(ru[j], r);
    }
    before[r - 1] = cnt;
  }
}

// The other vertices' work items (at most kPullItem edges of one vertex), a
// warp each, eight edges' loads in flight per lane; the items of one vertex
// add into its zeroed count.
__global__ void __launch_bounds__(kBlock)
    sweep_cross_heavy_kernel(const PullItem* __restrict__ items, int64_t nitems,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ drank,
                             int32_t* __restrict__ before) {
  constexpr int kB = 8;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp0; it < nitems; it += nwarps) {  // uniform in the warp
    const PullItem I = items[it];
    const uint32_t r = (uint32_t)drank[I.w];
    if (r == 0) continue;
    int cnt = 0;
    for (int k0 = 0; k0 < I.len; k0 += 32 * kB) {
      int32_t u[kB];
#pragma unroll
      for (int j = 0; j < kB; j++) {
        const int k = k0 + 32 * j + lane;
        u[j] = k < I.len ? col[I.beg + k] : -1;
      }
      uint32_t ru[kB];
#pragma unroll
      for (int j = 0; j < kB; j++) ru[j] = u[j] >= 0 ? (uint32_t)drank[u[j]] : 0u;
#pragma unroll
      for (int j = 0; j < kB; j++) cnt += ranked_before(ru[j], r);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0 && cnt) atomicAdd(&before[r - 1], cnt);
  }
}

__global__ void sweep_delta_kernel(const int64_t* __restrict__ d_i,
                                   const int32_t* __restrict__ before, int64_t N,
                                   int64_t* __restrict__ delta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    delta[i] = d_i[i] - 2 * (int64_t)before[i];
}

struct Best {
  int64_t cut, den, i;  // i = 0-based prefix index, -1 = none
};

__device__ inline bool better(const Best& a, const Best& b) {
  if (a.i < 0) return false;
  if (b.i < 0) return true;
  // a.cut / a.den < b.cut / b.den  <=>  a.cut * b.den < b.cut * a.den (all >= 0)
  const uint64_t x = (uint64_t)a.cut, y = (uint64_t)b.den;
  const uint64_t u = (uint64_t)b.cut, w = (uint64_t)a.den;
  const uint64_t lhs_hi = __umul64hi(x, y), lhs_lo = x * y;
  const uint64_t rhs_hi = __umul64hi(u, w), rhs_lo = u * w;
  if (lhs_hi != rhs_hi) return lhs_hi < rhs_hi;
  if (lhs_lo != rhs_lo) return lhs_lo < rhs_lo;
  return a.i < b.i;
}

__device__ inline Best shfl_best(const Best& b, int o) {
  Best r;
  r.cut = __shfl_xor_sync(0xffffffffu, b.cut, o);
  r.den = __shfl_xor_sync(0xffffffffu, b.den, o);
  r.i = __shfl_xor_sync(0xffffffffu, b.i, o);
  return r;
}

__device__ inline Best block_best(Best b) {
  __shared__ Best s[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) {
    Best c = shfl_best(b, o);
    if (better(c, b)) b = c;
  }
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    b = threadIdx.x < kBlock / 32 ? s[threadIdx.x] : Best{0, 0, -1};
    for (int o = 16; o > 0; o >>= 1) {
      Best c = shfl_best(b, o);
      if (better(c, b)) b = c;
    }
  }
  return b;
}

__global__ void argmin_kernel(const int64_t* __restrict__ cut, const int64_t* __restrict__ vol,
                              const unsigned long long* __restrict__ dN, int64_t two_m,
                              Best* __restrict__ out) {
  const int64_t N = (int64_t)*dN;
  Best b{0, 0, -1};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = vol[i];
    const int64_t den = v < two_m - v ? v : two_m - v;
    if (den > 0) {
      Best c{cut[i], den, i};
      if (better(c, b)) b = c;
    }
  }
  b = block_best(b);
  if (threadIdx.x == 0) out[blockIdx.x] = b;
}

__global__ void argmin_final_kernel(const Best* __restrict__ parts, int nparts,
                                    const int64_t* __restrict__ vol, Best* __restrict__ out,
                                    int64_t* __restrict__ out_vol) {
  Best b{0, 0, -1};
  for (int i = threadIdx.x; i < nparts; i += kBlock)
    if (better(parts[i], b)) b = parts[i];
  b = block_best(b);
  if (threadIdx.x == 0) {
    *out = b;
    *out_vol = b.i >= 0 ? vol[b.i] : 0;
  }
}

// ---------------------------------------------------------------------------
// Batched sweep: the vectors of B seeds in one pass.  Element i of the
// concatenation belongs to seed b with inoff[b] <= i < inoff[b + 1].  After
// the positive entries are kept (seed-major, ids ascending within a seed),
// one sort by key and a stable sort by seed give every seed's sweep order in
// its own segment [nbeg[b], nbeg[b + 1]); vol and cut are prefix sums over
// the whole concatenation, read per seed relative to the segment's start.
// ---------------------------------------------------------------------------
struct SweepIn {
  const int32_t* idx;
  const double* val;
};

__device__ inline int64_t seg_of(const int64_t* __restrict__ beg, int64_t B, int64_t i) {
  int64_t lo = 0, hi = B;  // last b with beg[b] <= i
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (beg[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void bsweep_keys_kernel(const SweepIn* __restrict__ in,
                                   const int64_t* __restrict__ inoff,
                                   int64_t B, int64_t M, const int32_t* __restrict__ deg, int64_t n,
                                   uint64_t* __restrict__ key, int32_t* __restrict__ id,
                                   int32_t* __restrict__ seg, int64_t* __restrict__ keep,
                                   int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = seg_of(inoff, B - 1, i);
    const int64_t j = i - inoff[b];
    int32_t v = in[b].idx[j];
    double pv = in[b].val[j];
    if (v < 0 || v >= n || deg[v] < 1) {
      atomicOr(bad, 1);
      v = 0;
      pv = 0.0;
    }
    const bool pos = pv > 0.0;
    key[i] = pos ? 0x7FFFFFFFFFFFFFFFull -
                       (uint64_t)__double_as_longlong(pv / (double)deg[v])
                 : ~0ull;
    id[i] = v;
    seg[i] = (int32_t)b;
    keep[i] = pos ? 1 : 0;
  }
}

// Compaction of the kept entries (order preserved); cnt[b] boundaries from
// the exclusive positions: nbeg[b] = pos[inoff[b]], nbeg[B] = total.
__global__ void bsweep_compact_kernel(const int64_t* __restrict__ keep,
                                      const int64_t* __restrict__ pos, int64_t M,
                                      const uint64_t* __restrict__ key,
                                      const int32_t* __restrict__ id,
                                      const int32_t* __restrict__ seg, uint64_t* __restrict__ ko,
                                      int32_t* __restrict__ eo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    ko[pos[i]] = key[i];
    eo[pos[i]] = (int32_t)i;  // element index: id[i], seg[i]
  }
}

__global__ void bsweep_bounds_kernel(const int64_t* __restrict__ inoff, int64_t B, int64_t M,
                                     const int64_t* __restrict__ pos,
                                     const int64_t* __restrict__ total,
                                     int64_t* __restrict__ nbeg) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= B;
       b += (int64_t)gridDim.x * blockDim.x)
    nbeg[b] = (b == B || inoff[b] >= M) ? *total : pos[inoff[b]];
}

__global__ void bsweep_segkey_kernel(const int32_t* __restrict__ elem, int64_t N,
                                     const int32_t* __restrict__ seg, uint32_t* __restrict__ sk) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    sk[i] = (uint32_t)seg[elem[i]];
}

// Sorted position i (seed b = sk[i], local rank i - nbeg[b] + 1): vertex id,
// its rank in seed b's table, its degree.
__global__ void bsweep_rank_kernel(const int32_t* __restrict__ elem, int64_t N,
                                   const uint32_t* __restrict__ sk,
                                   const int32_t* __restrict__ id, const int64_t* __restrict__ nbeg,
                                   const Table* __restrict__ tabs,
                                   const int32_t* __restrict__ deg, int32_t* __restrict__ order,
                                   int64_t* __restrict__ d_i, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = id[elem[i]];
    const uint32_t b = sk[i];
    order[i] = v;
    d_i[i] = deg[v];
    int ins = 0;
    const Table T = tabs[b];
    const int64_t s = ht_find_or_insert(T, v, &ins, err);
    if (s >= 0) {
      T.s[s].aux = (int32_t)(i - nbeg[b] + 1);
      if (!ins) atomicOr(err, kErrDuplicate);  // a vector names v twice
    }
  }
}

// Edge-balanced over all seeds' vol(S_N) edges: per sorted position i, the
// neighbours ranked before it in its own seed's order.
__global__ void __launch_bounds__(kBlock)
    bsweep_cross_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                        const int32_t* __restrict__ order, const uint32_t* __restrict__ sk,
                        const int64_t* __restrict__ nbeg, const int64_t* __restrict__ vol,
                        int64_t N, int64_t V, const int32_t* __restrict__ tile0,
                        const Table* __restrict__ tabs, int32_t* __restrict__ before) {
  __shared__ int64_t s_vol[kTile];
  __shared__ int64_t s_off[kTile];
  __shared__ int32_t s_cnt[kTile];
  const int64_t ntiles = (V + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTile, e1 = min(V, e0 + kTile);
    int64_t i0;
    const int cnt = tile_sources(tile0, tile, ntiles, N, &i0);
    for (int j = threadIdx.x; j < cnt; j += kBlock) {
      s_vol[j] = vol[i0 + j];
      s_off[j] = off[order[i0 + j]];
      s_cnt[j] = 0;
    }
    __syncthreads();
    for (int k = 0; k < kTileItems; k++) {
      const int64_t e = e0 + (int64_t)k * kBlock + threadIdx.x;
      if (e < e1) {
        int lo = 0, hi = cnt;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (s_vol[mid] <= e) lo = mid + 1;
          else hi = mid;
        }
        const int j = lo;
        if (j >= cnt) continue;
        const int64_t first = j > 0 ? s_vol[j - 1] : (i0 > 0 ? vol[i0 - 1] : 0);
        const int32_t w = col[s_off[j] + (e - first)];
        const uint32_t b = sk[i0 + j];
        const int64_t s = ht_find(tabs[b], w);
        if (s >= 0 && tabs[b].s[s].aux < i0 + j - nbeg[b] + 1) atomicAdd(&s_cnt[j], 1);
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kBlock)
      if (s_cnt[j]) atomicAdd(&before[i0 + j], s_cnt[j]);
    __syncthreads();
  }
}

// One CTA per seed: argmin over its segment of cut / min(vol, 2m - vol),
// with vol and cut taken relative to the segment's start.
__global__ void bsweep_argmin_kernel(const int64_t* __restrict__ cut,
                                     const int64_t* __restrict__ vol,
                                     const int64_t* __restrict__ nbeg, int64_t B, int64_t two_m,
                                     Best* __restrict__ best, int64_t* __restrict__ best_vol) {
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    const int64_t s0 = nbeg[b], s1 = nbeg[b + 1];
    const int64_t vb = s0 > 0 ? vol[s0 - 1] : 0, cb = s0 > 0 ? cut[s0 - 1] : 0;
    Best x{0, 0, -1};
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
      const int64_t v = vol[i] - vb;
      const int64_t den = v < two_m - v ? v : two_m - v;
      if (den > 0) {
        Best c{cut[i] - cb, den, i - s0};
        if (better(c, x)) x = c;
      }
    }
    x = block_best(x);
    if (threadIdx.x == 0) {
      best[b] = x;
      best_vol[b] = x.i >= 0 ? vol[s0 + x.i] - vb : 0;
    }
    __syncthreads();  // block_best's shared array is reused by the next seed
  }
}

}  // namespace

int run_sweep(lgc_ctx* ctx, lgc_graph* g, const lgc_svec* p, lgc_cluster** out) {
  *out = nullptr;
  if (!p || p->nnz < 0) return LGC_EINVAL;
  cudaStream_t s = ctx->stream;
  const int64_t n0 = p->nnz;
  int32_t* d_in_idx = nullptr;
  double* d_in_val = nullptr;
  uint64_t *key = nullptr, *key2 = nullptr;
  int32_t *id = nullptr, *id2 = nullptr, *before = nullptr;
  int64_t *d_i = nullptr, *vol = nullptr, *delta = nullptr, *misc = nullptr;
  Best *parts = nullptr, *best = nullptr;
  int32_t *drank = nullptr, *tile0 = nullptr;
  Table T;
  int status = LGC_OK;
  Best hb{0, 0, -1};
  int64_t N = 0, best_vol = 0;
  do {
    if ((status = dalloc_t(ctx, &misc, 4)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemsetAsync(misc, 0, 32, s));
    if (n0 == 0) break;
    const int32_t* idx = p->idx;
    const double* val = p->val;
    if (!p->on_device) {
      if ((status = dalloc_t(ctx, &d_in_idx, n0)) != LGC_OK) break;
      if ((status = dalloc_t(ctx, &d_in_val, n0)) != LGC_OK) break;
      LGC_CUDA_TRY(cudaMemcpyAsync(d_in_idx, p->idx, 4 * n0, cudaMemcpyHostToDevice, s));
      LGC_CUDA_TRY(cudaMemcpyAsync(d_in_val, p->val, 8 * n0, cudaMemcpyHostToDevice, s));
      idx = d_in_idx;
      val = d_in_val;
    }
    if ((status = dalloc_t(ctx, &key, n0)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &key2, n0)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &id, n0)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &id2, n0)) != LGC_OK) break;
    int grid = grid_for(n0);
    if (grid > (ctx->sms * 32)) grid = (ctx->sms * 32);
    // S1
    sweep_keys_kernel<<<grid, kBlock, 0, s>>>(idx, val, n0, g->deg, g->n, key, id,
                                               (unsigned long long*)misc, (int*)(misc + 3));
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    // S2
    if ((status = radix_sort_u64_i32(ctx, key, id, key2, id2, n0, 64)) != LGC_OK) break;
    // S3, S4 over all n0 entries: the N = misc[0] positive ones come first
    // and the rest weigh nothing, so no count is read back mid-call.  Ranks
    // in a dense array when the input is a sizeable part of the graph (one
    // 4-byte read per edge in S5), else in a hash table.
    const bool dense_rank = n0 >= g->n / 64 && g->n >= 1024;
    if (dense_rank) {
      if ((status = dalloc_t(ctx, &drank, g->n)) != LGC_OK) break;
      LGC_CUDA_TRY(cudaMemsetAsync(drank, 0, 4 * g->n, s));
    } else if ((status = table_create(ctx, &T, 2 * n0, false)) != LGC_OK) {
      break;
    }
    if ((status = dalloc_t(ctx, &d_i, n0)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &vol, n0)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &delta, n0)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &before, n0)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemsetAsync(before, 0, 4 * n0, s));
    LGC_CUDA_TRY(cudaMemsetAsync(&ctx->d_counters->err, 0, sizeof(int), s));
    const unsigned long long* dN = (const unsigned long long*)misc;
    rank_insert_kernel<<<grid, kBlock, 0, s>>>(id, n0, dN, T, drank, g->deg, d_i,
                                                &ctx->d_counters->err, (int*)(misc + 3));
    LGC_COUNT_LAUNCH(ctx);
    if ((status = scan_i64(ctx, d_i, vol, n0, true, misc + 1)) != LGC_OK) break;
    // S5.  A support of at least n/32 vertices (ranks in the dense array;
    // LGC_OPT_SWEEP_CROSS may force either form) walks the graph's
    // degree-binned lists: one thread per vertex of degree up to the graph's
    // light bin, a warp per work item of the others.
    const bool vertex_centric =
        dense_rank && (ctx->sweep_cross == 2 || (ctx->sweep_cross == 0 && n0 >= g->n / 32));
    if (vertex_centric) {
      // algorithmic bytes: 12 per edge (col 4, rank key 4, rank 4), 24 per vertex
      ProfScope ps(ctx, LGC_PROF_SWEEP, 0.0);
      if (g->nlight > 0) {
        const int lg = (int)std::min<int64_t>(ceil_div(g->nlight, kBlock), ctx->sms * 32);
        sweep_cross_light_kernel<<<lg, kBlock, 0, s>>>(g->light, g->nlight, g->col, drank,
                                                       before);
        LGC_COUNT_LAUNCH(ctx);
      }
      if (g->nitems > 0) {
        const int hg =
            (int)std::min<int64_t>(ceil_div(g->nitems, kBlock / 32), ctx->sms * 16);
        sweep_cross_heavy_kernel<<<hg, kBlock, 0, s>>>(g->items, g->nitems, g->col, drank,
                                                       before);
        LGC_COUNT_LAUNCH(ctx);
      }
    } else {
      // edge-balanced over V = misc[1] edges with a grid sized for the
      // largest possible V (the kernel loops over the tiles that exist); the
      // tiles' first vertices first, for at most min(2m, n0 * max degree)
      // edges
      const int64_t vmax = std::min<int64_t>(g->nnz, n0 * (int64_t)g->max_deg);
      const int64_t cap = vmax / kTile + 1;
      if ((status = dalloc_t(ctx, &tile0, cap)) != LGC_OK) break;
      tile_first_kernel<<<grid, kBlock, 0, s>>>(vol, dN, 0, tile0, cap, (int*)(misc + 3), 1);
      LGC_COUNT_LAUNCH(ctx);
      // algorithmic bytes: 12 per edge (col 4, rank key 4, rank 4), 24 per vertex
      ProfScope ps(ctx, LGC_PROF_SWEEP, 0.0);
      sweep_cross_kernel<<<ctx->sms * 16, kBlock, 0, s>>>(g->off, g->col, id, vol, dN, misc + 1,
                                                          tile0, cap, T, drank, before);
      LGC_COUNT_LAUNCH(ctx);
    }
    sweep_delta_kernel<<<grid, kBlock, 0, s>>>(d_i, before, n0, delta);
    LGC_COUNT_LAUNCH(ctx);
    // S6
    if ((status = scan_i64(ctx, delta, delta, n0, true, nullptr)) != LGC_OK) break;
    // S7
    int ag = grid;
    if (ag > 1024) ag = 1024;
    if ((status = dalloc_t(ctx, &parts, ag)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &best, 1)) != LGC_OK) break;
    argmin_kernel<<<ag, kBlock, 0, s>>>(delta, vol, dN, g->nnz, parts);
    LGC_COUNT_LAUNCH(ctx);
    argmin_final_kernel<<<1, kBlock, 0, s>>>(parts, ag, vol, best, misc + 2);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    LGC_CUDA_TRY(cudaMemcpyAsync(&hb, best, sizeof(Best), cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, misc, 32, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch + 4, &ctx->d_counters->err, 4,
                                 cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    if ((status = sort_check(ctx)) != LGC_OK) break;
    if (*(int*)(ctx->h_scratch + 3) != 0) {
      status = LGC_EINVAL;  // an entry is not a vertex of degree >= 1, or one is named twice
      break;
    }
    if (*(int32_t*)(ctx->h_scratch + 4) & kErrTableFull) status = LGC_ETABLEFULL;
    N = ctx->h_scratch[0];
    best_vol = ctx->h_scratch[2];
    if (ctx->profile && !ctx->prof_pending.empty())
      ctx->prof_pending.back().bytes = 12.0 * (double)ctx->h_scratch[1] + 24.0 * (double)N;
  } while (0);
  if (status == LGC_OK) {
    ClusterBox* b = new (std::nothrow) ClusterBox();
    if (!b) status = LGC_ENOMEM;
    if (b) {
      b->ctx = ctx;
      const int64_t size = hb.i >= 0 ? hb.i + 1 : 0;
      b->pub.size = size;
      b->pub.vol = hb.i >= 0 ? best_vol : 0;
      b->pub.cut = hb.i >= 0 ? hb.cut : 0;
      b->pub.conductance = hb.i >= 0 ? (double)hb.cut / (double)hb.den : INFINITY;
      b->pub.on_device = ctx->result_on_device ? 1 : 0;
      b->pub.ids = nullptr;
      if (ctx->result_on_device) {
        status = dalloc_t(ctx, &b->pub.ids, size);
        if (status == LGC_OK && size)
          if (cudaMemcpyAsync(b->pub.ids, id, 4 * size, cudaMemcpyDeviceToDevice, s) !=
              cudaSuccess)
            status = LGC_ECUDA;
      } else {
        b->pub.ids = (int32_t*)host_alloc(4 * (size ? size : 1));
        if (!b->pub.ids) status = LGC_ENOMEM;
        else if (size) {
          if (cudaMemcpyAsync(b->pub.ids, id, 4 * size, cudaMemcpyDeviceToHost, s) !=
                  cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess)
            status = LGC_ECUDA;
        }
      }
      if (status == LGC_OK) *out = &b->pub;
      else lgc_cluster_free(&b->pub);
    }
  }
  dfree(ctx, d_in_idx);
  dfree(ctx, d_in_val);
  dfree(ctx, key);
  dfree(ctx, key2);
  dfree(ctx, id);
  dfree(ctx, id2);
  dfree(ctx, before);
  dfree(ctx, d_i);
  dfree(ctx, vol);
  dfree(ctx, delta);
  dfree(ctx, misc);
  dfree(ctx, parts);
  dfree(ctx, best);
  dfree(ctx, drank);
  dfree(ctx, tile0);
  table_destroy(ctx, &T);
  return status;
}

// Sweep cuts of B vectors in one pass (see the batched kernels above).
int run_sweep_batch(lgc_ctx* ctx, lgc_graph* g, int64_t B, const lgc_svec* const* ps,
                    lgc_cluster** out) {
  if (B < 1 || B > (1 << 24) || !ps || !out) return LGC_EINVAL;
  for (int64_t b = 0; b < B; b++) {
    out[b] = nullptr;
    if (!ps[b] || ps[b]->nnz < 0) return LGC_EINVAL;
  }
  cudaStream_t s = ctx->stream;
  std::vector<int64_t> inoff(B + 1, 0);
  for (int64_t b = 0; b < B; b++) inoff[b + 1] = inoff[b] + ps[b]->nnz;
  const int64_t M = inoff[B];
  std::vector<SweepIn> hin(B);
  std::vector<int64_t> nbeg(B + 1, 0);
  std::vector<Best> hbest(B, Best{0, 0, -1});
  std::vector<int64_t> hbvol(B, 0);
  int32_t* hord = nullptr;
  int32_t* cidx = nullptr;  // host vectors, concatenated on the device
  double* cval = nullptr;
  SweepIn* d_in = nullptr;
  int64_t *d_inoff = nullptr, *keep = nullptr, *pos = nullptr, *tot = nullptr, *d_nbeg = nullptr;
  uint64_t *key = nullptr, *ko = nullptr, *ko2 = nullptr;
  int32_t *id = nullptr, *seg = nullptr, *eo = nullptr, *eo2 = nullptr, *order = nullptr,
          *before = nullptr, *tile0 = nullptr;
  uint32_t *sk = nullptr, *sk2 = nullptr;
  int64_t *d_i = nullptr, *vol = nullptr, *cut = nullptr, *d_bvol = nullptr;
  Best* d_best = nullptr;
  Table* d_tabs = nullptr;
  char* slab = nullptr;
  int* d_err = nullptr;
  int st = LGC_OK;
  int64_t N = 0;
  do {
    if ((st = dalloc_t(ctx, &d_err, 2)) != LGC_OK) break;
    if (cudaMemsetAsync(d_err, 0, 8, s) != cudaSuccess) { st = LGC_ECUDA; break; }
    if (M > 0) {
      // inputs: device vectors are read in place, host ones copied once
      int64_t host_nnz = 0;
      for (int64_t b = 0; b < B; b++)
        if (!ps[b]->on_device) host_nnz += ps[b]->nnz;
      if (host_nnz > 0) {
        if ((st = dalloc_t(ctx, &cidx, host_nnz)) || (st = dalloc_t(ctx, &cval, host_nnz))) break;
      }
      int64_t at = 0;
      for (int64_t b = 0; b < B && st == LGC_OK; b++) {
        const lgc_svec* p = ps[b];
        if (p->on_device || p->nnz == 0) {
          hin[b] = SweepIn{p->idx, p->val};
        } else {
          if (cudaMemcpyAsync(cidx + at, p->idx, 4 * p->nnz, cudaMemcpyHostToDevice, s) ||
              cudaMemcpyAsync(cval + at, p->val, 8 * p->nnz, cudaMemcpyHostToDevice, s))
            st = LGC_ECUDA;
          hin[b] = SweepIn{cidx + at, cval + at};
          at += p->nnz;
        }
      }
      if (st != LGC_OK) break;
      if ((st = dalloc_t(ctx, &d_in, B)) || (st = dalloc_t(ctx, &d_inoff, B + 1)) ||
          (st = dalloc_t(ctx, &key, M)) || (st = dalloc_t(ctx, &id, M)) ||
          (st = dalloc_t(ctx, &seg, M)) || (st = dalloc_t(ctx, &keep, M)) ||
          (st = dalloc_t(ctx, &pos, M)) || (st = dalloc_t(ctx, &tot, 1)) ||
          (st = dalloc_t(ctx, &d_nbeg, B + 1)))
        break;
      if (cudaMemcpyAsync(d_in, hin.data(), sizeof(SweepIn) * B, cudaMemcpyHostToDevice, s) ||
          cudaMemcpyAsync(d_inoff, inoff.data(), 8 * (B + 1), cudaMemcpyHostToDevice, s)) {
        st = LGC_ECUDA;
        break;
      }
      const int grid = (int)std::min<int64_t>(ceil_div(M, kBlock), (ctx->sms * 32));
      // S1: keys of the positive entries, seed-major, ids ascending per seed
      bsweep_keys_kernel<<<grid, kBlock, 0, s>>>(d_in, d_inoff, B, M, g->deg, g->n, key, id, seg,
                                                 keep, d_err);
      LGC_COUNT_LAUNCH(ctx);
      if ((st = scan_i64(ctx, keep, pos, M, false, tot)) != LGC_OK) break;
      bsweep_bounds_kernel<<<grid_for(B + 1), kBlock, 0, s>>>(d_inoff, B, M, pos, tot, d_nbeg);
      LGC_COUNT_LAUNCH(ctx);
      if (cudaMemcpyAsync(nbeg.data(), d_nbeg, 8 * (B + 1), cudaMemcpyDeviceToHost, s) ||
          cudaMemcpyAsync(ctx->h_scratch, d_err, 4, cudaMemcpyDeviceToHost, s) ||
          cudaStreamSynchronize(s)) {
        st = LGC_ECUDA;
        break;
      }
      if (*(int*)ctx->h_scratch) {
        st = LGC_EINVAL;  // an entry is not a vertex of degree >= 1
        break;
      }
      N = nbeg[B];
    }
    if (N > 0) {
      if ((st = dalloc_t(ctx, &ko, N)) || (st = dalloc_t(ctx, &ko2, N)) ||
          (st = dalloc_t(ctx, &eo, N)) || (st = dalloc_t(ctx, &eo2, N)) ||
          (st = dalloc_t(ctx, &sk, N)) || (st = dalloc_t(ctx, &sk2, N)) ||
          (st = dalloc_t(ctx, &order, N)) || (st = dalloc_t(ctx, &d_i, N)) ||
          (st = dalloc_t(ctx, &vol, N)) || (st = dalloc_t(ctx, &cut, N)) ||
          (st = dalloc_t(ctx, &before, N)))
        break;
      const int grid = (int)std::min<int64_t>(ceil_div(M, kBlock), (ctx->sms * 32));
      bsweep_compact_kernel<<<grid, kBlock, 0, s>>>(keep, pos, M, key, id, seg, ko, eo);
      LGC_COUNT_LAUNCH(ctx);
      // S2: by key, then stably by seed
      if ((st = radix_sort_u64_i32(ctx, ko, eo, ko2, eo2, N, 64)) != LGC_OK) break;
      bsweep_segkey_kernel<<<grid_for(N), kBlock, 0, s>>>(eo, N, seg, sk);
      LGC_COUNT_LAUNCH(ctx);
      if ((st = radix_sort_u32_i32(ctx, sk, eo, sk2, eo2, N, bits_for(B))) != LGC_OK) break;
      // S3: one rank table per seed, all in one cleared slab
      std::vector<Table> tabs(B);
      std::vector<int64_t> toff(B + 1, 0);
      for (int64_t b = 0; b < B; b++) {
        int64_t cap = 64;
        while (cap < 2 * (nbeg[b + 1] - nbeg[b])) cap <<= 1;
        toff[b + 1] = toff[b] + cap;
      }
      if ((st = dalloc_t(ctx, &slab, (size_t)(toff[B] * (int64_t)sizeof(Slot)))) != LGC_OK) break;
      if (cudaMemsetAsync(slab, 0, (size_t)(toff[B] * (int64_t)sizeof(Slot)), s)) {
        st = LGC_ECUDA;
        break;
      }
      for (int64_t b = 0; b < B; b++) {
        const int64_t cap = toff[b + 1] - toff[b];
        int lg = 0;
        while (((int64_t)1 << lg) < cap) lg++;
        tabs[b] = Table();
        tabs[b].cap = cap;
        tabs[b].shift = 32 - lg;
        tabs[b].s = reinterpret_cast<Slot*>(slab) + toff[b];
      }
      if ((st = dalloc_t(ctx, &d_tabs, B)) != LGC_OK) break;
      if (cudaMemcpyAsync(d_tabs, tabs.data(), sizeof(Table) * B, cudaMemcpyHostToDevice, s) ||
          cudaMemsetAsync(before, 0, 4 * N, s)) {
        st = LGC_ECUDA;
        break;
      }
      bsweep_rank_kernel<<<grid_for(N), kBlock, 0, s>>>(eo, N, sk, id, d_nbeg, d_tabs, g->deg,
                                                         order, d_i, d_err + 1);
      LGC_COUNT_LAUNCH(ctx);
      // S4: volumes over the whole concatenation
      if ((st = scan_i64(ctx, d_i, vol, N, true, tot)) != LGC_OK) break;
      if (cudaMemcpyAsync(ctx->h_scratch, tot, 8, cudaMemcpyDeviceToHost, s) ||
          cudaStreamSynchronize(s)) {
        st = LGC_ECUDA;
        break;
      }
      const int64_t V = ctx->h_scratch[0];
      // S5
      if (V > 0) {
        const int64_t tiles = ceil_div(V, kTile);
        if ((st = dalloc_t(ctx, &tile0, tiles)) != LGC_OK) break;
        tile_first_kernel<<<grid_for(N), kBlock, 0, s>>>(vol, nullptr, N, tile0, tiles,
                                                          d_err + 1, kErrDuplicate);
        LGC_COUNT_LAUNCH(ctx);
        ProfScope ps_(ctx, LGC_PROF_SWEEP, 12.0 * (double)V + 24.0 * (double)N);
        const int cg = (int)std::min<int64_t>(tiles, ctx->sms * 16);
        bsweep_cross_kernel<<<cg, kBlock, 0, s>>>(g->off, g->col, order, sk, d_nbeg, vol, N, V,
                                                  tile0, d_tabs, before);
        LGC_COUNT_LAUNCH(ctx);
      }
      sweep_delta_kernel<<<grid_for(N), kBlock, 0, s>>>(d_i, before, N, cut);
      LGC_COUNT_LAUNCH(ctx);
      // S6
      if ((st = scan_i64(ctx, cut, cut, N, true, nullptr)) != LGC_OK) break;
    }
    // S7, per seed
    if ((st = dalloc_t(ctx, &d_best, B)) || (st = dalloc_t(ctx, &d_bvol, B))) break;
    if (N > 0) {
      bsweep_argmin_kernel<<<(int)std::min<int64_t>(B, (ctx->sms * 8)), kBlock, 0, s>>>(
          cut, vol, d_nbeg, B, g->nnz, d_best, d_bvol);
      LGC_COUNT_LAUNCH(ctx);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(hbest.data(), d_best, sizeof(Best) * B, cudaMemcpyDeviceToHost, s) ||
          cudaMemcpyAsync(hbvol.data(), d_bvol, 8 * B, cudaMemcpyDeviceToHost, s) ||
          cudaMemcpyAsync(ctx->h_scratch, d_err + 1, 4, cudaMemcpyDeviceToHost, s)) {
        st = LGC_ECUDA;
        break;
      }
      if (!ctx->result_on_device) {
        hord = (int32_t*)host_alloc(4 * N);
        if (!hord) {
          st = LGC_ENOMEM;
          break;
        }
        if (cudaMemcpyAsync(hord, order, 4 * N, cudaMemcpyDeviceToHost, s)) {
          st = LGC_ECUDA;
          break;
        }
      }
      if (cudaStreamSynchronize(s)) {
        st = LGC_ECUDA;
        break;
      }
      if ((st = sort_check(ctx)) != LGC_OK) break;
      if (*(int*)ctx->h_scratch & kErrDuplicate) {
        st = LGC_EINVAL;
        break;
      }
      if (*(int*)ctx->h_scratch & kErrTableFull) {
        st = LGC_ETABLEFULL;
        break;
      }
    }
    for (int64_t b = 0; b < B && st == LGC_OK; b++) {
      const Best& hb = hbest[b];
      ClusterBox* box = new (std::nothrow) ClusterBox();
      if (!box) {
        st = LGC_ENOMEM;
        break;
      }
      box->ctx = ctx;
      const int64_t size = hb.i >= 0 ? hb.i + 1 : 0;
      box->pub.size = size;
      box->pub.vol = hb.i >= 0 ? hbvol[b] : 0;
      box->pub.cut = hb.i >= 0 ? hb.cut : 0;
      box->pub.conductance = hb.i >= 0 ? (double)hb.cut / (double)hb.den : INFINITY;
      box->pub.on_device = ctx->result_on_device ? 1 : 0;
      box->pub.ids = nullptr;
      if (ctx->result_on_device) {
        st = dalloc_t(ctx, &box->pub.ids, size);
        if (st == LGC_OK && size &&
            cudaMemcpyAsync(box->pub.ids, order + nbeg[b], 4 * size, cudaMemcpyDeviceToDevice, s))
          st = LGC_ECUDA;
      } else {
        box->pub.ids = (int32_t*)host_alloc(4 * (size ? size : 1));
        if (!box->pub.ids) st = LGC_ENOMEM;
        else if (size) memcpy(box->pub.ids, hord + nbeg[b], 4 * size);
      }
      if (st == LGC_OK) out[b] = &box->pub;
      else lgc_cluster_free(&box->pub);
    }
  } while (0);
  if (st != LGC_OK) {
    for (int64_t b = 0; b < B; b++) {
      lgc_cluster_free(out[b]);
      out[b] = nullptr;
    }
  }
  for (void* q : {(void*)cidx, (void*)cval, (void*)d_in, (void*)d_inoff, (void*)keep, (void*)pos,
                  (void*)tot, (void*)d_nbeg, (void*)key, (void*)ko, (void*)ko2, (void*)id,
                  (void*)seg, (void*)eo, (void*)eo2, (void*)order, (void*)before, (void*)sk,
                  (void*)sk2, (void*)d_i, (void*)vol, (void*)cut, (void*)d_bvol, (void*)d_best,
                  (void*)d_tabs, (void*)slab, (void*)d_err, (void*)tile0})
    dfree(ctx, q);
  host_free(hord);
  return st;
}

}  // namespace lgc

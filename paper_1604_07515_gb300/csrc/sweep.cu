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
//      off without materialising and sorting Z.  Edge-balanced over vol(S_N)
//  S6  cut_i = inclusive prefix sum of delta
//  S7  argmin of cut_i / min(vol_i, 2m - vol_i), compared exactly as
//      cut_i * den_j < cut_j * den_i on 128-bit products, first index on
//      ties, zero denominators skipped
#include <math.h>

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
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(npos, c);
}

// The rank set: a dense int32 array indexed by vertex id (0 = not in S_N)
// when the support is a sizeable part of the graph, else a hash table.
__global__ void rank_insert_kernel(const int32_t* __restrict__ order, int64_t N, Table T,
                                   int32_t* __restrict__ dense_rank,
                                   const int32_t* __restrict__ deg, int64_t* __restrict__ d_i,
                                   int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[i];
    if (dense_rank) {
      dense_rank[v] = (int32_t)(i + 1);
    } else {
      int ins = 0;
      const int64_t s = ht_find_or_insert(T, v, &ins, err);
      if (s >= 0) T.s[s].aux = (int32_t)(i + 1);
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

__device__ inline int64_t upper_bound_excl(const int64_t* a, int64_t n, int64_t x) {
  // a = inclusive prefix sums; the source of edge x is the first i with a[i] > x
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Edge-balanced over the vol(S_N) edges of the sorted vertices; counts, per
// vertex v_i, the neighbours ranked before it.
__global__ void __launch_bounds__(kBlock)
    sweep_cross_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                       const int32_t* __restrict__ order, const int64_t* __restrict__ vol,
                       int64_t N, int64_t V, Table T, const int32_t* __restrict__ dense_rank,
                       int32_t* __restrict__ before) {
  __shared__ int64_t s_vol[kTile];  // inclusive vol of the tile's sources
  __shared__ int64_t s_off[kTile];
  __shared__ int32_t s_cnt[kTile];
  __shared__ int64_t s_i0, s_i1;
  const int64_t ntiles = (V + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kTile, e1 = min(V, e0 + kTile);
    if (threadIdx.x == 0) s_i0 = upper_bound_excl(vol, N, e0);
    if (threadIdx.x == 32) s_i1 = upper_bound_excl(vol, N, e1 - 1);
    __syncthreads();
    const int64_t i0 = s_i0;
    int cnt = (int)(s_i1 - i0 + 1);
    if (cnt > kTile) cnt = kTile;  // unreachable: every swept vertex has d >= 1
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
                              int64_t N, int64_t two_m, Best* __restrict__ out) {
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
  int32_t* drank = nullptr;
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
    if (grid > 152 * 32) grid = 152 * 32;
    // S1
    sweep_keys_kernel<<<grid, kBlock, 0, s>>>(idx, val, n0, g->deg, g->n, key, id,
                                               (unsigned long long*)misc, (int*)(misc + 3));
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    // S2
    if ((status = radix_sort_u64_i32(ctx, key, id, key2, id2, n0, 64)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, misc, 32, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    if (*(int*)(ctx->h_scratch + 3) != 0) {
      status = LGC_EINVAL;  // an entry is not a vertex of degree >= 1
      break;
    }
    N = ctx->h_scratch[0];
    if (N == 0) break;
    // S3, S4: ranks in a dense array when the support is a sizeable part of
    // the graph (one 4-byte read per edge in S5), else in a hash table
    const bool dense_rank = N >= g->n / 64 && g->n >= 1024;
    if (dense_rank) {
      if ((status = dalloc_t(ctx, &drank, g->n)) != LGC_OK) break;
      LGC_CUDA_TRY(cudaMemsetAsync(drank, 0, 4 * g->n, s));
    } else if ((status = table_create(ctx, &T, 2 * N, false)) != LGC_OK) {
      break;
    }
    if ((status = dalloc_t(ctx, &d_i, N)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &vol, N)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &delta, N)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &before, N)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemsetAsync(before, 0, 4 * N, s));
    LGC_CUDA_TRY(cudaMemsetAsync(&ctx->d_counters->err, 0, sizeof(int), s));
    rank_insert_kernel<<<grid_for(N), kBlock, 0, s>>>(id, N, T, drank, g->deg, d_i,
                                                       &ctx->d_counters->err);
    LGC_COUNT_LAUNCH(ctx);
    if ((status = scan_i64(ctx, d_i, vol, N, true, misc + 1)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, misc + 1, 8, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t V = ctx->h_scratch[0];
    // S5
    if (V > 0) {
      int64_t tiles = ceil_div(V, kTile);
      int eg = (int)(tiles < 152 * 16 ? tiles : 152 * 16);
      // algorithmic bytes: 12 per edge (col 4, rank key 4, rank 4), 24 per vertex
      ProfScope ps(ctx, LGC_PROF_SWEEP, 12.0 * (double)V + 24.0 * (double)N);
      sweep_cross_kernel<<<eg, kBlock, 0, s>>>(g->off, g->col, id, vol, N, V, T, drank, before);
      LGC_COUNT_LAUNCH(ctx);
    }
    sweep_delta_kernel<<<grid_for(N), kBlock, 0, s>>>(d_i, before, N, delta);
    LGC_COUNT_LAUNCH(ctx);
    // S6
    if ((status = scan_i64(ctx, delta, delta, N, true, nullptr)) != LGC_OK) break;
    // S7
    int ag = grid_for(N);
    if (ag > 1024) ag = 1024;
    if ((status = dalloc_t(ctx, &parts, ag)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &best, 1)) != LGC_OK) break;
    argmin_kernel<<<ag, kBlock, 0, s>>>(delta, vol, N, g->nnz, parts);
    LGC_COUNT_LAUNCH(ctx);
    argmin_final_kernel<<<1, kBlock, 0, s>>>(parts, ag, vol, best, misc + 2);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    LGC_CUDA_TRY(cudaMemcpyAsync(&hb, best, sizeof(Best), cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch + 2, misc + 2, 8, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch + 3, &ctx->d_counters->err, 4,
                                 cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    if (*(int32_t*)(ctx->h_scratch + 3) & kErrTableFull) status = LGC_ETABLEFULL;
    best_vol = ctx->h_scratch[2];
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
        b->pub.ids = (int32_t*)malloc(4 * (size ? size : 1));
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
  table_destroy(ctx, &T);
  return status;
}

}  // namespace lgc

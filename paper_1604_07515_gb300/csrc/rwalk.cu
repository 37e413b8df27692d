// Randomized heat-kernel PageRank (Sec. 3.5): n_walks independent random
// walks from the seed, each of Poisson(t) length capped at K; the endpoints
// go to an array A, which is sorted; run lengths give p[v] = count / n_walks
// (the sort + prefix-sum + filter counting of Sec. 3.5, with the endpoint
// radix-sorted directly by vertex id).
#include <math.h>

#include "common.cuh"
#include "prim.cuh"

namespace lgc {

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplications of counter words 0 and 2; the high halves
// are XORed with counter words 1 and 3 and the round key, the words are
// permuted, and the key is bumped by the Weyl increments between rounds.
struct Philox {
  static constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  static constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
  __device__ static inline uint4 block(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
      const uint32_t hi0 = __umulhi(kMul0, c.x), lo0 = kMul0 * c.x;
      const uint32_t hi1 = __umulhi(kMul1, c.z), lo1 = kMul1 * c.z;
      c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
      k0 += kWeyl0;
      k1 += kWeyl1;
    }
    return c;
  }
};

constexpr int kMaxK = 128;
// Poisson CDF table, passed by value so concurrent calls on different
// streams cannot overwrite each other's table.
struct CdfTable {
  double c[kMaxK];
};

// One thread per walk.  Draw 0 (counter word 2 = 0) fixes the length k:
// u = (w0 * 2^21 + (w1 >> 11)) * 2^-53, k = min{k < K : u < CDF(k)}, else K.
// Draw s (word 2 = s) moves to neighbour floor(w0 * d / 2^32).
__global__ void walk_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                            int32_t x, int64_t n_walks, int K, const CdfTable cdf,
                            uint32_t k0, uint32_t k1,
                            int32_t* __restrict__ A, unsigned long long* steps) {
  unsigned long long my_steps = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_walks;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t ilo = (uint32_t)i, ihi = (uint32_t)((uint64_t)i >> 32);
    const uint4 w = Philox::block(make_uint4(ilo, ihi, 0u, 0u), k0, k1);
    const uint64_t u53 = ((uint64_t)w.x << 21) | (uint64_t)(w.y >> 11);
    const double u = (double)u53 * 0x1.0p-53;
    int k = K;
    for (int kk = 0; kk < K; kk++)
      if (u < cdf.c[kk]) {
        k = kk;
        break;
      }
    int32_t v = x;
    for (int s = 1; s <= k; s++) {
      const uint4 ws = Philox::block(make_uint4(ilo, ihi, (uint32_t)s, 0u), k0, k1);
      const int64_t o0 = off[v];
      const uint64_t d = (uint64_t)(off[v + 1] - o0);
      const uint32_t j = (uint32_t)(((uint64_t)ws.x * d) >> 32);
      v = col[o0 + j];
    }
    A[i] = v;
    my_steps += (unsigned long long)k;
  }
  for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_xor_sync(0xffffffffu, my_steps, o);
  if ((threadIdx.x & 31) == 0 && my_steps) atomicAdd(steps, my_steps);
}

__global__ void rle_heads_kernel(const uint32_t* __restrict__ a, int64_t n,
                                 int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || a[i] != a[i - 1]) ? 1 : 0;
}

// Run r starts at pos; its count is the next run's start minus pos.
__global__ void rle_emit_kernel(const uint32_t* __restrict__ a, int64_t n,
                                const int64_t* __restrict__ runid, int32_t* __restrict__ vid,
                                int64_t* __restrict__ start) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (i == 0 || a[i] != a[i - 1]) {
      vid[runid[i]] = (int32_t)a[i];
      start[runid[i]] = i;
    }
}

__global__ void rle_value_kernel(const int64_t* __restrict__ start, int64_t runs, int64_t n,
                                 int64_t n_walks, double* __restrict__ val) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < runs;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t end = r + 1 < runs ? start[r + 1] : n;
    val[r] = (double)(end - start[r]) / (double)n_walks;
  }
}

}  // namespace

int run_rand_hkpr(lgc_ctx* ctx, lgc_graph* g, int32_t x, const lgc_rand_hkpr_params* prm,
                  lgc_svec** p, lgc_stats* st_out) {
  int64_t dx = 0;
  LGC_TRY(validate_seed(ctx, g, x, &dx));
  const double t = prm->t;
  const int K = prm->K;
  const int64_t nw = prm->n_walks;
  if (!(t >= 0.0) || K < 0 || K > kMaxK || nw < 1 || nw > INT32_MAX) return LGC_EINVAL;
  // Poisson(t) CDF: term_0 = e^-t, term_{k+1} = term_k t / (k+1)
  CdfTable cdf;
  double term = exp(-t), acc = 0.0;
  for (int k = 0; k < kMaxK; k++) cdf.c[k] = 0.0;
  for (int k = 0; k < K; k++) {
    acc = acc + term;
    cdf.c[k] = acc;
    term = (term * t) / (double)(k + 1);
  }
  cudaStream_t s = ctx->stream;
  uint32_t *A = nullptr, *A2 = nullptr;
  int64_t *flag = nullptr, *runid = nullptr, *start = nullptr, *total = nullptr;
  int32_t* vid = nullptr;
  double* val = nullptr;
  int status = LGC_OK;
  lgc_stats st{};
  do {
    if ((status = dalloc_t(ctx, &A, nw)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &A2, nw)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &flag, nw)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &runid, nw)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &total, 2)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemsetAsync(total, 0, 16, s));
    int grid = grid_for(nw);
    if (grid > (ctx->sms * 64)) grid = (ctx->sms * 64);
    {
      // algorithmic bytes: 4 per walk (endpoint) now, 20 per step added below
      ProfScope ps(ctx, LGC_PROF_WALK, 4.0 * nw);
      walk_kernel<<<grid, kBlock, 0, s>>>(g->off, g->col, x, nw, K, cdf,
                                           (uint32_t)prm->rng_seed,
                                           (uint32_t)(prm->rng_seed >> 32), (int32_t*)A,
                                           (unsigned long long*)(total + 1));
      LGC_COUNT_LAUNCH(ctx);
    }
    LGC_CUDA_TRY(cudaGetLastError());
    const size_t walk_rec = ctx->prof_pending.size();
    if (ctx->trace) {
      if (ctx->d_endpoints) cudaFree(ctx->d_endpoints);
      ctx->d_endpoints = nullptr;
      LGC_CUDA_TRY(cudaMalloc((void**)&ctx->d_endpoints, 4 * nw));
      LGC_CUDA_TRY(cudaMemcpyAsync(ctx->d_endpoints, A, 4 * nw, cudaMemcpyDeviceToDevice, s));
      ctx->n_endpoints = nw;
    }
    if ((status = radix_sort_u32(ctx, A, A2, nw, bits_for(g->n))) != LGC_OK) break;
    rle_heads_kernel<<<grid_for(nw), kBlock, 0, s>>>(A, nw, flag);
    LGC_COUNT_LAUNCH(ctx);
    if ((status = scan_i64(ctx, flag, runid, nw, false, total)) != LGC_OK) break;
    LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, total, 16, cudaMemcpyDeviceToHost, s));
    LGC_CUDA_TRY(cudaStreamSynchronize(s));
    if ((status = sort_check(ctx)) != LGC_OK) break;
    const int64_t runs = ctx->h_scratch[0];
    st.pushed_edges = ctx->h_scratch[1];
    if (ctx->profile && walk_rec > 0 && walk_rec <= ctx->prof_pending.size())
      ctx->prof_pending[walk_rec - 1].bytes += 20.0 * (double)st.pushed_edges;
    if ((status = dalloc_t(ctx, &vid, runs)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &start, runs)) != LGC_OK) break;
    if ((status = dalloc_t(ctx, &val, runs)) != LGC_OK) break;
    rle_emit_kernel<<<grid_for(nw), kBlock, 0, s>>>(A, nw, runid, vid, start);
    LGC_COUNT_LAUNCH(ctx);
    rle_value_kernel<<<grid_for(runs), kBlock, 0, s>>>(start, runs, nw, nw, val);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    st.rounds = 1;
    st.pushes = nw;
    st.touched = runs;
    status = make_svec(ctx, vid, val, runs, ctx->result_on_device, p);
  } while (0);
  dfree(ctx, A);
  dfree(ctx, A2);
  dfree(ctx, flag);
  dfree(ctx, runid);
  dfree(ctx, start);
  dfree(ctx, total);
  dfree(ctx, vid);
  dfree(ctx, val);
  if (status == LGC_OK && st_out) *st_out = st;
  return status;
}

}  // namespace lgc

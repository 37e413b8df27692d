// lgc_sweep_noalloc: the sweep cut (same result as lgc_sweep) for callers
// that cannot allocate device memory during the call.
//
// Who needs it: a caller whose process hands all device memory to its own
// allocator up front (a serving process that reserved the GPU's memory, an
// embedded runtime with a fixed budget) cannot let a library call
// cudaMalloc, and a latency-critical caller cannot afford an allocation that
// may fail with out-of-memory or synchronize the device mid-request.  This
// entry point makes no allocation at all: every temporary buffer it needs is
// carved out of one file-scope device array of fixed size, held until the
// process exits.  With CUDA's lazy module loading (the default) the driver
// reserves that array on a device when this file's code is first used there
// -- the first lgc_sweep_noalloc call on the device -- so a caller that is
// about to hand the rest of the GPU's memory to its own allocator makes one
// call (an empty vector will do) before doing so.
//
// Limits and sharing:
//  * at most kMaxN = LGC_SWEEP_NOALLOC_MAX_N entries in the input vector
//    (larger inputs are rejected with LGC_EINVAL before any work is issued);
//    the scratch array is 5.6 MB on every device that loads the library;
//  * every call uses the same array; it keeps the previous call's contents,
//    so everything that must start at zero is cleared by the call itself;
//  * two calls that overlap on the GPU (on different streams, contexts or
//    host threads) race on the array and give wrong results: serialise them;
//  * the device address of the array is looked up once per device, on that
//    device's first call (cudaGetSymbolAddress with the device current); make
//    that first call before any stream capture.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "prim.cuh"

namespace lgc {
namespace {

constexpr int64_t kMaxN = LGC_SWEEP_NOALLOC_MAX_N;
constexpr int kTileItems = 8;
constexpr int kTileN = kBlock * kTileItems;                       // 2048 entries per sort tile
constexpr int64_t kMaxTiles = (kMaxN + kTileN - 1) / kTileN;      // 32
constexpr int64_t kSlots = 2 * kMaxN;                              // rank table, load <= 1/2
constexpr int kCrossTile = 1024;                                   // edges per crossing tile

// Scratch layout (bytes, every part 256-aligned).
constexpr size_t kOffKeyA = 0;
constexpr size_t kOffKeyB = kOffKeyA + 8 * kMaxN;
constexpr size_t kOffIdA = kOffKeyB + 8 * kMaxN;
constexpr size_t kOffIdB = kOffIdA + 4 * kMaxN;
constexpr size_t kOffDeg = kOffIdB + 4 * kMaxN;
constexpr size_t kOffVol = kOffDeg + 8 * kMaxN;
constexpr size_t kOffCut = kOffVol + 8 * kMaxN;
constexpr size_t kOffBefore = kOffCut + 8 * kMaxN;
constexpr size_t kOffSlots = kOffBefore + 4 * kMaxN;
constexpr size_t kOffHist = kOffSlots + 16 * kSlots;
constexpr size_t kOffPartial = kOffHist + 8 * 256 * kMaxTiles;
constexpr int64_t kPartial = 256;  // per-tile sums of a scan: ceil(8192 / 2048) or ceil(kMaxN / 2048)
constexpr size_t kOffMisc = kOffPartial + 8 * kPartial;
constexpr size_t kScratchBytes = kOffMisc + 256;

// The scratch memory: device-resident for the life of the process.  In host
// code its name is only a stand-in for the symbol, not a device address; the
// address is obtained with cudaGetSymbolAddress (scratch_base below).
static __device__ __align__(256) unsigned char g_sweep_scratch[kScratchBytes];

struct Misc {  // at kOffMisc
  unsigned long long npos;
  int bad;
  int err;
  int64_t best_i, best_cut, best_den, best_vol;
};

struct Scratch {
  uint64_t *keyA, *keyB;
  int32_t *idA, *idB;
  int64_t *deg, *vol, *cut;
  int32_t* before;
  Slot* slots;
  int64_t* hist;
  int64_t* partial;
  Misc* misc;
};

Scratch carve(unsigned char* base) {
  Scratch s;
  s.keyA = (uint64_t*)(base + kOffKeyA);
  s.keyB = (uint64_t*)(base + kOffKeyB);
  s.idA = (int32_t*)(base + kOffIdA);
  s.idB = (int32_t*)(base + kOffIdB);
  s.deg = (int64_t*)(base + kOffDeg);
  s.vol = (int64_t*)(base + kOffVol);
  s.cut = (int64_t*)(base + kOffCut);
  s.before = (int32_t*)(base + kOffBefore);
  s.slots = (Slot*)(base + kOffSlots);
  s.hist = (int64_t*)(base + kOffHist);
  s.partial = (int64_t*)(base + kOffPartial);
  s.misc = (Misc*)(base + kOffMisc);
  return s;
}

// Device address of the scratch array on the current device, looked up once
// per device.
int scratch_base(int device, unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[128] = {};
  if (device < 0 || device >= 128) return LGC_EINVAL;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sweep_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return LGC_ECUDA;
    }
    addr[device] = (unsigned char*)p;
  }
  *out = addr[device];
  return LGC_OK;
}

// S1: keys (non-increasing p/d becomes ascending key), entry validation.
__global__ void na_keys_kernel(const int32_t* __restrict__ idx, const double* __restrict__ val,
                               int64_t n0, const int32_t* __restrict__ deg, int64_t n, Scratch S) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n0;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = idx[i];
    double pv = val[i];
    if (v < 0 || v >= n || deg[v] < 1) {
      atomicOr(&S.misc->bad, 1);
      v = 0;
      pv = 0.0;
    }
    uint64_t k = ~0ull;
    if (pv > 0.0) {
      k = 0x7FFFFFFFFFFFFFFFull - (uint64_t)__double_as_longlong(pv / (double)deg[v]);
      c++;
    }
    S.keyA[i] = k;
    S.idA[i] = v;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&S.misc->npos, c);
}

// S3/S4: rank table and degrees in sweep order.
__global__ void na_rank_kernel(const int32_t* __restrict__ order, int64_t N, Table T,
                               const int32_t* __restrict__ deg, Scratch S) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int ins = 0;
    const int64_t s = ht_find_or_insert(T, order[i], &ins, &S.misc->err);
    if (s >= 0 && !ins) atomicOr(&S.misc->bad, 1);  // a vertex named twice
    if (s >= 0) T.s[s].aux = (int32_t)(i + 1);
    S.deg[i] = deg[order[i]];
  }
}

// S5: for every vertex v_i, the neighbours ranked before it; edge-balanced
// over the vol(S_N) edges (no per-edge scratch).
__global__ void __launch_bounds__(kBlock)
    na_cross_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                    const int32_t* __restrict__ order, int64_t N, int64_t V, Table T,
                    Scratch S) {
  __shared__ int64_t s_vol[kCrossTile];
  __shared__ int64_t s_off[kCrossTile];
  __shared__ int32_t s_cnt[kCrossTile];
  __shared__ int64_t s_i0, s_i1;
  const int64_t ntiles = (V + kCrossTile - 1) / kCrossTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * kCrossTile, e1 = min(V, e0 + kCrossTile);
    if (threadIdx.x == 0 || threadIdx.x == 32) {
      const int64_t x = threadIdx.x == 0 ? e0 : e1 - 1;
      int64_t lo = 0, hi = N;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (S.vol[mid] <= x) lo = mid + 1;
        else hi = mid;
      }
      if (threadIdx.x == 0) s_i0 = lo;
      else s_i1 = lo;
    }
    __syncthreads();
    const int64_t i0 = s_i0;
    int cnt = (int)(s_i1 - i0 + 1);
    if (cnt > kCrossTile) cnt = kCrossTile;
    for (int j = threadIdx.x; j < cnt; j += kBlock) {
      s_vol[j] = S.vol[i0 + j];
      s_off[j] = off[order[i0 + j]];
      s_cnt[j] = 0;
    }
    __syncthreads();
    for (int k = 0; k < kCrossTile / kBlock; k++) {
      const int64_t e = e0 + (int64_t)k * kBlock + threadIdx.x;
      if (e >= e1) continue;
      int lo = 0, hi = cnt;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_vol[mid] <= e) lo = mid + 1;
        else hi = mid;
      }
      const int j = lo;
      if (j >= cnt) continue;
      const int64_t first = j > 0 ? s_vol[j - 1] : (i0 > 0 ? S.vol[i0 - 1] : 0);
      const int64_t s = ht_find(T, col[s_off[j] + (e - first)]);
      const int64_t rw = s >= 0 ? T.s[s].aux : N + 1;
      if (rw < i0 + j + 1) atomicAdd(&s_cnt[j], 1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kBlock)
      if (s_cnt[j]) atomicAdd(&S.before[i0 + j], s_cnt[j]);
    __syncthreads();
  }
}

__global__ void na_delta_kernel(int64_t N, Scratch S) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    S.cut[i] = S.deg[i] - 2 * (int64_t)S.before[i];
}

// S7: exact argmin of cut_i / min(vol_i, 2m - vol_i), first index on ties,
// by one block; also copies the chosen prefix into the caller's buffer.
__global__ void na_argmin_kernel(int64_t N, int64_t two_m, Scratch S, int32_t* __restrict__ ids) {
  __shared__ int64_t sc[1024], sd[1024], si[1024];
  int64_t bc = 0, bd = 0, bi = -1;
  auto better = [](int64_t c1, int64_t d1, int64_t i1, int64_t c2, int64_t d2, int64_t i2) {
    if (i1 < 0) return false;
    if (i2 < 0) return true;
    const uint64_t lh = __umul64hi((uint64_t)c1, (uint64_t)d2), ll = (uint64_t)c1 * (uint64_t)d2;
    const uint64_t rh = __umul64hi((uint64_t)c2, (uint64_t)d1), rl = (uint64_t)c2 * (uint64_t)d1;
    if (lh != rh) return lh < rh;
    if (ll != rl) return ll < rl;
    return i1 < i2;
  };
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const int64_t v = S.vol[i];
    const int64_t den = v < two_m - v ? v : two_m - v;
    if (den > 0 && better(S.cut[i], den, i, bc, bd, bi)) {
      bc = S.cut[i];
      bd = den;
      bi = i;
    }
  }
  sc[threadIdx.x] = bc;
  sd[threadIdx.x] = bd;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o &&
        better(sc[threadIdx.x + o], sd[threadIdx.x + o], si[threadIdx.x + o], sc[threadIdx.x],
               sd[threadIdx.x], si[threadIdx.x])) {
      sc[threadIdx.x] = sc[threadIdx.x + o];
      sd[threadIdx.x] = sd[threadIdx.x + o];
      si[threadIdx.x] = si[threadIdx.x + o];
    }
    __syncthreads();
  }
  const int64_t best = si[0];
  if (threadIdx.x == 0) {
    S.misc->best_i = best;
    S.misc->best_cut = sc[0];
    S.misc->best_den = sd[0];
    S.misc->best_vol = best >= 0 ? S.vol[best] : 0;
  }
  for (int64_t i = threadIdx.x; i <= best; i += blockDim.x) ids[i] = S.idA[i];
}

}  // namespace
}  // namespace lgc

using namespace lgc;

extern "C" int lgc_sweep_noalloc(lgc_graph* g, int64_t nnz, const int32_t* d_idx,
                                 const double* d_val, int32_t* d_ids, lgc_cluster* out) {
  if (!g || !out || nnz < 0 || (nnz > 0 && (!d_idx || !d_val || !d_ids))) return LGC_EINVAL;
  if (nnz > kMaxN) return LGC_EINVAL;  // beyond the fixed scratch
  lgc_ctx* ctx = g->ctx;
  cudaStream_t st = ctx->stream;
  LGC_CUDA_TRY(cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  LGC_TRY(scratch_base(ctx->device, &base));
  const Scratch S = carve(base);
  out->size = 0;
  out->ids = d_ids;
  out->vol = 0;
  out->cut = 0;
  out->conductance = INFINITY;
  out->on_device = 1;
  LGC_CUDA_TRY(cudaMemsetAsync(S.misc, 0, sizeof(Misc), st));
  if (nnz == 0) return LGC_OK;
  // S1
  na_keys_kernel<<<(unsigned)((nnz + kBlock - 1) / kBlock), kBlock, 0, st>>>(
      d_idx, d_val, nnz, g->deg, g->n, S);
  // S2: stable LSD radix sort of (key, id), 8 passes of 8 bits, in the
  // scratch array (histograms and scan partials included)
  LGC_TRY(radix_sort_u64_i32_with(ctx, S.keyA, S.idA, S.keyB, S.idB, nnz, 64, S.hist,
                                  S.partial));
  LGC_CUDA_TRY(cudaGetLastError());
  Misc m;
  LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, S.misc, sizeof(Misc), cudaMemcpyDeviceToHost, st));
  LGC_CUDA_TRY(cudaStreamSynchronize(st));
  memcpy(&m, ctx->h_scratch, sizeof(Misc));
  if (m.bad) return LGC_EINVAL;  // an entry is not a vertex of degree >= 1
  const int64_t N = (int64_t)m.npos;
  if (N == 0) return LGC_OK;
  // S3, S4 (the table and the counters start at zero on every call)
  Table T;
  T.s = S.slots;
  T.cap = kSlots;
  int lg = 0;
  while (((int64_t)1 << lg) < kSlots) lg++;
  T.shift = 32 - lg;
  LGC_CUDA_TRY(cudaMemsetAsync(S.slots, 0, sizeof(Slot) * kSlots, st));
  LGC_CUDA_TRY(cudaMemsetAsync(S.before, 0, sizeof(int32_t) * N, st));
  na_rank_kernel<<<(unsigned)((N + kBlock - 1) / kBlock), kBlock, 0, st>>>(S.idA, N, T, g->deg, S);
  LGC_TRY(scan_i64_with(ctx, S.deg, S.vol, N, true, nullptr, S.partial));
  LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, S.vol + N - 1, 8, cudaMemcpyDeviceToHost, st));
  LGC_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t V = ctx->h_scratch[0];
  // S5, S6
  if (V > 0) {
    int64_t tiles = (V + kCrossTile - 1) / kCrossTile;
    const int64_t cap = (int64_t)ctx->sms * 8;
    na_cross_kernel<<<(unsigned)(tiles < cap ? tiles : cap), kBlock, 0, st>>>(
        g->off, g->col, S.idA, N, V, T, S);
  }
  na_delta_kernel<<<(unsigned)((N + kBlock - 1) / kBlock), kBlock, 0, st>>>(N, S);
  LGC_TRY(scan_i64_with(ctx, S.cut, S.cut, N, true, nullptr, S.partial));
  // S7
  na_argmin_kernel<<<1, 1024, 0, st>>>(N, g->nnz, S, d_ids);
  LGC_CUDA_TRY(cudaGetLastError());
  LGC_CUDA_TRY(cudaMemcpyAsync(ctx->h_scratch, S.misc, sizeof(Misc), cudaMemcpyDeviceToHost, st));
  LGC_CUDA_TRY(cudaStreamSynchronize(st));
  memcpy(&m, ctx->h_scratch, sizeof(Misc));
  if (m.bad) return LGC_EINVAL;  // a vertex named twice (as lgc_sweep)
  if (m.err) return LGC_ETABLEFULL;
  if (m.best_i >= 0) {
    out->size = m.best_i + 1;
    out->vol = m.best_vol;
    out->cut = m.best_cut;
    out->conductance = (double)m.best_cut / (double)m.best_den;
  }
  return LGC_OK;
}

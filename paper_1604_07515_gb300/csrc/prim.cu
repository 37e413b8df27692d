// Prefix sums and LSD radix sort, written for sm_103a.
#include <algorithm>

#include "lookback.cuh"
#include "prim.cuh"

namespace lgc {

namespace {

constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;  // 2048

// Inclusive block-wide scan of one int64 per thread; returns the inclusive
// value and the block total.
__device__ inline int64_t block_inclusive_scan(int64_t x, int64_t* warp_tot, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < (kBlock / 32) ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kBlock / 32)) warp_tot[lane] = w;
  }
  __syncthreads();
  int64_t offset = warp > 0 ? warp_tot[warp - 1] : 0;
  *total = warp_tot[kBlock / 32 - 1];
  __syncthreads();
  return x + offset;
}

__global__ void scan_reduce_kernel(const int64_t* __restrict__ in, int64_t n,
                                   int64_t* __restrict__ partial) {
  __shared__ int64_t warp_tot[kBlock / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) s += in[i];
  }
  int64_t tot;
  block_inclusive_scan(s, warp_tot, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Scans one tile, starting from offsets[blockIdx.x] (an exclusive block
// prefix), or, with tile_sums set, from the sum of offsets[0, blockIdx.x)
// (the tiles' own sums: one launch fewer when there are few tiles), or 0.
__global__ void scan_tile_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                 int64_t n, const int64_t* __restrict__ offsets, int inclusive,
                                 int64_t* __restrict__ total, int tile_sums) {
  __shared__ int64_t tile[kScanTile];
  __shared__ int64_t warp_tot[kBlock / 32];
  __shared__ int64_t pre_tot[kBlock / 32];
  int64_t pre = 0;
  if (offsets && tile_sums) {
    int64_t part = 0;
    for (int64_t j = threadIdx.x; j < (int64_t)blockIdx.x; j += blockDim.x) part += offsets[j];
    block_inclusive_scan(part, pre_tot, &pre);
  } else if (offsets) {
    pre = offsets[blockIdx.x];
  }
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    tile[k * kBlock + threadIdx.x] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; k++) {
    v[k] = tile[threadIdx.x * kScanItems + k];
    s += v[k];
  }
  int64_t tot;
  int64_t incl = block_inclusive_scan(s, warp_tot, &tot);
  int64_t run = incl - s + pre;
  for (int k = 0; k < kScanItems; k++) {
    int64_t x = v[k];
    tile[threadIdx.x * kScanItems + k] = inclusive ? run + x : run;
    run += x;
  }
  __syncthreads();
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) out[i] = tile[k * kBlock + threadIdx.x];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kBlock - 1) {
    // last element's inclusive value = grand total
    *total = run;
  }
}

__global__ void write_zero_kernel(int64_t* p) { *p = 0; }

}  // namespace

int grid_for(int64_t work, int block) {
  int64_t g = ceil_div(work, block);
  if (g < 1) g = 1;
  if (g > (1ll << 30)) g = 1ll << 30;
  return (int)g;
}

int bits_for(int64_t max_value) {
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) < max_value) b++;
  return b < 1 ? 1 : b;
}

int scan_lb(lgc_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, bool inclusive,
            int64_t* total);

int scan_i64_with(lgc_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, bool inclusive,
                  int64_t* total, int64_t* partial_scratch) {
  cudaStream_t st = ctx->stream;
  if (n <= 0) {
    if (total) {
      write_zero_kernel<<<1, 1, 0, st>>>(total);
      LGC_COUNT_LAUNCH(ctx);
    }
    return LGC_OK;
  }
  int64_t nb = ceil_div(n, kScanTile);
  if (nb == 1) {
    scan_tile_kernel<<<1, kBlock, 0, st>>>(in, out, n, nullptr, inclusive, total, 0);
    LGC_COUNT_LAUNCH(ctx);
    LGC_CUDA_TRY(cudaGetLastError());
    return LGC_OK;
  }
  if (!partial_scratch) return scan_lb(ctx, in, out, n, inclusive, total);
  int64_t* partial = partial_scratch;
  if (partial_scratch && nb > kScanTile) return LGC_EINVAL;  // the caller's scratch is one level
  if (!partial) LGC_TRY(dalloc_t(ctx, &partial, nb));
  scan_reduce_kernel<<<(unsigned)nb, kBlock, 0, st>>>(in, n, partial);
  LGC_COUNT_LAUNCH(ctx);
  LGC_CUDA_TRY(cudaGetLastError());
  // up to kScanTile tiles: each block sums the tile sums before its own
  // (at most kScanTile loads); beyond that the sums are scanned first
  const bool direct = nb <= kScanTile;
  int s = direct ? LGC_OK : scan_i64(ctx, partial, partial, nb, false, nullptr);
  if (s == LGC_OK) {
    scan_tile_kernel<<<(unsigned)nb, kBlock, 0, st>>>(in, out, n, partial, inclusive, total,
                                                      direct ? 1 : 0);
    LGC_COUNT_LAUNCH(ctx);
    if (cudaGetLastError() != cudaSuccess) s = LGC_ECUDA;
  }
  if (!partial_scratch) dfree(ctx, partial);
  return s;
}

int scan_i64(lgc_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, bool inclusive,
             int64_t* total) {
  return scan_i64_with(ctx, in, out, n, inclusive, total, nullptr);
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  Per pass: per-tile digit histograms, an
// exclusive scan over (digit, tile) in digit-major order, and a stable
// scatter.  Inside a tile each warp owns a contiguous run of 32 * kItems
// elements and ranks equal digits with __match_any_sync, so the order of
// equal keys is kept.
// ---------------------------------------------------------------------------
namespace {

constexpr int kItems = 8;
constexpr int kTile = kBlock * kItems;  // 2048
constexpr int kWarps = kBlock / 32;
constexpr int kRadix = 256;

template <class K>
__global__ void radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                                  int64_t* __restrict__ hist, int64_t ntiles) {
  __shared__ int h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kBlock) h[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int k = 0; k < kItems; k++) {
    int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & (K)0xFF)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kBlock)
    hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

template <class K, class V>
__global__ void radix_scatter_kernel(const K* __restrict__ keys_in, const V* __restrict__ vals_in,
                                     K* __restrict__ keys_out, V* __restrict__ vals_out,
                                     int64_t n, int shift, const int64_t* __restrict__ offs,
                                     int64_t ntiles, int has_vals) {
  __shared__ int wcnt[kWarps][kRadix];
  __shared__ int64_t goff[kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += kBlock) {
    goff[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    for (int w = 0; w < kWarps; w++) wcnt[w][d] = 0;
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * (32 * kItems);
  K key[kItems];
  V val[kItems];
  int rank[kItems];
  int digit[kItems];
  const unsigned lt = (1u << lane) - 1;
  for (int k = 0; k < kItems; k++) {
    int64_t i = base + (int64_t)k * 32 + lane;
    bool ok = i < n;
    key[k] = ok ? keys_in[i] : (K)0;
    if (has_vals) val[k] = ok ? vals_in[i] : V();
    int d = ok ? (int)((key[k] >> shift) & (K)0xFF) : kRadix;  // kRadix = padding
    digit[k] = d;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int r = __popc(peers & lt);
    int before = d < kRadix ? wcnt[warp][d] : 0;
    __syncwarp();
    rank[k] = before + r;
    int leader = __ffs(peers) - 1;
    if (lane == leader && d < kRadix) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, per digit
  for (int d = threadIdx.x; d < kRadix; d += kBlock) {
    int run = 0;
    for (int w = 0; w < kWarps; w++) {
      int c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int k = 0; k < kItems; k++) {
    int d = digit[k];
    if (d < kRadix) {
      int64_t pos = goff[d] + wcnt[warp][d] + rank[k];
      keys_out[pos] = key[k];
      if (has_vals) vals_out[pos] = val[k];
    }
  }
}

// ---------------------------------------------------------------------------
// LSD radix sort with one launch per 8-bit digit, after the single-pass
// scheme of Adinets and Merrill ("Onesweep", 2022): one histogram launch
// counts every digit position of every key; each digit pass then takes
// tiles in the order its blocks start (a counter, so every earlier tile
// belongs to a block already running), ranks the tile's keys by digit in
// shared memory (warps own contiguous runs; __match_any_sync orders equal
// digits by lane, so equal keys keep their order), publishes the tile's
// count per digit, adds up the counts of the tiles before it by a
// decoupled look-back (a published inclusive prefix ends the walk), and
// writes the keys digit run by digit run.  A pass whose digit is the same
// in every key (the histogram shows it) is skipped; which buffer holds a
// pass's input follows from the histogram on the device.  The status words
// and their epochs are those of lookback.cuh (each pass its own epoch,
// 256 words per tile: one per digit).
// ---------------------------------------------------------------------------
constexpr int kOsItems = 8;
constexpr int kOsTile = kBlock * kOsItems;  // 2048 keys
constexpr int kOsLook = 8;  // status words loaded at once in the look-back
// histogram of 8 digit positions, 8 pass counters, the ticket counter
constexpr int64_t kSortAuxWords = 8 * 256 + 5;
static_assert(kBlock == kRadix, "one thread per digit");

// Counts of every digit position q < D of the keys into hist[q * 256 + d]
// (zeroed before).  A warp whose keys share a digit adds them at once.
template <class K>
__global__ void os_hist_kernel(const K* __restrict__ keys, int64_t n, int D,
                               unsigned long long* __restrict__ hist) {
  __shared__ uint32_t h[8 * kRadix];
  for (int i = threadIdx.x; i < 8 * kRadix; i += kBlock) h[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {  // uniform in the block
    const int64_t i = base + threadIdx.x;
    const bool ok = i < n;
    const K k = ok ? keys[i] : (K)0;
    const unsigned act = __ballot_sync(0xffffffffu, ok);  // lane 0 is in it if any lane is
    for (int q = 0; q < D; q++) {
      const int d = (int)((k >> (8 * q)) & (K)0xFF);
      const int d0 = __shfl_sync(0xffffffffu, d, 0);
      if (__all_sync(0xffffffffu, !ok || d == d0)) {
        if (lane == 0 && act) atomicAdd(&h[q * kRadix + d0], (uint32_t)__popc(act));
      } else if (ok) {
        atomicAdd(&h[q * kRadix + d], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < D * kRadix; i += kBlock)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// Whether digit pass q is skipped: one digit holds all n keys.  Called by
// every thread of the block (thread t reads digit t).
__device__ inline bool os_trivial(const unsigned long long* hist, int q, int64_t n) {
  return __syncthreads_or(hist[q * kRadix + threadIdx.x] == (unsigned long long)n) != 0;
}

template <class K, class V>
__global__ void __launch_bounds__(kBlock)
    os_pass_kernel(K* keys0, V* vals0, K* keys1, V* vals1, int64_t n, int pass,
                   const unsigned long long* __restrict__ hist, unsigned int* ctr,
                   unsigned long long* status, uint32_t epoch, int* err, int has_vals) {
  __shared__ int wcnt[kWarps][kRadix];
  __shared__ int bstart[kRadix];
  __shared__ unsigned long long gbase[kRadix];
  __shared__ int64_t s_red[kBlock / 32];
  __shared__ K skey[kOsTile];
  __shared__ V sval[kOsTile];
  __shared__ int64_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the pass's input buffer: one swap per pass before it that was not skipped
  int swaps = 0;
  for (int q = 0; q < pass; q++) swaps += os_trivial(hist, q, n) ? 0 : 1;
  if (os_trivial(hist, pass, n)) return;  // the same in every block
  const K* kin = (swaps & 1) ? keys1 : keys0;
  const V* vin = (swaps & 1) ? vals1 : vals0;
  K* kout = (swaps & 1) ? keys0 : keys1;
  V* vout = (swaps & 1) ? vals0 : vals1;
  if (tid == 0) s_tile = (int64_t)atomicAdd(&ctr[pass], 1u);
  for (int w = 0; w < kWarps; w++) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile >= (int64_t)gridDim.x) return;  // cannot happen: the counter is cleared per sort
  const int shift = 8 * pass;
  // rank: warp w owns keys [w * 32 kOsItems, (w + 1) * 32 kOsItems) of the tile
  const int64_t base = tile * kOsTile + (int64_t)warp * (32 * kOsItems);
  K key[kOsItems];
  V val[kOsItems];
  int dr[kOsItems];  // digit (kRadix: padding) | rank within the warp's run << 9
  const unsigned lt = (1u << lane) - 1;
#pragma unroll
  for (int k = 0; k < kOsItems; k++) {
    const int64_t i = base + (int64_t)k * 32 + lane;
    const bool ok = i < n;
    key[k] = ok ? kin[i] : (K)0;
    if (has_vals) val[k] = ok ? vin[i] : V();
  }
#pragma unroll
  for (int k = 0; k < kOsItems; k++) {
    const int64_t i = base + (int64_t)k * 32 + lane;
    const int d = i < n ? (int)((key[k] >> shift) & (K)0xFF) : kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = d < kRadix ? wcnt[warp][d] : 0;
    __syncwarp();
    dr[k] = d | ((before + __popc(peers & lt)) << 9);
    if (lane == __ffs(peers) - 1 && d < kRadix) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread d: the digit's prefix over warps, the tile's count, published
  const int d = tid;
  int cnt = 0;
  for (int w = 0; w < kWarps; w++) {
    const int c = wcnt[w][d];
    wcnt[w][d] = cnt;
    cnt += c;
  }
  volatile unsigned long long* st = status + tile * kRadix + d;
  *st = lb_word(epoch, tile == 0 ? kLbInclusive : kLbAggregate, (uint64_t)cnt);
  int64_t tot;
  bstart[d] = (int)(block_inclusive_scan(cnt, s_red, &tot) - cnt);
  const int64_t h = (int64_t)hist[pass * kRadix + d];
  const int64_t gofs = block_inclusive_scan(h, s_red, &tot) - h;
  // look-back: the counts of this digit in the tiles before this one, the
  // words of kOsLook tiles loaded at once (tile 0 is always inclusive)
  uint64_t excl = 0;
  if (tile > 0) {
    bool done = false;
    for (int64_t j = tile - 1; !done; j -= kOsLook) {
      uint64_t w[kOsLook];
#pragma unroll
      for (int i = 0; i < kOsLook; i++)
        w[i] = j - i >= 0 ? ((const volatile unsigned long long*)status)[(j - i) * kRadix + d]
                          : lb_word(epoch, kLbInclusive, 0);
#pragma unroll
      for (int i = 0; i < kOsLook; i++) {
        if (done) break;
        const volatile unsigned long long* pj = status + (j - i) * kRadix + d;
        for (int spins = 0; (uint32_t)(w[i] >> 40) != epoch; w[i] = *pj) {
          if (++spins > kLbSpinLimit) {
            atomicOr(err, 1);
            w[i] = lb_word(epoch, kLbInclusive, 0);
            break;
          }
          if (spins > 16) __nanosleep(64);
        }
        excl += w[i] & kLbValue;
        done = (w[i] & kLbInclusive) != 0;
      }
    }
    *st = lb_word(epoch, kLbInclusive, excl + (uint64_t)cnt);
  }
  gbase[d] = (unsigned long long)gofs + excl;
  __syncthreads();
  // the tile in digit order in shared memory, then out run by run
#pragma unroll
  for (int k = 0; k < kOsItems; k++) {
    const int dk = dr[k] & 0x1FF;
    if (dk < kRadix) {
      const int lp = bstart[dk] + wcnt[warp][dk] + (dr[k] >> 9);
      skey[lp] = key[k];
      if (has_vals) sval[lp] = val[k];
    }
  }
  __syncthreads();
  const int64_t left = n - tile * kOsTile;
  const int tcount = left < kOsTile ? (int)left : kOsTile;
  for (int i = tid; i < tcount; i += kBlock) {
    const K kk = skey[i];
    const int dk = (int)((kk >> shift) & (K)0xFF);
    const unsigned long long pos = gbase[dk] + (unsigned long long)(i - bstart[dk]);
    kout[pos] = kk;
    if (has_vals) vout[pos] = sval[i];
  }
}

// ---------------------------------------------------------------------------
// One-launch prefix sum: tiles of kScanTile elements in start order (a
// ticket); each tile publishes its sum and finds its prefix by a decoupled
// look-back over the earlier tiles' words.  Sums travel as 38-bit two's
// complement: a partial sum outside [-2^37, 2^37) is recorded in *err.
// ---------------------------------------------------------------------------
__device__ inline bool lb_fits(int64_t x) {
  return x >= -(int64_t{1} << 37) && x < (int64_t{1} << 37);
}

__global__ void __launch_bounds__(kBlock)
    scan_lb_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                   int64_t ntiles, int inclusive, int64_t* __restrict__ total,
                   unsigned long long* ticket, unsigned long long ticket0,
                   unsigned long long* status, uint32_t epoch, int* err) {
  __shared__ int64_t tile[kScanTile];
  __shared__ int64_t warp_tot[kBlock / 32];
  __shared__ int64_t s_t, s_pre;
  if (threadIdx.x == 0) s_t = (int64_t)(atomicAdd(ticket, 1ull) - ticket0);
  __syncthreads();
  const int64_t t = s_t;
  if (t < 0 || t >= ntiles) {  // a ticket count out of step with the host's: flagged
    if (threadIdx.x == 0) atomicOr(err, 4);
    return;
  }
  const int64_t base = t * kScanTile;
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    tile[k * kBlock + threadIdx.x] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; k++) {
    v[k] = tile[threadIdx.x * kScanItems + k];
    s += v[k];
  }
  int64_t tot;
  const int64_t incl = block_inclusive_scan(s, warp_tot, &tot);
  if (threadIdx.x < 32) {
    volatile unsigned long long* st = status + t;
    if (threadIdx.x == 0)
      *st = lb_word(epoch, t == 0 ? kLbInclusive : kLbAggregate, (uint64_t)tot & kLbValue);
    const int64_t excl = lookback_warp(status, t, epoch, err);
    if (threadIdx.x == 0) {
      if (t > 0) *st = lb_word(epoch, kLbInclusive, (uint64_t)(excl + tot) & kLbValue);
      if (!lb_fits(tot) || !lb_fits(excl + tot)) atomicOr(err, 2);
      s_pre = excl;
    }
  }
  __syncthreads();
  int64_t run = incl - s + s_pre;
  for (int k = 0; k < kScanItems; k++) {
    const int64_t x = v[k];
    tile[threadIdx.x * kScanItems + k] = inclusive ? run + x : run;
    run += x;
  }
  __syncthreads();
  for (int k = 0; k < kScanItems; k++) {
    const int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) out[i] = tile[k * kBlock + threadIdx.x];
  }
  if (total && t == ntiles - 1 && threadIdx.x == kBlock - 1) *total = run;
}

// After D passes: an odd number of them not skipped left the result in the
// second buffers; copy it back.
template <class K, class V>
__global__ void os_final_kernel(K* keys0, V* vals0, const K* keys1, const V* vals1, int64_t n,
                                int D, const unsigned long long* __restrict__ hist,
                                int has_vals) {
  int swaps = 0;
  for (int q = 0; q < D; q++) swaps += os_trivial(hist, q, n) ? 0 : 1;
  if (!(swaps & 1)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys0[i] = keys1[i];
    if (has_vals) vals0[i] = vals1[i];
  }
}

// Short arrays: one CTA sorts (key masked to its low bits, original index)
// pairs in shared memory with a bitonic network; ordering by the index among
// equal keys makes it stable, so the result is the LSD radix sort's.
constexpr int kSmallSort = 1024;

template <class K, class V>
__global__ void __launch_bounds__(kSmallSort)
    small_sort_kernel(K* keys, V* vals, int n, K mask, int has_vals) {
  __shared__ K sk[kSmallSort];   // sort keys, permuted by the network
  __shared__ uint16_t si[kSmallSort];
  __shared__ K kf[kSmallSort];   // full keys, in input order
  __shared__ V sv[kSmallSort];   // values, in input order
  const int t = threadIdx.x;
  int N = 1;
  while (N < n) N <<= 1;
  if (t < N) {
    if (t < n) {
      const K k = keys[t];
      kf[t] = k;
      sk[t] = k & mask;
      if (has_vals) sv[t] = vals[t];
    } else {
      sk[t] = ~(K)0;  // padding sorts after every real key (larger index on ties)
    }
    si[t] = (uint16_t)t;
  }
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      __syncthreads();
      const int q = t ^ j;
      if (t < N && q > t) {
        const bool up = (t & k) == 0;
        const K a = sk[t], b = sk[q];
        const uint16_t ia = si[t], ib = si[q];
        const bool gt = a > b || (a == b && ia > ib);
        if (gt == up) {
          sk[t] = b;
          sk[q] = a;
          si[t] = ib;
          si[q] = ia;
        }
      }
    }
  }
  __syncthreads();
  if (t < n) {
    keys[t] = kf[si[t]];
    if (has_vals) vals[t] = sv[si[t]];
  }
}

// Room for `words` status words and `epochs` fresh epochs in the context's
// status array (cleared when it grows or the epochs would wrap), and its
// auxiliary block.
int status_reserve(lgc_ctx* ctx, int64_t words, int epochs) {
  if (words > ctx->sort_status_cap || ctx->sort_epoch + (uint32_t)epochs >= (1u << 24)) {
    if (words > ctx->sort_status_cap) {
      const int64_t cap = std::max<int64_t>(words, 2 * ctx->sort_status_cap);
      dfree(ctx, ctx->sort_status);
      ctx->sort_status = nullptr;
      ctx->sort_status_cap = 0;
      LGC_TRY(dalloc_t(ctx, &ctx->sort_status, (size_t)cap));
      ctx->sort_status_cap = cap;
    }
    LGC_CUDA_TRY(cudaMemsetAsync(ctx->sort_status, 0, 8 * ctx->sort_status_cap, ctx->stream));
    ctx->sort_epoch = 0;
  }
  if (!ctx->sort_aux) {
    LGC_TRY(dalloc_t(ctx, &ctx->sort_aux, kSortAuxWords));
    LGC_CUDA_TRY(cudaMemsetAsync(ctx->sort_aux, 0, 8 * kSortAuxWords, ctx->stream));
    ctx->lb_ticket = 0;
  }
  return LGC_OK;
}

// The running ticket counter of the one-launch scans and compactions: every
// block of such a launch takes one ticket, so the launch's tiles are the
// tickets [ctx->lb_ticket, ctx->lb_ticket + blocks), in the order the blocks
// start (no clearing between launches).
unsigned long long* lb_counter(lgc_ctx* ctx) { return ctx->sort_aux + 8 * kRadix + 4; }

// The one-launch-per-digit sort with the context's status array and epochs.
template <class K, class V>
int onesweep_sort(lgc_ctx* ctx, K* keys, V* vals, K* keys_tmp, V* vals_tmp, int64_t n,
                  int bits) {
  cudaStream_t st = ctx->stream;
  const int D = (bits + 7) / 8;
  const int64_t ntiles = ceil_div(n, kOsTile);
  LGC_TRY(status_reserve(ctx, ntiles * kRadix, D));
  unsigned long long* hist = ctx->sort_aux;                      // 8 * 256
  unsigned int* ctr = (unsigned int*)(ctx->sort_aux + 8 * kRadix);  // 8
  LGC_CUDA_TRY(cudaMemsetAsync(ctx->sort_aux, 0, 8 * (8 * kRadix + 4), st));
  const int hg = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kBlock), ctx->sms * 8));
  os_hist_kernel<K><<<hg, kBlock, 0, st>>>(keys, n, D, hist);
  LGC_COUNT_LAUNCH(ctx);
  for (int q = 0; q < D; q++) {
    os_pass_kernel<K, V><<<(unsigned)ntiles, kBlock, 0, st>>>(
        keys, vals, keys_tmp, vals_tmp, n, q, hist, ctr, ctx->sort_status, ++ctx->sort_epoch,
        ctx->d_sort_err, vals != nullptr);
    LGC_COUNT_LAUNCH(ctx);
  }
  os_final_kernel<K, V><<<hg, kBlock, 0, st>>>(keys, vals, keys_tmp, vals_tmp, n, D, hist,
                                               vals != nullptr);
  LGC_COUNT_LAUNCH(ctx);
  return cudaGetLastError() == cudaSuccess ? LGC_OK : LGC_ECUDA;
}

template <class K, class V>
int radix_sort_impl(lgc_ctx* ctx, K* keys, V* vals, K* keys_tmp, V* vals_tmp, int64_t n,
                    int bits, int64_t* hist_scratch = nullptr,
                    int64_t* partial_scratch = nullptr) {
  if (n <= 1) return LGC_OK;
  cudaStream_t st = ctx->stream;
  if (n <= kSmallSort) {
    const K mask = bits >= (int)(8 * sizeof(K)) ? ~(K)0 : (K)((((K)1) << bits) - 1);
    small_sort_kernel<K, V><<<1, kSmallSort, 0, st>>>(keys, vals, (int)n, mask,
                                                       vals != nullptr);
    LGC_COUNT_LAUNCH(ctx);
    return cudaGetLastError() == cudaSuccess ? LGC_OK : LGC_ECUDA;
  }
  // the caller's scratch (nothing may be allocated): the three-launch passes
  if (!hist_scratch) return onesweep_sort<K, V>(ctx, keys, vals, keys_tmp, vals_tmp, n, bits);
  const int64_t ntiles = ceil_div(n, kTile);
  int64_t* hist = hist_scratch;
  if (!hist) LGC_TRY(dalloc_t(ctx, &hist, (size_t)kRadix * ntiles));
  K* a = keys;
  V* va = vals;
  K* b = keys_tmp;
  V* vb = vals_tmp;
  int passes = 0;
  int status = LGC_OK;
  for (int shift = 0; shift < bits; shift += 8, passes++) {
    radix_hist_kernel<K><<<(unsigned)ntiles, kBlock, 0, st>>>(a, n, shift, hist, ntiles);
    LGC_COUNT_LAUNCH(ctx);
    status = scan_i64_with(ctx, hist, hist, (int64_t)kRadix * ntiles, false, nullptr,
                           partial_scratch);
    if (status != LGC_OK) break;
    radix_scatter_kernel<K, V><<<(unsigned)ntiles, kBlock, 0, st>>>(
        a, va, b, vb, n, shift, hist, ntiles, vals != nullptr);
    LGC_COUNT_LAUNCH(ctx);
    K* t = a;
    a = b;
    b = t;
    V* tv = va;
    va = vb;
    vb = tv;
  }
  if (status == LGC_OK && a != keys) {
    cudaMemcpyAsync(keys, a, sizeof(K) * n, cudaMemcpyDeviceToDevice, st);
    if (vals) cudaMemcpyAsync(vals, va, sizeof(V) * n, cudaMemcpyDeviceToDevice, st);
  }
  if (!hist_scratch) dfree(ctx, hist);
  if (status == LGC_OK && cudaGetLastError() != cudaSuccess) status = LGC_ECUDA;
  return status;
}

}  // namespace

int radix_sort_u32_f64(lgc_ctx* ctx, uint32_t* keys, double* vals, uint32_t* keys_tmp,
                       double* vals_tmp, int64_t n, int bits) {
  return radix_sort_impl<uint32_t, double>(ctx, keys, vals, keys_tmp, vals_tmp, n, bits);
}
int radix_sort_u64_f64(lgc_ctx* ctx, uint64_t* keys, double* vals, uint64_t* keys_tmp,
                       double* vals_tmp, int64_t n, int bits) {
  return radix_sort_impl<uint64_t, double>(ctx, keys, vals, keys_tmp, vals_tmp, n, bits);
}
int radix_sort_u64_i32(lgc_ctx* ctx, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                       int32_t* vals_tmp, int64_t n, int bits) {
  return radix_sort_impl<uint64_t, int32_t>(ctx, keys, vals, keys_tmp, vals_tmp, n, bits);
}
int radix_sort_u64_i32_with(lgc_ctx* ctx, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                            int32_t* vals_tmp, int64_t n, int bits, int64_t* hist,
                            int64_t* partial) {
  return radix_sort_impl<uint64_t, int32_t>(ctx, keys, vals, keys_tmp, vals_tmp, n, bits, hist,
                                            partial);
}
int radix_sort_u32_i32(lgc_ctx* ctx, uint32_t* keys, int32_t* vals, uint32_t* keys_tmp,
                       int32_t* vals_tmp, int64_t n, int bits) {
  return radix_sort_impl<uint32_t, int32_t>(ctx, keys, vals, keys_tmp, vals_tmp, n, bits);
}
int radix_sort_u32(lgc_ctx* ctx, uint32_t* keys, uint32_t* keys_tmp, int64_t n, int bits) {
  return radix_sort_impl<uint32_t, int32_t>(ctx, keys, (int32_t*)nullptr, keys_tmp,
                                            (int32_t*)nullptr, n, bits);
}

int lb_begin(lgc_ctx* ctx, int64_t ntiles, uint32_t* epoch, unsigned long long** ticket,
             unsigned long long* ticket0) {
  LGC_TRY(status_reserve(ctx, ntiles, 1));
  *epoch = ++ctx->sort_epoch;
  *ticket = lb_counter(ctx);
  *ticket0 = ctx->lb_ticket;
  return LGC_OK;
}

namespace {
struct BitsWord {
  const uint32_t* bits;
  __device__ uint32_t operator()(int64_t w) const { return bits[w]; }
};
}  // namespace

int bits_compact(lgc_ctx* ctx, const uint32_t* bits, int64_t words, const int32_t* deg,
                 int32_t* out_v, int32_t* out_s, int32_t cap, Counters* C) {
  if (words <= 0) return LGC_OK;
  const int64_t ntiles = ceil_div(words, kCmpTileWords);
  uint32_t epoch;
  unsigned long long *ticket, t0;
  LGC_TRY(lb_begin(ctx, ntiles, &epoch, &ticket, &t0));
  compact_words_kernel<BitsWord><<<(unsigned)ntiles, kBlock, 0, ctx->stream>>>(
      BitsWord{bits}, words, ntiles, deg, out_v, out_s, cap, ticket, t0, ctx->sort_status, epoch,
      ctx->d_sort_err, C);
  LGC_COUNT_LAUNCH(ctx);
  if (cudaGetLastError() != cudaSuccess) return LGC_ECUDA;  // not launched: no tickets taken
  lb_commit(ctx, ntiles);
  return LGC_OK;
}

// The multi-tile prefix sum in one launch (scan_lb_kernel).
int scan_lb(lgc_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, bool inclusive,
            int64_t* total) {
  const int64_t ntiles = ceil_div(n, kScanTile);
  LGC_TRY(status_reserve(ctx, ntiles, 1));
  scan_lb_kernel<<<(unsigned)ntiles, kBlock, 0, ctx->stream>>>(
      in, out, n, ntiles, inclusive ? 1 : 0, total, lb_counter(ctx), ctx->lb_ticket,
      ctx->sort_status, ++ctx->sort_epoch, ctx->d_sort_err);
  LGC_COUNT_LAUNCH(ctx);
  if (cudaGetLastError() != cudaSuccess) return LGC_ECUDA;  // not launched: no tickets taken
  ctx->lb_ticket += (uint64_t)ntiles;
  return LGC_OK;
}

}  // namespace lgc

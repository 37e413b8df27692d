// Decoupled look-back (Merrill and Garland's single-pass prefix scan): the
// status words the one-launch scans, sorts and compactions publish per tile,
// the warp-wide look-back over them, and the one-launch ordered compaction
// of a vertex bitmap (or of one computed word by word).
//
// A status word: epoch (24 bits) | state (2 bits: aggregate, inclusive
// prefix) | value (38 bits).  Every launch (every radix pass) has its own
// epoch, so the status array is cleared only when it is (re)allocated or the
// epochs wrap; a word of another epoch is "not yet published".  A look-back
// wait that exceeds kLbSpinLimit polls (it cannot, as every earlier tile's
// block is running) records the failure in *err and counts the tile as
// empty.
#pragma once

#include "common.cuh"

namespace lgc {

constexpr uint64_t kLbValue = (1ull << 38) - 1;
constexpr uint64_t kLbAggregate = 1ull << 38;
constexpr uint64_t kLbInclusive = 2ull << 38;
constexpr int kLbSpinLimit = 1 << 22;

__device__ inline uint64_t lb_word(uint32_t epoch, uint64_t state, uint64_t count) {
  return ((uint64_t)epoch << 40) | state | count;
}

// A value of a single-value status word: 38-bit two's complement.
__device__ inline int64_t lb_value(uint64_t w) { return (int64_t)(w << 26) >> 26; }

// Look-back by one whole warp for tiles with one status word each: the sum
// of the values of tiles [0, t), lane l reading tile j - l of a 32-tile
// window, the walk ending at the nearest inclusive word.  The warp waits
// until every word of the window is published (bounded: past kLbSpinLimit
// polls *err records it and unpublished words count as empty inclusive
// ones).  Every lane of the warp calls it and gets the sum.
__device__ inline int64_t lookback_warp(const unsigned long long* status, int64_t t,
                                        uint32_t epoch, int* err) {
  const int lane = threadIdx.x & 31;
  int64_t excl = 0;
  for (int64_t j = t - 1; j >= 0; j -= 32) {  // uniform in the warp
    const int64_t tj = j - lane;
    const volatile unsigned long long* pj = status + (tj >= 0 ? tj : 0);
    uint64_t w = tj >= 0 ? *pj : lb_word(epoch, kLbInclusive, 0);
    for (int spins = 0;; spins++) {
      const bool ready = (uint32_t)(w >> 40) == epoch;
      if (__all_sync(0xffffffffu, ready)) break;
      if (spins > kLbSpinLimit) {  // the same count in every lane
        if (lane == 0) atomicOr(err, 1);
        if (!ready) w = lb_word(epoch, kLbInclusive, 0);
        break;
      }
      if (spins > 16) __nanosleep(64);
      if (!ready) w = *pj;
    }
    const unsigned incl = __ballot_sync(0xffffffffu, (w & kLbInclusive) != 0);
    const int last = incl ? __ffs(incl) - 1 : 31;  // lanes 0..last count
    int64_t v = lane <= last ? lb_value(w) : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (incl) break;
  }
  return excl;
}

// ---------------------------------------------------------------------------
// Ordered compaction of a vertex bitmap in one launch.  The bitmap's words
// come from a functor (word(w): the set bits of word w, for w < words), so
// that a filter can compute them on the fly.  Tiles of
// kCmpTileWords words are taken in start order (a counter); warp w of a tile
// takes 32 * kCmpRounds consecutive words, 32 per round, lane l word l of
// the round; the tile's count goes to the status array and its offset comes
// from a decoupled look-back over the earlier tiles (one status word per
// tile, as in the sort).  A set bit's vertex is written at its position:
// a round's words are taken in turn, lane l writing bit l, so a warp's
// stores are consecutive.
// ---------------------------------------------------------------------------
constexpr int kCmpRounds = 1;
constexpr int64_t kCmpTileWords = (int64_t)kBlock * kCmpRounds;  // 256 words

template <class WordFn>
__global__ void __launch_bounds__(kBlock)
    compact_words_kernel(WordFn word, int64_t words, int64_t ntiles,
                        const int32_t* __restrict__ deg, int32_t* nfv, int32_t* nfs,
                        int32_t ncap, unsigned long long* ticket,
                        unsigned long long ticket0, unsigned long long* status, uint32_t epoch,
                        int* err, Counters* C) {
  __shared__ int64_t s_tile, s_base;
  __shared__ int s_wtot[kBlock / 32];
  __shared__ int64_t s_deg[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = (int64_t)(atomicAdd(ticket, 1ull) - ticket0);
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile < 0 || tile >= ntiles) {  // a ticket count out of step with the host's: flagged
    if (threadIdx.x == 0) atomicOr(err, 4);
    return;
  }
  const int64_t wbase = tile * kCmpTileWords + (int64_t)warp * (32 * kCmpRounds);
  uint32_t q[kCmpRounds];
  int pre[kCmpRounds];  // set bits before this lane's word in the warp's words
  int run = 0;
#pragma unroll
  for (int k = 0; k < kCmpRounds; k++) {
    const int64_t w = wbase + 32 * k + lane;
    q[k] = w < words ? word(w) : 0u;
    const int c = __popc(q[k]);
    int inc = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    pre[k] = run + inc - c;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) s_wtot[warp] = run;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t tot = 0;  // every lane of warp 0 sums the warps' counts
    for (int w = 0; w < kBlock / 32; w++) tot += s_wtot[w];
    __syncwarp();
    volatile unsigned long long* st = status + tile;
    if (threadIdx.x == 0) {
      int64_t run = 0;
      for (int w = 0; w < kBlock / 32; w++) {  // exclusive over warps
        const int c = s_wtot[w];
        s_wtot[w] = (int)run;
        run += c;
      }
      *st = lb_word(epoch, tile == 0 ? kLbInclusive : kLbAggregate, (uint64_t)tot);
    }
    const int64_t excl = lookback_warp(status, tile, epoch, err);
    if (threadIdx.x == 0) {
      if (tile > 0) *st = lb_word(epoch, kLbInclusive, (uint64_t)(excl + tot));
      s_base = excl;
      if (tile == ntiles - 1) C->next_size = (int32_t)(excl + tot);
    }
  }
  __syncthreads();
  const int64_t wb = s_base + s_wtot[warp];
  const uint32_t below = (1u << lane) - 1u;
  int64_t dsum = 0;
#pragma unroll
  for (int k = 0; k < kCmpRounds; k++) {
    if (!__any_sync(0xffffffffu, q[k] != 0u)) continue;
    for (int j0 = 0; j0 < 32; j0 += 8) {
      int32_t dk[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint32_t qj = __shfl_sync(0xffffffffu, q[k], j0 + j);
        const int pj = __shfl_sync(0xffffffffu, pre[k], j0 + j);
        dk[j] = 0;
        if ((qj >> lane) & 1u) {
          const int64_t v = (wbase + 32 * k + j0 + j) * 32 + lane;
          const int64_t at = wb + pj + __popc(qj & below);
          if (at < ncap) {
            nfv[at] = (int32_t)v;
            nfs[at] = (int32_t)v;
          } else {
            atomicOr(&C->err, kErrFrontierOverflow);
          }
          if (deg) dk[j] = deg[v];
        }
      }
#pragma unroll
      for (int j = 0; j < 8; j++) dsum += dk[j];
    }
  }
  if (deg) {
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lane == 0) s_deg[warp] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t t = 0;
      for (int w = 0; w < kBlock / 32; w++) t += s_deg[w];
      if (t) atomicAdd((unsigned long long*)&C->next_edges, (unsigned long long)t);
    }
  }
}

// The host side of a look-back launch over `ntiles` tiles: room in the
// context's status array, a fresh epoch, and the first ticket of the launch
// (lb_commit after a successful launch takes its tickets).
int lb_begin(lgc_ctx* ctx, int64_t ntiles, uint32_t* epoch, unsigned long long** ticket,
             unsigned long long* ticket0);
inline void lb_commit(lgc_ctx* ctx, int64_t ntiles) { ctx->lb_ticket += (uint64_t)ntiles; }

}  // namespace lgc

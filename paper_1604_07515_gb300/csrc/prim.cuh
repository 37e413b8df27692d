// Device-wide primitives: prefix sums and LSD radix sort (Sec. 2,
// "Parallel Primitives": prefix sum, filter, integer sort).
#pragma once

#include "common.cuh"

namespace lgc {

// out[i] = sum_{j < i} in[j] (exclusive) or sum_{j <= i} in[j] (inclusive),
// int64.  If total != nullptr, the sum of all n inputs is written to
// *total (device).  in and out may alias.
int scan_i64(lgc_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, bool inclusive,
             int64_t* total);
// As scan_i64 with the caller's scratch for the per-tile sums
// (partial_scratch: ceil(n / 2048) int64, n <= 2048 * 2048), so that nothing
// is allocated; partial_scratch == nullptr is scan_i64.
int scan_i64_with(lgc_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, bool inclusive,
                  int64_t* total, int64_t* partial_scratch);

// Stable LSD radix sort of (key, value) pairs by key bits [0, bits), 8 bits
// per pass.  keys/vals hold the input; the sorted result ends in keys/vals
// (the tmp buffers are scratch of the same length).
int radix_sort_u32_f64(lgc_ctx* ctx, uint32_t* keys, double* vals, uint32_t* keys_tmp,
                       double* vals_tmp, int64_t n, int bits);
int radix_sort_u64_f64(lgc_ctx* ctx, uint64_t* keys, double* vals, uint64_t* keys_tmp,
                       double* vals_tmp, int64_t n, int bits);
int radix_sort_u64_i32(lgc_ctx* ctx, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                       int32_t* vals_tmp, int64_t n, int bits);
int radix_sort_u32_i32(lgc_ctx* ctx, uint32_t* keys, int32_t* vals, uint32_t* keys_tmp,
                       int32_t* vals_tmp, int64_t n, int bits);
// As radix_sort_u64_i32 with the caller's scratch, allocating nothing: hist
// holds 256 * ceil(n / 2048) int64 and partial ceil(hist entries / 2048)
// int64 (hist entries <= 2048 * 2048).
int radix_sort_u64_i32_with(lgc_ctx* ctx, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                            int32_t* vals_tmp, int64_t n, int bits, int64_t* hist,
                            int64_t* partial);
// Keys only.
int radix_sort_u32(lgc_ctx* ctx, uint32_t* keys, uint32_t* keys_tmp, int64_t n, int bits);

// Ordered compaction of the n-bit vertex bitmap bits (words = ceil(n / 32))
// into out_v = out_s = the set vertices in ascending id, one launch: C's
// next_size becomes their number, and with deg their degrees are added to
// C's next_edges; positions past cap are not written and flag
// kErrFrontierOverflow in C's err.  C is device memory, zeroed by the caller
// as needed.
int bits_compact(lgc_ctx* ctx, const uint32_t* bits, int64_t words, const int32_t* deg,
                 int32_t* out_v, int32_t* out_s, int32_t cap, Counters* C);

int bits_for(int64_t max_value);  // number of bits needed for values < max_value

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int grid_for(int64_t work, int block = kBlock);

}  // namespace lgc

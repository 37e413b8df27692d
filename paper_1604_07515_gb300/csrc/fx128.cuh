// Exact sums of non-negative doubles in 128-bit fixed point.
//
// The gather of a pull round adds, for every vertex, the shares of its
// in-frontier neighbours (the edgeMap's r'[w] += share of Sec. 3.3, read in
// the pull direction).  GB300 issues FP64 adds at a small fraction of its
// integer rate, so the atomic mode does not add doubles per edge: each
// frontier share is converted once to an unsigned integer X with
// share = X * 2^L (L fixed for the round), the integers are summed with
// carries, and each vertex's total is rounded to double once (round to
// nearest, ties to even).
//
// L is the larger of
//   * the weight of the lowest mantissa bit of the smallest nonzero share, so
//     that every share is an integer multiple of 2^L, and
//   * the value that keeps any vertex's total below 2^127 (at most max_deg
//     terms, each below 2^(top bit of the largest share + 1)).
// When the first bound wins the sum is exact and the result is the correctly
// rounded sum; when the second wins (shares spanning more than ~2^56) the
// smallest shares lose bits below 2^L, at most max_share * 2^-(126 - G - 53)
// each.  Bit 127 is not part of the value: the pull encoding uses it to mark
// frontier membership (a member's share may be zero).
//
// Usable from host code too (the host test of the conversions compiles this
// header with a C++ compiler).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define LGC_HD __host__ __device__ __forceinline__
#else
#define LGC_HD inline
#endif

namespace lgc {

struct __align__(16) Fx {
  uint64_t lo;
  uint64_t hi;  // bit 63: membership flag, not value
};

constexpr uint64_t kFxFlag = 1ull << 63;
constexpr uint64_t kFxMask = ~kFxFlag;

LGC_HD int fx_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

LGC_HD uint64_t fx_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  __builtin_memcpy(&b, &x, 8);
  return b;
#endif
}

LGC_HD double fx_from_bits(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}

// Biased exponent field of a non-negative double's bits (0 for zero and
// subnormals).
LGC_HD int fx_bexp(uint64_t bits) { return (int)(bits >> 52) & 0x7ff; }

// Weight (power of two) of the lowest mantissa bit and one past the top
// possible bit of a positive finite double with biased exponent be:
// x = m * 2^lsb with m < 2^53, and x < 2^top.
LGC_HD int fx_lsb(int be) { return be ? be - 1075 : -1074; }
LGC_HD int fx_top(int be) { return be ? be - 1022 : -1022; }

// The round's scale from the smallest and largest biased exponents among the
// nonzero shares (be_min > be_max means there are none) and the bound on
// terms per sum, max_terms < 2^g.
LGC_HD int fx_scale(int be_min, int be_max, int g) {
  if (be_min > be_max) return 0;
  const int a = fx_lsb(be_min);
  const int b = fx_top(be_max) + g - 127;
  return a > b ? a : b;
}

// share (>= 0 or -0.0, finite) -> X = floor(share / 2^L); exact when
// L <= lsb(share).  X < 2^127 whenever L came from fx_scale over a set
// containing share.
LGC_HD Fx fx_from_double(double x, int L) {
  Fx r = {0, 0};
  const uint64_t bits = fx_bits(x) & kFxMask;  // -0.0 -> +0.0
  if (bits == 0) return r;
  const int be = fx_bexp(bits);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (be) m |= 1ull << 52;
  const int sh = fx_lsb(be) - L;
  if (sh >= 0) {
    if (sh >= 128) return r;  // cannot happen under fx_scale; keeps shifts defined
    if (sh >= 64) {
      r.hi = m << (sh - 64);
    } else {
      r.lo = m << sh;
      r.hi = sh ? m >> (64 - sh) : 0;
    }
  } else {
    const int rs = -sh;
    r.lo = rs >= 64 ? 0 : m >> rs;
  }
  return r;
}

// x << s and x >> s for every s < 2^32, zero once s >= 64: the PTX shifts
// clamp the shift amount to the register width; host code says so.
LGC_HD uint64_t fx_shl(uint64_t x, uint32_t s) {
#if defined(__CUDA_ARCH__)
  uint64_t r;
  asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
#else
  return s >= 64 ? 0 : x << s;
#endif
}
LGC_HD uint64_t fx_shr(uint64_t x, uint32_t s) {
#if defined(__CUDA_ARCH__)
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
#else
  return s >= 64 ? 0 : x >> s;
#endif
}

// fx_from_double of a share's bits without branches (the pull gathers
// convert one 8-byte share per edge).  With m the significand and
// sh = lsb - L, X = m * 2^sh: for 0 <= sh the low word is m << sh and the
// high word m >> (64 - sh) or m << (sh - 64); for sh < 0 the low word is
// m >> -sh.  Every out-of-range shift gives zero, so the four terms combine
// by OR (at sh = 0 and sh = 64 the two terms of a word are equal), and the
// result equals fx_from_double's for every input, sh >= 128 included.
LGC_HD Fx fx_from_bits(uint64_t bits, int L) {
  bits &= kFxMask;  // -0.0 -> +0.0
  const int be = fx_bexp(bits);
  const uint64_t m = (bits & ((1ull << 52) - 1)) | ((uint64_t)(be != 0) << 52);
  const int sh = fx_lsb(be) - L;
  Fx r;
  r.lo = fx_shl(m, (uint32_t)sh) | fx_shr(m, (uint32_t)(-sh));
  r.hi = fx_shr(m, (uint32_t)(64 - sh)) | fx_shl(m, (uint32_t)(sh - 64));
  return r;
}

// a += b over the 127 value bits (b's flag is dropped).
LGC_HD void fx_add(Fx& a, const Fx& b) {
  const uint64_t lo = a.lo + b.lo;
  a.hi += (b.hi & kFxMask) + (lo < b.lo ? 1ull : 0ull);
  a.lo = lo;
}

// RN(X * 2^L) as a double, X < 2^127 (the flag bit is ignored).
LGC_HD double fx_to_double(Fx X, int L) {
  const uint64_t hi = X.hi & kFxMask, lo = X.lo;
  if ((hi | lo) == 0) return 0.0;
  const int p = hi ? 127 - fx_clz64(hi) : 63 - fx_clz64(lo);  // top set bit
  // Right shift that leaves 53 significant bits, or fewer when the result
  // is subnormal (lowest kept bit of weight 2^-1074).
  int r = p - 52;
  if (-1074 - L > r) r = -1074 - L;
  uint64_t mant;
  if (r <= 0) {
    mant = lo << (-r);  // here p - r <= 52, so the value sits in lo
  } else {
    // q = X >> r, round bit = bit r-1, sticky = bits below it
    uint64_t qlo, rbit, sticky;
    if (r >= 128) {
      qlo = 0;
      rbit = 0;
      sticky = (hi | lo) != 0;
    } else if (r >= 64) {
      const int s = r - 64;
      qlo = hi >> s;
      rbit = s ? (hi >> (s - 1)) & 1 : lo >> 63;
      sticky = s ? ((hi & ((1ull << (s - 1)) - 1)) | lo) != 0
                 : (lo & ((1ull << 63) - 1)) != 0;
    } else {
      qlo = (lo >> r) | (r ? hi << (64 - r) : 0);  // at most 53 bits remain: hi >> r is zero
      rbit = (lo >> (r - 1)) & 1;
      sticky = r > 1 ? (lo & ((1ull << (r - 1)) - 1)) != 0 : 0;
    }
    mant = qlo;
    if (rbit && (sticky || (mant & 1))) mant++;
  }
  // value = mant * 2^(L + r); mant <= 2^53 with the carry of the rounding
  // moving into the exponent field (see the encoding of IEEE binary64).
  const int64_t e = (int64_t)L + r + 1074;
  if (e >= 2046 && mant >= (1ull << 52)) return fx_from_bits(0x7ffull << 52);  // +inf
  return fx_from_bits(((uint64_t)e << 52) + mant);
}

// ---------------------------------------------------------------------------
// The left fold acc <- RN(acc + s) of non-negative doubles, one binade at a
// time in integers (the deterministic pull gather).  While acc stays in the
// binade bu (bu >= 1; bu = 1 also holds zero and the subnormals),
// acc = A * u with u = 2^(bu-1075) and A < 2^53.  For s / u = Q + f with
// 0 <= f < 1, RN(acc + s) = (A + Q + [f > 1/2]) * u, except at f = 1/2 (a
// tie), where it is the even one of A + Q and A + Q + 1, provided the result
// stays below 2^53 * u.  A share is therefore a step A -> A + g[A & 1], and
// steps compose into steps of the same form.
// ---------------------------------------------------------------------------
struct FoldStep {
  int64_t g0, g1;
};

constexpr int64_t kFoldTop = int64_t{1} << 53;
constexpr int64_t kFoldBig = int64_t{1} << 54;  // a share that leaves the binade by itself

LGC_HD int fold_binade(double acc) {
  const int be = fx_bexp(fx_bits(acc) & kFxMask);
  return be > 1 ? be : 1;
}

// acc / u for acc in its own binade.
LGC_HD int64_t fold_int(double acc) {
  const uint64_t b = fx_bits(acc) & kFxMask;
  const uint64_t m = b & ((1ull << 52) - 1);
  return (int64_t)(fx_bexp(b) ? (m | (1ull << 52)) : m);
}

// A * u as a double (A < 2^53).
LGC_HD double fold_double(int64_t A, int bu) {
  return fx_from_bits(((uint64_t)(bu - 1) << 52) + (uint64_t)A);
}

LGC_HD FoldStep fold_step(double s, int bu) {
  const uint64_t b = fx_bits(s) & kFxMask;  // -0.0 adds nothing
  if (b == 0) return {0, 0};
  const int be = fx_bexp(b);
  uint64_t m = b & ((1ull << 52) - 1);
  if (be) m |= 1ull << 52;
  const int sh = fx_lsb(be) - (bu - 1075);
  if (sh >= 2) return {kFoldBig, kFoldBig};
  if (sh >= 0) {
    const int64_t Q = (int64_t)(m << sh);
    return {Q, Q};
  }
  const int rs = -sh;
  if (rs >= 64) return {0, 0};  // s < u / 2^10: rounds away
  const int64_t Q = (int64_t)(m >> rs);
  const uint64_t R = m & ((1ull << rs) - 1), half = 1ull << (rs - 1);
  if (R != half) {
    const int64_t D = Q + (R > half ? 1 : 0);
    return {D, D};
  }
  return {Q + (Q & 1), Q + ((Q + 1) & 1)};
}

// first a, then b
LGC_HD FoldStep fold_compose(FoldStep a, FoldStep b) {
  return {a.g0 + ((a.g0 & 1) ? b.g1 : b.g0), a.g1 + ((a.g1 & 1) ? b.g0 : b.g1)};
}

LGC_HD int64_t fold_apply(FoldStep f, int64_t A) { return A + ((A & 1) ? f.g1 : f.g0); }

}  // namespace lgc

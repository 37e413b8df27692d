// Host build of the fixed-point conversions used by the atomic pull gather
// (paper_1604_07515_gb300/csrc/fx128.cuh), exported for the host test.
#define __align__(n) alignas(n)
#include "../paper_1604_07515_gb300/csrc/fx128.cuh"

extern "C" {
int fxh_scale(int be_min, int be_max, int g) { return lgc::fx_scale(be_min, be_max, g); }
void fxh_from_double(double x, int L, uint64_t* lo, uint64_t* hi) {
  lgc::Fx r = lgc::fx_from_double(x, L);
  *lo = r.lo;
  *hi = r.hi;
}
void fxh_from_bits(double x, int L, uint64_t* lo, uint64_t* hi) {
  lgc::Fx r = lgc::fx_from_bits(lgc::fx_bits(x), L);
  *lo = r.lo;
  *hi = r.hi;
}
double fxh_to_double(uint64_t lo, uint64_t hi, int L) { return lgc::fx_to_double({lo, hi}, L); }
// Sum of n shares at the scale their range gives, rounded once.
double fxh_sum(const double* x, int n, int g, int* L_out) {
  int bmin = 2047, bmax = 0;
  for (int i = 0; i < n; i++) {
    uint64_t b;
    __builtin_memcpy(&b, &x[i], 8);
    b &= lgc::kFxMask;
    if (!b) continue;
    int be = lgc::fx_bexp(b);
    if (be < bmin) bmin = be;
    if (be > bmax) bmax = be;
  }
  int L = lgc::fx_scale(bmin, bmax, g);
  lgc::Fx acc = {0, 0};
  for (int i = 0; i < n; i++) lgc::fx_add(acc, lgc::fx_from_double(x[i], L));
  *L_out = L;
  return lgc::fx_to_double(acc, L);
}
}

// The deterministic gather's fold, emulating its warp (32 lanes of 8
// consecutive shares per batch of 256) sequentially: per-lane composed
// steps, an exclusive prefix over lanes, the first position leaving the
// binade redone in FP64, restart after it.
static double fold_batch_host(double acc, const double* v /*256*/) {
  using namespace lgc;
  int start = 0;
  while (start < 256) {
    const int bu = fold_binade(acc);
    const int64_t A0 = fold_int(acc);
    FoldStep st[256], F[32];
    for (int l = 0; l < 32; l++) {
      F[l] = {0, 0};
      for (int j = 0; j < 8; j++) {
        const int i = 8 * l + j;
        st[i] = i >= start ? fold_step(v[i], bu) : FoldStep{0, 0};
        F[l] = fold_compose(F[l], st[i]);
      }
    }
    FoldStep E = {0, 0};
    int cross = -1;
    int64_t before = 0, Aend = 0;
    for (int l = 0; l < 32; l++) {
      int64_t A = fold_apply(E, A0);
      for (int j = 0; j < 8; j++) {
        const int64_t nx = fold_apply(st[8 * l + j], A);
        if (cross < 0 && nx >= kFoldTop) {
          cross = 8 * l + j;
          before = A;
        }
        A = nx;
      }
      Aend = A;
      E = fold_compose(E, F[l]);
    }
    if (cross < 0) return fold_double(Aend, bu);
    acc = fold_double(before, bu) + v[cross];
    start = cross + 1;
  }
  return acc;
}

extern "C" {
// Fold of n shares from acc, batch by batch; *seq gets the plain FP64 fold.
double fxh_fold(double acc, const double* v, int n, double* seq) {
  double s = acc;
  for (int i = 0; i < n; i++) s = s + v[i];
  *seq = s;
  double buf[256];
  for (int b = 0; b < n; b += 256) {
    for (int i = 0; i < 256; i++) buf[i] = b + i < n ? v[b + i] : 0.0;
    acc = fold_batch_host(acc, buf);
  }
  return acc;
}
}

extern "C" {
// The deterministic gather's segment-parallel fold for long lists, emulated:
// per 256-share segment a plain sum, a running sum of them predicting the
// binade at each segment start, the segment's composed step for that
// binade, then the in-order walk that takes the step when the binade
// matches and the value stays below 2^53, and folds the segment element by
// element otherwise.  *redone counts the segments folded element by element.
double fxh_fold_segmented(double acc, const double* v, int n, int* redone) {
  using namespace lgc;
  const int nseg = (n + 255) / 256;
  double buf[256];
  double pacc = acc;
  int* pred = new int[nseg];
  FoldStep* st = new FoldStep[nseg];
  for (int k = 0; k < nseg; k++) {
    pred[k] = fold_binade(pacc);
    double s = 0.0;
    for (int i = 256 * k; i < n && i < 256 * k + 256; i++) s += v[i];
    pacc += s;
  }
  for (int k = 0; k < nseg; k++) {
    FoldStep F = {0, 0};
    for (int i = 256 * k; i < n && i < 256 * k + 256; i++)
      F = fold_compose(F, fold_step(v[i], pred[k]));
    st[k] = F;
  }
  *redone = 0;
  for (int k = 0; k < nseg; k++) {
    const int bu = fold_binade(acc);
    if (bu == pred[k]) {
      const int64_t A = fold_apply(st[k], fold_int(acc));
      if (A < kFoldTop) {
        acc = fold_double(A, bu);
        continue;
      }
    }
    (*redone)++;
    for (int i = 0; i < 256; i++) buf[i] = 256 * k + i < n ? v[256 * k + i] : 0.0;
    acc = fold_batch_host(acc, buf);
  }
  delete[] pred;
  delete[] st;
  return acc;
}
}

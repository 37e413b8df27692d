// Oracle for "Parallel Local Graph Clustering" (Shun, Roosta-Khorasani,
// Fountoulakis, Mahoney; arXiv:1604.07515).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
// restatement of the paper's algorithms.  It exists so that tests can check
// the CUDA library against it.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load it; the library never does.  It
// shares no code, header, table or constant generator with the CUDA path.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared (no FMA
// contraction, so every expression below is evaluated as written, with one
// IEEE round-to-nearest per operation).
//
// Conventions
//  * Graphs are undirected CSR: off[n+1] (int64), col[off[n]] (int32), each
//    adjacency list sorted ascending, no self loops, no duplicates (Sec. 2,
//    "Graph Notation"; Sec. 4, "Input Graphs").
//  * A sparse set (Sec. 2, "Sparse Sets") maps a vertex id to a double and
//    reads a missing key as 0.  Here it is a dense array plus a membership
//    flag and the list of keys that were created; the oracle does not need
//    locality, only the set semantics.
//  * Every frontier (vertexSubset) is iterated in ascending vertex id and
//    every adjacency list in stored (ascending) order.  So each destination
//    receives its contributions in ascending source order, starting from the
//    value it holds when the edgeMap begins.  This is the canonical
//    deterministic result the CUDA deterministic mode must reproduce bit for
//    bit.
//  * parity: PR-Nibble, Nibble, HK-PR and the sweep cut are pinned by the
//    CPU tests (dense linear-algebra closed forms, invariants, the paper's
//    worked sweep example, brute force).  The Philox4x32-10 words are pinned
//    to cuRAND's host-side Philox4x32-10 generator (a library routine) over
//    several keys and counters with words 0-2 in use, the words rand_hkpr
//    draws from, plus uniformity and avalanche checks.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <utility>
#include <vector>

namespace {

struct Graph {
  int64_t n;
  const int64_t* off;
  const int32_t* col;
  int64_t deg(int32_t v) const { return off[v + 1] - off[v]; }
  int64_t two_m() const { return off[n]; }
};

// Sparse set with bottom = 0 (Sec. 2, "Sparse Sets").
struct SparseSet {
  std::vector<double> val;
  std::vector<char> present;
  std::vector<int32_t> keys;  // creation order
  explicit SparseSet(int64_t n) : val(n, 0.0), present(n, 0) {}
  double get(int32_t k) const { return present[k] ? val[k] : 0.0; }
  double& at(int32_t k) {  // creates (k, 0) if missing
    if (!present[k]) {
      present[k] = 1;
      val[k] = 0.0;
      keys.push_back(k);
    }
    return val[k];
  }
  void clear() {
    for (int32_t k : keys) {
      present[k] = 0;
      val[k] = 0.0;
    }
    keys.clear();
  }
  std::vector<int32_t> sorted_keys() const {
    std::vector<int32_t> s(keys);
    std::sort(s.begin(), s.end());
    return s;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// Result object handed to Python.
// ---------------------------------------------------------------------------
enum {
  ORC_IDX = 0,      // int32: main vector ids (ascending)
  ORC_VAL = 1,      // double: main vector values
  ORC_IDX2 = 2,     // int32: secondary vector ids (PR-Nibble residual r)
  ORC_VAL2 = 3,     // double: secondary vector values
  ORC_TRACE = 4,    // int32: all frontiers concatenated, round by round
  ORC_TRACE_N = 5,  // int64: frontier size per round
  ORC_ORDER = 6,    // int32: sweep order v_1..v_N
  ORC_VOL = 7,      // int64: vol(S_i)
  ORC_CUT = 8,      // int64: cut(S_i)
  ORC_ENDPT = 9,    // int32: rand-HK-PR walk endpoints A[i]
  ORC_Z1 = 10,      // int64: Z pair first values (sweep Z path)
  ORC_Z2 = 11,      // int64: Z pair second values
  ORC_ZS1 = 12,     // int64: Z sorted, first values
  ORC_ZS2 = 13,     // int64: Z sorted, second values
  ORC_ZSUM = 14,    // int64: Z sorted, prefix-summed first values
  ORC_PUSHED = 15,  // int64: pushed edges per round
  ORC_NFIELDS = 16
};

enum {
  ORC_ST_ROUNDS = 0,
  ORC_ST_PUSHES = 1,
  ORC_ST_PUSHED_EDGES = 2,
  ORC_ST_TOUCHED = 3,
  ORC_ST_STATUS = 4,  // 0 ok, -4 max rounds reached, -1 invalid input
  ORC_ST_BEST = 5,    // sweep: best prefix length i* (0 if none)
  ORC_ST_BEST_VOL = 6,
  ORC_ST_BEST_CUT = 7,
  ORC_NSTATS = 8
};

struct orc_result {
  std::vector<int32_t> i32[ORC_NFIELDS];
  std::vector<int64_t> i64[ORC_NFIELDS];
  std::vector<double> f64[ORC_NFIELDS];
  int64_t stats[ORC_NSTATS] = {0, 0, 0, 0, 0, 0, 0, 0};
  double conductance = INFINITY;
};

static void emit_sorted(const SparseSet& s, std::vector<int32_t>& idx, std::vector<double>& val,
                        bool positive_only) {
  for (int32_t k : s.sorted_keys()) {
    double v = s.val[k];
    if (positive_only && !(v > 0.0)) continue;
    idx.push_back(k);
    val.push_back(v);
  }
}

extern "C" {

int64_t orc_len(const orc_result* r, int field, int kind) {
  if (kind == 0) return (int64_t)r->i32[field].size();
  if (kind == 1) return (int64_t)r->i64[field].size();
  return (int64_t)r->f64[field].size();
}
void orc_copy(const orc_result* r, int field, int kind, void* dst) {
  if (kind == 0) std::memcpy(dst, r->i32[field].data(), r->i32[field].size() * 4);
  else if (kind == 1) std::memcpy(dst, r->i64[field].data(), r->i64[field].size() * 8);
  else std::memcpy(dst, r->f64[field].data(), r->f64[field].size() * 8);
}
void orc_stats(const orc_result* r, int64_t* out) {
  for (int i = 0; i < ORC_NSTATS; i++) out[i] = r->stats[i];
}
double orc_conductance(const orc_result* r) { return r->conductance; }
void orc_free(orc_result* r) { delete r; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11), written from the published description: each of
// the 10 rounds multiplies counter words 0 and 2 by the two round multipliers
// (high and low 32-bit halves of the 64-bit products), XORs the high halves
// with the other two counter words and the key, and permutes; between rounds
// the key is advanced by the two Weyl constants.
// ---------------------------------------------------------------------------
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ---------------------------------------------------------------------------
// Parallel (synchronous) PR-Nibble, Sec. 3.3, "Parallel Implementation",
// Fig. alg:pr-nibble (original rule) and Fig. alg:pr-nibble2 (optimized
// rule).  Every vertex with r[v] >= eps*d(v) pushes in the same round, all
// reading r as it was at the start of the round; r' starts equal to r (the
// prose of Sec. 3.3); the frontier is then {v : r[v] >= eps*d(v)}.
//
// r and r' are held in one array: every read of r in a round is of r[v] for
// a frontier vertex v, and those values are copied into rv[] before anything
// is written, so writing r' in place gives the same result as two vectors.
//
// rule 0 (optimized, Sec. 3.3 "An Optimization"):
//   p[v] += (2a/(1+a)) r[v];  r'[w] += ((1-a)/(1+a)) r[v]/d(v);  r'[v] = 0
// rule 1 (original, following Andersen-Chung-Lang):
//   p[v] += a r[v];  r'[w] += (1-a) r[v]/(2 d(v));  r'[v] = (1-a) r[v]/2
// ---------------------------------------------------------------------------
orc_result* orc_prnibble(int64_t n, const int64_t* off, const int32_t* col, int32_t x,
                         double alpha, double eps, int rule, int64_t max_rounds, int trace) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  if (x < 0 || x >= n || g.deg(x) < 1 || !(alpha > 0.0 && alpha < 1.0) || !(eps > 0.0)) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  SparseSet p(n), r(n);
  r.at(x) = 1.0;
  std::vector<int32_t> F{x};
  const double cs = (2.0 * alpha) / (1.0 + alpha);
  const double cn = (1.0 - alpha) / (1.0 + alpha);
  int64_t rounds = 0, pushes = 0, pushed_edges = 0;
  while (!F.empty()) {
    if (rounds == max_rounds) {
      res->stats[ORC_ST_STATUS] = -4;
      break;
    }
    if (trace) {
      res->i32[ORC_TRACE].insert(res->i32[ORC_TRACE].end(), F.begin(), F.end());
      res->i64[ORC_TRACE_N].push_back((int64_t)F.size());
    }
    // r at the start of the round, for every frontier vertex.
    std::vector<double> rv(F.size());
    for (size_t i = 0; i < F.size(); i++) rv[i] = r.get(F[i]);
    // vertexMap(Frontier, UpdateSelf)
    for (size_t i = 0; i < F.size(); i++) {
      int32_t v = F[i];
      if (rule == 0) {
        p.at(v) = p.get(v) + cs * rv[i];
        r.at(v) = 0.0;
      } else {
        p.at(v) = p.get(v) + alpha * rv[i];
        r.at(v) = ((1.0 - alpha) * rv[i]) / 2.0;
      }
    }
    // edgeMap(G, Frontier, UpdateNgh)
    int64_t round_edges = 0;
    for (size_t i = 0; i < F.size(); i++) {
      int32_t v = F[i];
      int64_t d = g.deg(v);
      double share = (rule == 0) ? (cn * rv[i]) / (double)d
                                 : ((1.0 - alpha) * rv[i]) / (2.0 * (double)d);
      for (int64_t e = off[v]; e < off[v + 1]; e++) {
        int32_t w = col[e];
        r.at(w) = r.get(w) + share;
      }
      round_edges += d;
    }
    rounds++;
    pushes += (int64_t)F.size();
    pushed_edges += round_edges;
    if (trace) res->i64[ORC_PUSHED].push_back(round_edges);
    // Frontier = {v | r[v] >= d(v) eps}, over every entry of r.
    std::vector<int32_t> next;
    for (int32_t k : r.sorted_keys())
      if (r.val[k] >= eps * (double)g.deg(k)) next.push_back(k);
    F.swap(next);
  }
  res->stats[ORC_ST_ROUNDS] = rounds;
  res->stats[ORC_ST_PUSHES] = pushes;
  res->stats[ORC_ST_PUSHED_EDGES] = pushed_edges;
  res->stats[ORC_ST_TOUCHED] = (int64_t)r.keys.size();
  emit_sorted(p, res->i32[ORC_IDX], res->f64[ORC_VAL], true);
  emit_sorted(r, res->i32[ORC_IDX2], res->f64[ORC_VAL2], false);
  return res;
}

// ---------------------------------------------------------------------------
// Synchronous PR-Nibble from a seed set, with the beta-fraction rounds of
// Sec. 3.3 (the variant that, each iteration, processes only the top
// beta-fraction of {v : r[v] >= d(v) eps} by r[v]/d(v)).  Readings:
//  * seed set (Sec. 3: the algorithms extend to seed sets): r starts as the
//    distribution w_i / W on the k distinct seeds, W the sum of the weights
//    added left to right; every seed is on the first frontier;
//  * selection: the candidates are sorted by r[v]/d(v) (binary64, r as at the
//    start of the round) descending, ties by ascending id, and the first
//    ceil(beta * |F|) of them (at least one) push; the others stay in the
//    frontier, which is again every v with r[v] >= d(v) eps after the round;
//  * the selected vertices push exactly as in orc_prnibble, in ascending id.
// With one seed of weight 1 and beta = 1 this is orc_prnibble.
// ---------------------------------------------------------------------------
orc_result* orc_prnibble_set(int64_t n, const int64_t* off, const int32_t* col, int64_t k,
                             const int32_t* seeds, const double* weights, double alpha,
                             double eps, int rule, double beta, int64_t max_rounds, int trace) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  bool bad = k < 1 || !(alpha > 0.0 && alpha < 1.0) || !(eps > 0.0) || !(beta > 0.0 && beta <= 1.0);
  double W = 0.0;
  std::vector<int32_t> F;
  for (int64_t i = 0; i < k && !bad; i++) {
    const int32_t x = seeds[i];
    if (x < 0 || x >= n || g.deg(x) < 1 || !(weights[i] > 0.0)) bad = true;
    else {
      W = W + weights[i];
      F.push_back(x);
    }
  }
  std::sort(F.begin(), F.end());
  if (!bad && std::adjacent_find(F.begin(), F.end()) != F.end()) bad = true;
  if (bad) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  SparseSet p(n), r(n);
  for (int64_t i = 0; i < k; i++) r.at(seeds[i]) = weights[i] / W;
  const double cs = (2.0 * alpha) / (1.0 + alpha);
  const double cn = (1.0 - alpha) / (1.0 + alpha);
  int64_t rounds = 0, pushes = 0, pushed_edges = 0;
  while (!F.empty()) {
    if (rounds == max_rounds) {
      res->stats[ORC_ST_STATUS] = -4;
      break;
    }
    // the pushing set S: the top ceil(beta |F|) by r/d, then in ascending id
    std::vector<int32_t> S = F;
    if (beta < 1.0) {
      int64_t m = (int64_t)std::ceil(beta * (double)F.size());
      if (m < 1) m = 1;
      if (m > (int64_t)F.size()) m = (int64_t)F.size();
      std::vector<std::pair<double, int32_t>> byk;
      for (int32_t v : F) byk.push_back({r.get(v) / (double)g.deg(v), v});
      std::stable_sort(byk.begin(), byk.end(), [](const std::pair<double, int32_t>& a,
                                                    const std::pair<double, int32_t>& b) {
        return a.first > b.first || (a.first == b.first && a.second < b.second);
      });
      S.clear();
      for (int64_t i = 0; i < m; i++) S.push_back(byk[i].second);
      std::sort(S.begin(), S.end());
    }
    if (trace) {
      res->i32[ORC_TRACE].insert(res->i32[ORC_TRACE].end(), S.begin(), S.end());
      res->i64[ORC_TRACE_N].push_back((int64_t)S.size());
    }
    std::vector<double> rv(S.size());
    for (size_t i = 0; i < S.size(); i++) rv[i] = r.get(S[i]);
    for (size_t i = 0; i < S.size(); i++) {
      int32_t v = S[i];
      if (rule == 0) {
        p.at(v) = p.get(v) + cs * rv[i];
        r.at(v) = 0.0;
      } else {
        p.at(v) = p.get(v) + alpha * rv[i];
        r.at(v) = ((1.0 - alpha) * rv[i]) / 2.0;
      }
    }
    int64_t round_edges = 0;
    for (size_t i = 0; i < S.size(); i++) {
      int32_t v = S[i];
      int64_t d = g.deg(v);
      double share = (rule == 0) ? (cn * rv[i]) / (double)d
                                 : ((1.0 - alpha) * rv[i]) / (2.0 * (double)d);
      for (int64_t e = off[v]; e < off[v + 1]; e++) {
        int32_t w = col[e];
        r.at(w) = r.get(w) + share;
      }
      round_edges += d;
    }
    rounds++;
    pushes += (int64_t)S.size();
    pushed_edges += round_edges;
    std::vector<int32_t> next;
    for (int32_t kk : r.sorted_keys())
      if (r.val[kk] >= eps * (double)g.deg(kk)) next.push_back(kk);
    F.swap(next);
  }
  res->stats[ORC_ST_ROUNDS] = rounds;
  res->stats[ORC_ST_PUSHES] = pushes;
  res->stats[ORC_ST_PUSHED_EDGES] = pushed_edges;
  res->stats[ORC_ST_TOUCHED] = (int64_t)r.keys.size();
  emit_sorted(p, res->i32[ORC_IDX], res->f64[ORC_VAL], true);
  emit_sorted(r, res->i32[ORC_IDX2], res->f64[ORC_VAL2], false);
  return res;
}

// ---------------------------------------------------------------------------
// Sequential PR-Nibble with a FIFO queue, Sec. 3.3 (following Andersen,
// Chung, Lang): push one vertex at a time using the latest r, append a
// neighbour to the queue when it reaches eps*d, and keep pushing the popped
// vertex while it stays at or above its threshold.  Used to compare push
// counts with the synchronous version (Table table:pr-nibble), not for
// parity of values.
// ---------------------------------------------------------------------------
orc_result* orc_prnibble_queue(int64_t n, const int64_t* off, const int32_t* col, int32_t x,
                               double alpha, double eps, int rule) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  if (x < 0 || x >= n || g.deg(x) < 1) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  SparseSet p(n), r(n);
  std::vector<char> queued(n, 0);
  r.at(x) = 1.0;
  std::deque<int32_t> Q{x};
  queued[x] = 1;
  const double cs = (2.0 * alpha) / (1.0 + alpha);
  const double cn = (1.0 - alpha) / (1.0 + alpha);
  int64_t pushes = 0, pushed_edges = 0;
  while (!Q.empty()) {
    int32_t v = Q.front();
    Q.pop_front();
    queued[v] = 0;
    int64_t d = g.deg(v);
    do {
      double rv = r.get(v);
      double share;
      if (rule == 0) {
        p.at(v) = p.get(v) + cs * rv;
        r.at(v) = 0.0;
        share = (cn * rv) / (double)d;
      } else {
        p.at(v) = p.get(v) + alpha * rv;
        r.at(v) = ((1.0 - alpha) * rv) / 2.0;
        share = ((1.0 - alpha) * rv) / (2.0 * (double)d);
      }
      for (int64_t e = off[v]; e < off[v + 1]; e++) {
        int32_t w = col[e];
        r.at(w) = r.get(w) + share;
        if (!queued[w] && w != v && r.val[w] >= eps * (double)g.deg(w)) {
          queued[w] = 1;
          Q.push_back(w);
        }
      }
      pushes++;
      pushed_edges += d;
    } while (r.get(v) >= eps * (double)d);
  }
  res->stats[ORC_ST_ROUNDS] = pushes;
  res->stats[ORC_ST_PUSHES] = pushes;
  res->stats[ORC_ST_PUSHED_EDGES] = pushed_edges;
  res->stats[ORC_ST_TOUCHED] = (int64_t)r.keys.size();
  emit_sorted(p, res->i32[ORC_IDX], res->f64[ORC_VAL], true);
  emit_sorted(r, res->i32[ORC_IDX2], res->f64[ORC_VAL2], false);
  return res;
}

// ---------------------------------------------------------------------------
// Parallel Nibble, Sec. 3.2, Fig. alg:nibble.  For t = 1..T: p' = {};
// vertexMap sets p'[v] = p[v]/2 on the frontier; edgeMap adds p[s]/(2 d(s))
// to p'[w]; the frontier becomes {v : p'[v] >= d(v) eps}; if it is empty the
// loop stops and p (the previous vector) is returned, else p = p'.  The
// vector returned is the untruncated p of the last step that kept a
// non-empty frontier; entries below the threshold stay in it but do not
// propagate (they are not in the next frontier).
// ---------------------------------------------------------------------------
orc_result* orc_nibble(int64_t n, const int64_t* off, const int32_t* col, int32_t x, int T,
                       double eps, int trace) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  if (x < 0 || x >= n || g.deg(x) < 1 || T < 0 || !(eps >= 0.0)) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  SparseSet pa(n), pb(n);
  SparseSet* p = &pa;
  SparseSet* pp = &pb;
  p->at(x) = 1.0;
  std::vector<int32_t> F{x};
  int64_t rounds = 0, pushes = 0, pushed_edges = 0;
  for (int t = 1; t <= T; t++) {
    if (trace) {
      res->i32[ORC_TRACE].insert(res->i32[ORC_TRACE].end(), F.begin(), F.end());
      res->i64[ORC_TRACE_N].push_back((int64_t)F.size());
    }
    pp->clear();  // p' = {}
    for (int32_t v : F) pp->at(v) = p->get(v) / 2.0;  // UpdateSelf
    int64_t round_edges = 0;
    for (int32_t v : F) {  // UpdateNgh
      int64_t d = g.deg(v);
      double share = p->get(v) / (2.0 * (double)d);
      for (int64_t e = off[v]; e < off[v + 1]; e++) {
        int32_t w = col[e];
        pp->at(w) = pp->get(w) + share;
      }
      round_edges += d;
    }
    rounds++;
    pushes += (int64_t)F.size();
    pushed_edges += round_edges;
    if (trace) res->i64[ORC_PUSHED].push_back(round_edges);
    std::vector<int32_t> next;
    for (int32_t k : pp->sorted_keys())
      if (pp->val[k] >= eps * (double)g.deg(k)) next.push_back(k);
    F.swap(next);
    if (F.empty()) break;
    std::swap(p, pp);  // p = p'
  }
  res->stats[ORC_ST_ROUNDS] = rounds;
  res->stats[ORC_ST_PUSHES] = pushes;
  res->stats[ORC_ST_PUSHED_EDGES] = pushed_edges;
  res->stats[ORC_ST_TOUCHED] = (int64_t)p->keys.size();
  emit_sorted(*p, res->i32[ORC_IDX], res->f64[ORC_VAL], true);
  return res;
}

// ---------------------------------------------------------------------------
// Heat-kernel PageRank helpers, Sec. 3.4.
//   psi_k = sum_{m=0}^{N-k} k!/(m+k)! t^m, computed by the equivalent
//   recurrence psi_N = 1, psi_k = 1 + (t/(k+1)) psi_{k+1} (the tests check it
//   against the sum).  The entry threshold for level j is
//   c_j * d(v) with c_j = e^t eps / (2 N psi_j)  (Fig. alg:hkpr; the sign of
//   the exponent is the parallel figure's).
// ---------------------------------------------------------------------------
void orc_hkpr_psi(double t, int N, double* psi) {
  psi[N] = 1.0;
  for (int k = N - 1; k >= 0; k--) psi[k] = 1.0 + (t / (double)(k + 1)) * psi[k + 1];
}

// sign = -1 takes e^{-t} in place of e^{t}: the sequential description of
// Sec. 3.4 writes the threshold with e^{-t}, the parallel figure with e^{t};
// +1 is the reading followed everywhere, -1 exists to compare the two.
static std::vector<double> hk_thresholds(double t, int N, double eps, int sign = 1) {
  std::vector<double> psi(N + 1), c(N + 1);
  orc_hkpr_psi(t, N, psi.data());
  const double et = sign < 0 ? std::exp(-t) : std::exp(t);
  for (int j = 0; j <= N; j++) c[j] = (et * eps) / (2.0 * (double)N * psi[j]);
  return c;
}

// Parallel HK-PR, Sec. 3.4, Fig. alg:hkpr.  Level j = 0, 1, ...: vertexMap
// adds r[v] into p[v] on the frontier.  If j+1 < N, edgeMap adds
// t r[s]/((j+1) d(s)) into a fresh r'[w], r = r', and the frontier becomes
// {v : r[v] >= c_{j+1} d(v)}.  Otherwise (the last level) edgeMap adds
// r[s]/d(s) into p[w] and the loop ends.  The loop also ends when the
// frontier is empty.  p is returned unscaled.
orc_result* orc_hkpr_signed(int64_t n, const int64_t* off, const int32_t* col, int32_t x,
                            double t, int N, double eps, int trace, int sign) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  if (x < 0 || x >= n || g.deg(x) < 1 || N < 1 || !(t > 0.0) || !(eps >= 0.0)) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  std::vector<double> c = hk_thresholds(t, N, eps, sign);
  SparseSet p(n), ra(n), rb(n);
  SparseSet* r = &ra;
  SparseSet* rr = &rb;
  r->at(x) = 1.0;
  std::vector<int32_t> F{x};
  int j = 0;
  int64_t rounds = 0, pushes = 0, pushed_edges = 0;
  while (!F.empty()) {
    if (trace) {
      res->i32[ORC_TRACE].insert(res->i32[ORC_TRACE].end(), F.begin(), F.end());
      res->i64[ORC_TRACE_N].push_back((int64_t)F.size());
    }
    for (int32_t v : F) p.at(v) = p.get(v) + r->get(v);  // UpdateSelf
    pushes += (int64_t)F.size();
    int64_t round_edges = 0;
    if (j + 1 < N) {
      rr->clear();  // r' = {}
      for (int32_t v : F) {  // UpdateNgh
        int64_t d = g.deg(v);
        double M = (t * r->get(v)) / ((double)(j + 1) * (double)d);
        for (int64_t e = off[v]; e < off[v + 1]; e++) {
          int32_t w = col[e];
          rr->at(w) = rr->get(w) + M;
        }
        round_edges += d;
      }
      std::swap(r, rr);  // r = r'
      std::vector<int32_t> next;
      for (int32_t k : r->sorted_keys())
        if (r->val[k] >= c[j + 1] * (double)g.deg(k)) next.push_back(k);
      F.swap(next);
      rounds++;
      j++;
    } else {  // last level: UpdateNghLast
      for (int32_t v : F) {
        int64_t d = g.deg(v);
        double share = r->get(v) / (double)d;
        for (int64_t e = off[v]; e < off[v + 1]; e++) {
          int32_t w = col[e];
          p.at(w) = p.get(w) + share;
        }
        round_edges += d;
      }
      rounds++;
      F.clear();
    }
    pushed_edges += round_edges;
    if (trace) res->i64[ORC_PUSHED].push_back(round_edges);
  }
  res->stats[ORC_ST_ROUNDS] = rounds;
  res->stats[ORC_ST_PUSHES] = pushes;
  res->stats[ORC_ST_PUSHED_EDGES] = pushed_edges;
  res->stats[ORC_ST_TOUCHED] = (int64_t)p.keys.size();
  emit_sorted(p, res->i32[ORC_IDX], res->f64[ORC_VAL], true);
  return res;
}

orc_result* orc_hkpr(int64_t n, const int64_t* off, const int32_t* col, int32_t x, double t,
                     int N, double eps, int trace) {
  return orc_hkpr_signed(n, off, col, x, t, N, eps, trace, 1);
}

// Sequential HK-PR with a queue over (vertex, level) pairs, Sec. 3.4
// (following Kloster and Gleich).  (w, j+1) enters the queue when an update
// takes r[(w, j+1)] from below c_{j+1} d(w) to at least it.  The queue is
// FIFO, so all level-j pairs are processed before any level-(j+1) pair; the
// vector equals the level-synchronous one up to the order of additions.
orc_result* orc_hkpr_queue(int64_t n, const int64_t* off, const int32_t* col, int32_t x,
                           double t, int N, double eps) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  if (x < 0 || x >= n || g.deg(x) < 1 || N < 1) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  std::vector<double> c = hk_thresholds(t, N, eps);
  SparseSet p(n);
  std::map<std::pair<int32_t, int>, double> r;  // r[(v, j)]
  std::deque<std::pair<int32_t, int>> Q;
  r[{x, 0}] = 1.0;
  Q.push_back({x, 0});
  int64_t pushes = 0, pushed_edges = 0;
  while (!Q.empty()) {
    auto [v, j] = Q.front();
    Q.pop_front();
    double rvj = r[{v, j}];
    int64_t d = g.deg(v);
    p.at(v) = p.get(v) + rvj;
    double M = (t * rvj) / ((double)(j + 1) * (double)d);
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      int32_t w = col[e];
      if (j + 1 == N) {
        p.at(w) = p.get(w) + rvj / (double)d;
      } else {
        double thr = c[j + 1] * (double)g.deg(w);
        double& rw = r[{w, j + 1}];
        if (rw < thr && rw + M >= thr) Q.push_back({w, j + 1});
        rw = rw + M;
      }
    }
    pushes++;
    pushed_edges += d;
  }
  res->stats[ORC_ST_PUSHES] = pushes;
  res->stats[ORC_ST_PUSHED_EDGES] = pushed_edges;
  res->stats[ORC_ST_TOUCHED] = (int64_t)p.keys.size();
  emit_sorted(p, res->i32[ORC_IDX], res->f64[ORC_VAL], true);
  return res;
}

// ---------------------------------------------------------------------------
// Randomized heat-kernel PageRank, Sec. 3.5 (following Chung and Simpson).
// n_walks walks start at x.  Walk i draws its length k with probability
// e^{-t} t^k / k!, capped at K (all the mass of k >= K goes to K), then takes
// k steps, each to a uniformly chosen neighbour.  p[v] = (number of walks
// ending at v) / n_walks.
//
// Random stream (the paper fixes none): Philox4x32-10 with key
// (seed low word, seed high word) and counter (i low, i high, s, 0) for draw
// s of walk i.  Draw 0 gives the length: u = (w0 * 2^21 + (w1 >> 11)) / 2^53
// and k = the smallest k < K with u < CDF(k), else K.  Draw s >= 1 gives step
// s: neighbour index floor(w0 * d / 2^32).  CDF(k) is summed in double from
// term_0 = e^{-t}, term_{k+1} = term_k * t / (k + 1).
// ---------------------------------------------------------------------------
orc_result* orc_rand_hkpr(int64_t n, const int64_t* off, const int32_t* col, int32_t x,
                          double t, int K, int64_t n_walks, uint64_t seed) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  if (x < 0 || x >= n || g.deg(x) < 1 || K < 0 || n_walks < 1) {
    res->stats[ORC_ST_STATUS] = -1;
    return res;
  }
  std::vector<double> cdf(K > 0 ? K : 1);
  double term = std::exp(-t), acc = 0.0;
  for (int k = 0; k < K; k++) {
    acc = acc + term;
    cdf[k] = acc;
    term = (term * t) / (double)(k + 1);
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  std::vector<int32_t>& A = res->i32[ORC_ENDPT];
  A.resize(n_walks);
  int64_t steps = 0;
  for (int64_t i = 0; i < n_walks; i++) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 0u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t u53 = ((uint64_t)w[0] << 21) | (uint64_t)(w[1] >> 11);
    double u = (double)u53 * 0x1.0p-53;
    int k = K;
    for (int kk = 0; kk < K; kk++)
      if (u < cdf[kk]) {
        k = kk;
        break;
      }
    int32_t v = x;
    for (int s = 1; s <= k; s++) {
      ctr[2] = (uint32_t)s;
      orc_philox4x32_10(ctr, key, w);
      int64_t d = g.deg(v);
      uint32_t j = (uint32_t)(((uint64_t)w[0] * (uint64_t)d) >> 32);
      v = col[off[v] + j];
    }
    steps += k;
    A[i] = v;
  }
  // Count walks per endpoint and divide by the number of walks.
  std::map<int32_t, int64_t> count;
  for (int32_t v : A) count[v] += 1;
  for (auto& kv : count) {
    res->i32[ORC_IDX].push_back(kv.first);
    res->f64[ORC_VAL].push_back((double)kv.second / (double)n_walks);
  }
  res->stats[ORC_ST_PUSHED_EDGES] = steps;
  res->stats[ORC_ST_TOUCHED] = (int64_t)count.size();
  return res;
}

// ---------------------------------------------------------------------------
// Sequential sweep cut, Sec. 3.1.  The nonzeros of p (entries with p > 0)
// are sorted by p[v]/d(v) non-increasing, ties broken by ascending vertex id.
// Vertices are added one at a time; vol grows by d(v_i) and, for each edge
// (v_i, w), the boundary drops by one if w is already in S and grows by one
// otherwise.  phi_i = cut_i / min(vol_i, 2m - vol_i); a prefix with a zero
// denominator is skipped.  The first prefix with the smallest phi (compared
// exactly as cut_i * den_j < cut_j * den_i in 128-bit integers) is returned.
// ---------------------------------------------------------------------------
orc_result* orc_sweep(int64_t n, const int64_t* off, const int32_t* col, int64_t nnz,
                      const int32_t* idx, const double* val) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  std::vector<std::pair<double, int32_t>> items;
  for (int64_t i = 0; i < nnz; i++)
    if (val[i] > 0.0) items.push_back({val[i] / (double)g.deg(idx[i]), idx[i]});
  std::sort(items.begin(), items.end(), [](const auto& a, const auto& b) {
    if (a.first != b.first) return a.first > b.first;
    return a.second < b.second;
  });
  const int64_t two_m = g.two_m();
  std::vector<char> inS(n, 0);
  int64_t vol = 0, cut = 0;
  int64_t best = 0, best_cut = 0, best_den = 0, best_vol = 0;
  for (size_t i = 0; i < items.size(); i++) {
    int32_t v = items[i].second;
    inS[v] = 1;
    vol += g.deg(v);
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      if (inS[col[e]]) cut -= 1;
      else cut += 1;
    }
    res->i32[ORC_ORDER].push_back(v);
    res->i64[ORC_VOL].push_back(vol);
    res->i64[ORC_CUT].push_back(cut);
    int64_t den = std::min(vol, two_m - vol);
    if (den > 0) {
      if (best == 0 || (__int128)cut * best_den < (__int128)best_cut * den) {
        best = (int64_t)i + 1;
        best_cut = cut;
        best_den = den;
        best_vol = vol;
      }
    }
  }
  res->stats[ORC_ST_BEST] = best;
  res->stats[ORC_ST_BEST_VOL] = best_vol;
  res->stats[ORC_ST_BEST_CUT] = best_cut;
  res->conductance = best ? (double)best_cut / (double)best_den : INFINITY;
  return res;
}

// Parallel sweep cut of Theorem thm:sweep, written out sequentially: rank the
// sorted vertices 1..N (N+1 for vertices outside S_N); for every edge (v, w)
// of every v in S_N, in sweep order, append (1, rank v), (-1, rank w) when
// rank w > rank v and (0, rank v), (0, rank w) otherwise; stably sort Z by
// the second value; prefix-sum the first values.  The boundary of S_i is the
// summed first value of the last pair whose second value is i.  Input is the
// sweep order itself (the same sort as orc_sweep).
orc_result* orc_sweep_zpath(int64_t n, const int64_t* off, const int32_t* col, int64_t N,
                            const int32_t* order) {
  orc_result* res = new orc_result();
  Graph g{n, off, col};
  std::vector<int64_t> rank(n, N + 1);
  for (int64_t i = 0; i < N; i++) rank[order[i]] = i + 1;
  std::vector<std::pair<int64_t, int64_t>> Z;
  int64_t vol = 0;
  for (int64_t i = 0; i < N; i++) {
    int32_t v = order[i];
    vol += g.deg(v);
    res->i64[ORC_VOL].push_back(vol);
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      int32_t w = col[e];
      if (rank[w] > rank[v]) {
        Z.push_back({1, rank[v]});
        Z.push_back({-1, rank[w]});
      } else {
        Z.push_back({0, rank[v]});
        Z.push_back({0, rank[w]});
      }
    }
  }
  std::vector<std::pair<int64_t, int64_t>> Zs(Z);
  std::stable_sort(Zs.begin(), Zs.end(),
                   [](const auto& a, const auto& b) { return a.second < b.second; });
  std::vector<int64_t> summed(Zs.size());
  int64_t s = 0;
  for (size_t k = 0; k < Zs.size(); k++) {
    s += Zs[k].first;
    summed[k] = s;
  }
  std::vector<int64_t> cut(N, 0);
  for (size_t k = 0; k < Zs.size(); k++) {
    bool last = (k + 1 == Zs.size()) || (Zs[k + 1].second != Zs[k].second);
    if (last && Zs[k].second >= 1 && Zs[k].second <= N) cut[Zs[k].second - 1] = summed[k];
  }
  for (auto& z : Z) {
    res->i64[ORC_Z1].push_back(z.first);
    res->i64[ORC_Z2].push_back(z.second);
  }
  for (size_t k = 0; k < Zs.size(); k++) {
    res->i64[ORC_ZS1].push_back(Zs[k].first);
    res->i64[ORC_ZS2].push_back(Zs[k].second);
    res->i64[ORC_ZSUM].push_back(summed[k]);
  }
  res->i64[ORC_CUT] = cut;
  return res;
}

}  // extern "C"

/* Seeded synthetic graph generator (inputs only; no clustering arithmetic).
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM'04) with edge factor ef: M = ef *
 * 2^scale samples.  Sample i picks one of four quadrants per level, most
 * significant bit first, with probabilities a, b, c, 1-a-b-c; no noise and no
 * vertex permutation, so vertex 0 is the hub.  The graph is then symmetrised,
 * self loops and duplicate edges are dropped and each adjacency list is
 * sorted, giving an undirected CSR (int64 offsets, int32 columns) like the
 * paper's inputs (Sec. 4, "Input Graphs": self and duplicate edges removed).
 *
 * Random numbers: counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA'14):
 * word k of stream `seed` is mix64(seed + (k + 1) * 0x9E3779B97F4A7C15).
 * Sample i, levels 2j and 2j+1 use the high and low 32 bits of word
 * k = i * ceil(scale / 2) + j.  A 32-bit draw u picks quadrant 0 if
 * u < floor(a 2^32), 1 if u < floor((a+b) 2^32), 2 if u < floor((a+b+c) 2^32),
 * else 3.  Integer-only, so results are identical on every host.
 *
 * Threads only split independent work; the output does not depend on their
 * number.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t gg_splitmix64(uint64_t seed, uint64_t k) {
  return mix64(seed + (k + 1) * 0x9E3779B97F4A7C15ull);
}

typedef struct {
  int scale;
  uint64_t seed, lo, hi;
  uint32_t tA, tAB, tABC;
  uint64_t* keys;  /* output: 2 per sample (or fewer, self loops skipped) */
  int64_t count;   /* keys written */
  int64_t base;    /* write offset */
  int phase;       /* 0: count only, 1: write */
} gen_job;

static void* gen_worker(void* arg) {
  gen_job* J = (gen_job*)arg;
  const int halves = (J->scale + 1) / 2;
  int64_t cnt = 0;
  for (uint64_t i = J->lo; i < J->hi; i++) {
    uint64_t src = 0, dst = 0;
    for (int j = 0; j < halves; j++) {
      uint64_t w = gg_splitmix64(J->seed, i * (uint64_t)halves + (uint64_t)j);
      for (int h = 0; h < 2; h++) {
        int level = 2 * j + h;
        if (level >= J->scale) break;
        uint32_t u = h == 0 ? (uint32_t)(w >> 32) : (uint32_t)w;
        int q = u < J->tA ? 0 : (u < J->tAB ? 1 : (u < J->tABC ? 2 : 3));
        src = (src << 1) | (uint64_t)(q >> 1);
        dst = (dst << 1) | (uint64_t)(q & 1);
      }
    }
    if (src == dst) continue;
    if (J->phase == 1) {
      J->keys[J->base + cnt] = (src << J->scale) | dst;
      J->keys[J->base + cnt + 1] = (dst << J->scale) | src;
    }
    cnt += 2;
  }
  J->count = cnt;
  return NULL;
}

/* ---- parallel LSD radix sort of uint64 keys (11-bit digits) ---- */
#define RBITS 11
#define RBUCK (1 << RBITS)

typedef struct {
  const uint64_t* in;
  uint64_t* out;
  int64_t lo, hi;
  int shift;
  int64_t* hist; /* RBUCK entries, then replaced by write offsets */
} radix_job;

static void* radix_count(void* arg) {
  radix_job* J = (radix_job*)arg;
  memset(J->hist, 0, sizeof(int64_t) * RBUCK);
  for (int64_t i = J->lo; i < J->hi; i++) J->hist[(J->in[i] >> J->shift) & (RBUCK - 1)]++;
  return NULL;
}

static void* radix_scatter(void* arg) {
  radix_job* J = (radix_job*)arg;
  for (int64_t i = J->lo; i < J->hi; i++) {
    uint64_t k = J->in[i];
    J->out[J->hist[(k >> J->shift) & (RBUCK - 1)]++] = k;
  }
  return NULL;
}

static void run_threads(int nt, void* (*fn)(void*), void* jobs, size_t jsz) {
  pthread_t th[256];
  for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, fn, (char*)jobs + t * jsz);
  for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

/* Sorts keys[0..m) by their low `bits` bits; returns the buffer holding the result. */
static uint64_t* radix_sort(uint64_t* keys, uint64_t* tmp, int64_t m, int bits, int nt) {
  radix_job jobs[256];
  int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * RBUCK * nt);
  uint64_t *a = keys, *b = tmp;
  for (int shift = 0; shift < bits; shift += RBITS) {
    for (int t = 0; t < nt; t++) {
      jobs[t].in = a;
      jobs[t].out = b;
      jobs[t].lo = m * t / nt;
      jobs[t].hi = m * (t + 1) / nt;
      jobs[t].shift = shift;
      jobs[t].hist = hist + (int64_t)t * RBUCK;
    }
    run_threads(nt, radix_count, jobs, sizeof(radix_job));
    int64_t run = 0; /* digit-major, thread-minor: stable */
    for (int d = 0; d < RBUCK; d++)
      for (int t = 0; t < nt; t++) {
        int64_t c = hist[(int64_t)t * RBUCK + d];
        hist[(int64_t)t * RBUCK + d] = run;
        run += c;
      }
    run_threads(nt, radix_scatter, jobs, sizeof(radix_job));
    uint64_t* s = a;
    a = b;
    b = s;
  }
  free(hist);
  return a;
}

typedef struct {
  int64_t n, nnz;
  int64_t* off;
  int32_t* col;
} gg_graph;

/* Builds the symmetric CSR of an R-MAT graph.  Returns NULL on allocation failure. */
gg_graph* gg_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed,
                  int nthreads) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return NULL;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  const int64_t n = (int64_t)1 << scale;
  const uint64_t M = (uint64_t)edge_factor << scale;
  gen_job jobs[64];
  const double two32 = 4294967296.0;
  uint32_t tA = (uint32_t)(a * two32), tAB = (uint32_t)((a + b) * two32);
  double abc = (a + b + c) * two32;
  uint32_t tABC = abc >= two32 ? 0xFFFFFFFFu : (uint32_t)abc;
  for (int t = 0; t < nthreads; t++) {
    jobs[t].scale = scale;
    jobs[t].seed = seed;
    jobs[t].lo = M * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = M * (uint64_t)(t + 1) / (uint64_t)nthreads;
    jobs[t].tA = tA;
    jobs[t].tAB = tAB;
    jobs[t].tABC = tABC;
    jobs[t].phase = 0;
    jobs[t].keys = NULL;
  }
  run_threads(nthreads, gen_worker, jobs, sizeof(gen_job));
  int64_t m2 = 0;
  for (int t = 0; t < nthreads; t++) {
    jobs[t].base = m2;
    m2 += jobs[t].count;
  }
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (m2 > 0 ? m2 : 1));
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (m2 > 0 ? m2 : 1));
  if (!keys || !tmp) {
    free(keys);
    free(tmp);
    return NULL;
  }
  for (int t = 0; t < nthreads; t++) {
    jobs[t].keys = keys;
    jobs[t].phase = 1;
  }
  run_threads(nthreads, gen_worker, jobs, sizeof(gen_job));
  uint64_t* sorted = radix_sort(keys, tmp, m2, 2 * scale, nthreads);
  uint64_t* other = sorted == keys ? tmp : keys;
  free(other);
  /* unique + CSR */
  gg_graph* G = (gg_graph*)malloc(sizeof(gg_graph));
  G->n = n;
  G->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t u = 0;
  for (int64_t i = 0; i < m2; i++)
    if (i == 0 || sorted[i] != sorted[i - 1]) sorted[u++] = sorted[i];
  G->nnz = u;
  G->col = (int32_t*)malloc(sizeof(int32_t) * (u > 0 ? u : 1));
  for (int64_t i = 0; i < u; i++) {
    G->col[i] = (int32_t)(sorted[i] & (uint64_t)(n - 1));
    G->off[(sorted[i] >> scale) + 1]++;
  }
  for (int64_t v = 0; v < n; v++) G->off[v + 1] += G->off[v];
  free(sorted);
  return G;
}

int64_t gg_n(const gg_graph* G) { return G->n; }
int64_t gg_nnz(const gg_graph* G) { return G->nnz; }
void gg_copy(const gg_graph* G, int64_t* off, int32_t* col) {
  memcpy(off, G->off, sizeof(int64_t) * (size_t)(G->n + 1));
  memcpy(col, G->col, sizeof(int32_t) * (size_t)G->nnz);
}
void gg_free(gg_graph* G) {
  if (!G) return;
  free(G->off);
  free(G->col);
  free(G);
}

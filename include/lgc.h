/*
 * lgc.h -- C ABI of liblgc, GB300 (sm_103a) local graph clustering.
 *
 * Implements the parallel local clustering methods of Shun,
 * Roosta-Khorasani, Fountoulakis and Mahoney, "Parallel Local Graph
 * Clustering" (arXiv:1604.07515): the synchronous frontier push of PR-Nibble
 * (Sec. 3.3), Nibble (Sec. 3.2), deterministic heat-kernel PageRank
 * (Sec. 3.4), randomized heat-kernel PageRank (Sec. 3.5) and the parallel
 * sweep cut (Sec. 3.1, Theorem thm:sweep).  Every step runs in the library's
 * own CUDA kernels on one GPU; all values are IEEE binary64.
 *
 * Conventions
 *  - Every function returns LGC_OK (0) on success or a negative LGC_E* code;
 *    lgc_poll also returns LGC_PENDING (1).  Nothing aborts the process.
 *  - Inputs are copied; the library keeps no caller pointer after a call
 *    returns.  Outputs (lgc_svec, lgc_cluster, lgc_result) are owned by the
 *    library and released with the matching *_free function.  Host outputs
 *    live in page-locked memory from a process-wide pool and stay valid after
 *    their context is destroyed; device outputs must be released before
 *    their context.
 *  - Graphs are undirected and unweighted: CSR with int64 offsets[n+1] and
 *    int32 cols[offsets[n]], every edge stored in both directions, each
 *    adjacency list sorted ascending, no self loops, no duplicate edges
 *    (Sec. 2, "Graph Notation"; Sec. 4, "Input Graphs").
 *  - A seed x must satisfy 0 <= x < n and d(x) >= 1, else LGC_EINVAL.
 *  - Calls on one context are serialised by the caller (one stream per
 *    context); lgc_submit / lgc_poll / lgc_wait are thread-safe.
 */
#ifndef LGC_H_
#define LGC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LGC_OK 0
#define LGC_PENDING 1          /* lgc_poll: request not finished yet */
#define LGC_EINVAL (-1)        /* bad argument (seed, parameter, graph) */
#define LGC_ENOMEM (-2)        /* device or host allocation failed */
#define LGC_ETABLEFULL (-3)    /* a hash table probe exceeded its bound */
#define LGC_EMAXROUNDS (-4)    /* max_rounds reached; the partial p is still returned */
#define LGC_ECUDA (-5)         /* a CUDA runtime call failed */
#define LGC_EBUSY (-6)         /* submit refused: queue full or over memory budget */
#define LGC_ENOTFOUND (-7)     /* unknown ticket */
#define LGC_ETIMEOUT (-8)      /* a bounded device wait gave up */

typedef struct lgc_ctx lgc_ctx;
typedef struct lgc_graph lgc_graph;

/* Sparse vector: nnz entries, idx ascending, values > 0 (the sparse sets of
 * Sec. 2, "Sparse Sets", with only the non-zero entries kept).  idx/val are
 * device pointers when on_device != 0, host pointers otherwise. */
typedef struct {
  int64_t nnz;
  int32_t *idx;
  double *val;
  int on_device;
} lgc_svec;

/* Sweep-cut result (Sec. 3.1): ids = S_{i*} in sweep order (non-increasing
 * p/d, ties by ascending id), vol = vol(S_{i*}), cut = |boundary(S_{i*})|,
 * conductance = cut / min(vol, 2m - vol) (+inf for an empty result). */
typedef struct {
  int64_t size;
  int32_t *ids;
  int64_t vol, cut;
  double conductance;
  int on_device;
} lgc_cluster;

/* Per-call counters.  rounds: push rounds (levels for HK-PR, steps for
 * Nibble); pushes: sum of frontier sizes; pushed_edges: sum over rounds of
 * the frontier's degrees (walk steps for rand-HK-PR); touched: keys in the
 * result's sparse set; table_capacity: final hash-table slots. */
typedef struct {
  int64_t rounds, pushes, pushed_edges, touched, table_capacity;
  int status_detail;
} lgc_stats;

enum { LGC_RULE_OPT = 0, LGC_RULE_ORIG = 1 };
/* LGC_MODE_ATOMIC: scatter with fetch-and-add (Sec. 2, "Atomic Operations"),
 *   result within rounding of the canonical order.
 * LGC_MODE_DET: every destination sums its contributions starting from the
 *   value it holds when the edge phase begins, then in ascending source id;
 *   results, frontiers and rounds are bit-reproducible. */
enum { LGC_MODE_ATOMIC = 0, LGC_MODE_DET = 1 };

/* PR-Nibble (Sec. 3.3; Fig. alg:pr-nibble with the original rule,
 * Fig. alg:pr-nibble2 with the optimized rule).  0 < alpha < 1, eps > 0;
 * max_rounds <= 0 means no limit. */
typedef struct {
  double alpha, eps;
  int rule;
  int mode;
  int64_t max_rounds;
} lgc_prnibble_params;

/* Nibble (Sec. 3.2, Fig. alg:nibble): T >= 0 lazy-walk steps, eps >= 0. */
typedef struct {
  int T;
  double eps;
  int mode;
} lgc_nibble_params;

/* HK-PR (Sec. 3.4, Fig. alg:hkpr): t > 0, N >= 1 Taylor terms, eps >= 0.
 * The entry threshold for level j is e^t eps d(v) / (2 N psi_j). */
typedef struct {
  double t, eps;
  int N;
  int mode;
} lgc_hkpr_params;

/* rand-HK-PR (Sec. 3.5): 1 <= n_walks <= INT32_MAX walks of Poisson(t)
 * length capped at K, 0 <= K <= 128, t >= 0; random stream Philox4x32-10
 * keyed by rng_seed.  Other values: LGC_EINVAL. */
typedef struct {
  double t;
  int K;
  int64_t n_walks;
  uint64_t rng_seed;
} lgc_rand_hkpr_params;

/* ---- context ---- */

/* Creates a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * owned by the caller (for example torch.cuda.current_stream().cuda_stream),
 * or NULL for a stream owned by the context.  All work of the context is
 * ordered on that stream. */
int lgc_ctx_create(int device, void *cuda_stream, lgc_ctx **out);
void lgc_ctx_destroy(lgc_ctx *ctx);

/* Device memory from the caller's allocator instead of the device's
 * stream-ordered pool (for example PyTorch's caching allocator, so that the
 * library's graphs and temporaries come out of the same memory as the
 * caller's tensors).  alloc(bytes, stream, user) returns device memory for
 * work ordered on `stream` (the context's stream), or NULL (the call then
 * fails with LGC_ENOMEM); free(ptr, stream, user) may be called while work
 * that reads ptr is still queued on that stream, so the allocator must not
 * hand the block to another stream before that work is done (a stream-ordered
 * pool keyed by stream, as PyTorch's is, satisfies this).  Both are called
 * only from the thread that calls into the context.  The request loop's
 * worker contexts (lgc_submit) keep the device pool. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *user);
  void (*free)(void *ptr, void *stream, void *user);
  void *user;
} lgc_alloc_fns;
/* lgc_ctx_create with the allocator `fns` (copied; NULL: the device pool).
 * LGC_EINVAL if fns has a NULL alloc or free. */
int lgc_ctx_create_with_alloc(int device, const lgc_alloc_fns *fns, void *cuda_stream,
                              lgc_ctx **out);

enum {
  LGC_OPT_RESULT_ON_DEVICE = 1, /* 1: outputs stay in device memory (default 0: host) */
  LGC_OPT_TRACE = 2,            /* 1: record every round's frontier (tests) */
  LGC_OPT_SERVE_MEM_BUDGET = 3, /* bytes of hash-table memory admitted at once */
  LGC_OPT_SERVE_MAX_BATCH = 4,  /* requests resident on the device at once */
  LGC_OPT_TABLE_FORM = 6,       /* sparse sets: 0 automatic (dense once a set may reach
                                   n/8 keys; in lgc_prnibble_batch, once a seed's hashed
                                   table would take more memory than the dense form), 1
                                   always hashed, 2 always dense (lgc_prnibble_batch: as 0) */
  LGC_OPT_PULL = 7,             /* deterministic rounds gather from the frontier instead of
                                   sorting pushed records: 0 automatic (rounds of >= 2m/16
                                   edges), 1 never, 2 always; same results either way */
  LGC_OPT_DEVICE_ROUNDS = 8,    /* 1 (default): consecutive small rounds of atomic-mode
                                   PR-Nibble run in one cooperative launch without returning
                                   to the host in between; 0: one launch per step.  Request-
                                   loop workers never use it.  Same results either way */
  LGC_OPT_PULL_BATCH = 9,       /* edges per lane per batch in the heavy-vertex pull gather:
                                   0 (default) the graph's tuned value (see
                                   lgc_graph_autotune), or 4, 8, 16 */
  LGC_OPT_PULL_GROUP = 10,      /* lanes per work item in the heavy-vertex pull gather: 0
                                   (default) the graph's tuned value, or 8, 16, 32 (only
                                   the pairs lgc_graph_autotune tries are compiled: 4 with
                                   32; 8 and 16 with 8, 16, 32) */
  LGC_OPT_PULL_SHARE = 11,      /* bytes per gathered share in atomic pull rounds: 0
                                   (default) the graph's tuned value, 16 (fixed-point
                                   records) or 8 (doubles, converted per edge); same
                                   results either way */
  LGC_OPT_BATCH_HANDOFF = 12,   /* lgc_prnibble_batch: a seed whose frontier's degree sum
                                   reaches this many edges leaves the batch and finishes
                                   alone (pull rounds, dense sets), with the same result;
                                   0 (default) the graph's value (see
                                   lgc_graph_batch_handoff), -1 never */
  LGC_OPT_SERVE_LANE = 14,      /* request loop: PR-Nibble requests resident at once in its
                                   batched lane (their rounds run together, requests join
                                   as they are admitted); 0 runs them on the worker
                                   contexts like the other requests.  Default 1024; set
                                   before the first lgc_submit (LGC_EBUSY after) */
  LGC_OPT_HK_THRESHOLD_SIGN = 13, /* debug: the sign of the exponent in lgc_hkpr's entry
                                   thresholds.  +1 (default): e^t eps d(v) / (2 N psi_j),
                                   as in the parallel HK-PR figure (Sec. 3.4); -1: e^-t,
                                   as in the sequential description of Sec. 3.4, which
                                   makes the diffusion spread much further.  Request-loop
                                   workers always use +1 */
  LGC_OPT_SWEEP_CROSS = 15      /* lgc_sweep's crossing counts (step S5): 0 (default)
                                   automatic (vertex-centric for a support of at least n/32
                                   vertices), 1 edge-balanced over the swept vertices'
                                   edges, 2 vertex-centric over the graph's degree-binned
                                   lists whenever the ranks are kept in a dense array (a
                                   support of at least n/64 vertices, n >= 1024); same
                                   results either way */
};
int lgc_ctx_set_option(lgc_ctx *ctx, int option, int64_t value);
/* Waits for all work issued on the context's stream. */
int lgc_ctx_synchronize(lgc_ctx *ctx);

/* ---- graph ---- */
#define LGC_GRAPH_VALIDATE 1     /* check symmetry, order, no self loops / duplicates */
#define LGC_GRAPH_DEVICE_INPUT 2 /* offsets / cols are device pointers */
/* Copies the CSR (Sec. 2) to the device.  Errors: LGC_EINVAL for n < 0, NULL
 * arrays, or a failed validation; LGC_ENOMEM. */
int lgc_graph_create(lgc_ctx *ctx, int64_t n, const int64_t *offsets, const int32_t *cols,
                     int flags, lgc_graph **out);
void lgc_graph_destroy(lgc_graph *g);
/* Tunes the graph's launch shapes by timing them on the graph itself (the
 * paper has no counterpart; it affects speed only, never results):
 *  - for the pull gathers of atomic rounds, the degree bin (vertices of
 *    degree <= 32, 64, 128 or 256 gather one thread each, the others in work items
 *    of up to 4096 edges; see lgc_graph_set_pull_light) and the heavy
 *    gather's edges per lane per batch and lanes per work item, from (4, 32),
 *    (8, 32), (16, 32), (8, 16), (16, 16), (8, 8), (16, 8), each with 16- and
 *    8-byte gathered shares, on a frontier of all vertices (a few launches of
 *    the light and the heavy gather per candidate); the shape is written to
 *    *pull_batch, *pull_group, *pull_share (nullable);
 *  - for lgc_prnibble_batch and the request loop's PR-Nibble lane, the
 *    frontier size (in edges) at which a seed leaves the batch and finishes
 *    alone, from 2m/64, 2m/16, 2m/4 (each at least 2^20) and never, timing
 *    one batch of 256 seeds of the graph at each (lgc_graph_batch_handoff
 *    reports the choice).
 * Until it is called the graph uses (8, 32, 16) and max(2^20, 2m/64). */
int lgc_graph_autotune(lgc_graph *g, int *pull_batch, int *pull_group, int *pull_share);
/* The hand-off threshold (edges) the graph's batches use while
 * LGC_OPT_BATCH_HANDOFF is 0: the tuned value, else max(2^20, 2m/64);
 * INT64_MAX means never. */
int64_t lgc_graph_batch_handoff(const lgc_graph *g);
/* The degree bin of the graph's atomic pull rounds: vertices of degree
 * 1..light gather with one thread each, the others in work items.  The
 * deterministic pull rounds keep their own bins at any light: degree 1..32
 * folded in one thread each, up to 1024 one lane each, longer lists
 * segment-parallel.  Default 32;
 * lgc_graph_autotune picks one of 32, 64, 128, 256.  lgc_graph_set_pull_light
 * rebuilds the graph's vertex lists for 4 <= light <= 256 (LGC_EINVAL
 * otherwise); it waits for the request loop's requests on the graph.  Speed
 * only: results do not depend on it. */
int lgc_graph_pull_light(const lgc_graph *g);
int lgc_graph_set_pull_light(lgc_graph *g, int light);
int64_t lgc_graph_num_vertices(const lgc_graph *g);
int64_t lgc_graph_num_entries(const lgc_graph *g); /* 2m */

/* ---- diffusions: seed + parameters -> sparse vector p ---- */
/* Synchronous PR-Nibble (Sec. 3.3, "Parallel Implementation"): every vertex
 * with r[v] >= eps d(v) pushes in the same round, reading r from the start of
 * the round; returns p.  st may be NULL. */
int lgc_prnibble(lgc_graph *g, int32_t seed, const lgc_prnibble_params *prm, lgc_svec **p,
                 lgc_stats *st);
/* PR-Nibble from a seed set with beta-fraction rounds.  Sec. 3 notes that the
 * algorithms extend to seed sets and Sec. 3.3 describes the variant that
 * processes, each iteration, only the top beta-fraction of
 * {v : r[v] >= eps d(v)} by r[v]/d(v).  Here r starts as the distribution
 * w_i / W over the k distinct seeds (W = the weights summed left to right;
 * weights NULL: all 1), all seeds on the first frontier; each round the first
 * ceil(beta |F|) (at least one) candidates by r/d descending, ties by
 * ascending id, push as in lgc_prnibble and the others stay candidates.
 * beta in (0, 1]; k = 1 with beta = 1 is lgc_prnibble.  Errors: LGC_EINVAL
 * for a repeated or invalid seed, a weight <= 0, beta outside (0, 1]. */
int lgc_prnibble_set(lgc_graph *g, int64_t k, const int32_t *seeds, const double *weights,
                     double beta, const lgc_prnibble_params *prm, lgc_svec **p,
                     lgc_stats *st);
/* Parallel Nibble (Sec. 3.2, Fig. alg:nibble); returns p_T, or p_{i-1} when
 * the frontier of step i is empty. */
int lgc_nibble(lgc_graph *g, int32_t seed, const lgc_nibble_params *prm, lgc_svec **p,
               lgc_stats *st);
/* Parallel HK-PR (Sec. 3.4, Fig. alg:hkpr); returns the unscaled p. */
int lgc_hkpr(lgc_graph *g, int32_t seed, const lgc_hkpr_params *prm, lgc_svec **p,
             lgc_stats *st);
/* Parallel rand-HK-PR (Sec. 3.5): p[v] = (walks ending at v) / n_walks.
 * Walk i uses Philox4x32-10 with key (rng_seed low, high word) and counter
 * (i low, i high, s, 0) for its draw s: draw 0 sets the length (53-bit
 * uniform against the Poisson(t) CDF, capped at K), draw s >= 1 picks the
 * neighbour floor(word0 * d / 2^32). */
int lgc_rand_hkpr(lgc_graph *g, int32_t seed, const lgc_rand_hkpr_params *prm, lgc_svec **p,
                  lgc_stats *st);
/* Optional: the endpoints A[0..n_walks) of the last lgc_rand_hkpr call on
 * this context, copied to host memory `out` (n_walks int32).  Tests only. */
int lgc_rand_hkpr_endpoints(lgc_ctx *ctx, int32_t *out, int64_t n_walks);

/* ---- many seeds at once ---- */
/* PR-Nibble (Sec. 3.3) for B seeds in one batch: every round runs the push of
 * all seeds that still have a frontier with one launch per kernel, each seed
 * on its own sparse sets with its own parameters (seeds[b], prm[b]), so each
 * result is the same as lgc_prnibble's for that seed (bit-identical in
 * LGC_MODE_DET; within rounding in LGC_MODE_ATOMIC).  All prm[b].mode must
 * be equal.  p_out[b] receives seed b's vector (host or device per
 * LGC_OPT_RESULT_ON_DEVICE); st (nullable) B counters.  The paper names
 * running many local computations independently in parallel as the
 * straightforward use of parallelism (Sec. 1), and its network community
 * profiles run PR-Nibble from 10^5 seeds (Sec. 4). */
int lgc_prnibble_batch(lgc_graph *g, int64_t B, const int32_t *seeds,
                       const lgc_prnibble_params *prm, lgc_svec **p_out, lgc_stats *st);

/* ---- sweep cut (Sec. 3.1, Theorem thm:sweep) ---- */
/* Sorts the entries of p with p > 0 by p[v]/d(v) non-increasing (ties by
 * ascending id), computes vol and boundary of every prefix by prefix sums,
 * and returns the prefix of smallest conductance (exact rational comparison,
 * first index on ties; prefixes with min(vol, 2m - vol) = 0 are skipped).
 * p may be on the host or the device (p->on_device).  Errors: LGC_EINVAL if
 * an entry is not a vertex of degree >= 1 or names a vertex a second time. */
int lgc_sweep(lgc_graph *g, const lgc_svec *p, lgc_cluster **out);

/* Sweep cuts of B vectors in one pass: out[b] is lgc_sweep(g, p[b], ...) for
 * every b (the same cluster, vol, cut and conductance), computed with one
 * sort of all their entries (by key, then stably by vector), one rank table
 * per vector and one edge-balanced crossing count over all of them.  The
 * vectors may be on the host or the device, each its own.  Errors: as
 * lgc_sweep, for the whole batch (no out[b] is set then). */
int lgc_sweep_batch(lgc_graph *g, int64_t B, const lgc_svec *const *p, lgc_cluster **out);

/* ---- sweep cut without device allocation ---- */
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory during a call: processes
 * whose device memory is all handed to their own allocator up front (for
 * example a serving process that reserved the GPU's memory), or
 * latency-critical paths that cannot risk an out-of-memory failure or an
 * allocation's device synchronisation mid-request.
 *
 * Same result as lgc_sweep on the entries (d_idx[i], d_val[i]), i < nnz,
 * which are DEVICE pointers (idx ascending, as for lgc_sweep).  The caller
 * provides d_ids, a device buffer of at least nnz int32, which receives the
 * cluster in sweep order; *out (host memory owned by the caller) receives
 * size, vol, cut and conductance, with out->ids = d_ids and out->on_device = 1.
 * Do not pass *out to lgc_cluster_free.
 *
 * No device memory is allocated or freed by the call: all temporaries live
 * in one fixed-size device array (about 5.6 MB), held until the process
 * exits.  With CUDA's lazy module loading (the default) the driver reserves
 * that array on a device at the first lgc_sweep_noalloc call there (an empty
 * vector, nnz = 0, will do): make that call before handing the rest of the
 * GPU's memory to another allocator.  Limits and behaviour:
 *  - nnz > LGC_SWEEP_NOALLOC_MAX_N is rejected with LGC_EINVAL;
 *  - an entry that is not a vertex of degree >= 1, or a vertex named twice:
 *    LGC_EINVAL (as lgc_sweep);
 *  - all calls share the array, so calls that overlap on the GPU (different
 *    streams, contexts or threads) race and return wrong results; serialise
 *    them;
 *  - the first call on a device looks up the array's device address; make it
 *    before any stream capture;
 *  - runs on the graph's context stream and waits for it before returning. */
#define LGC_SWEEP_NOALLOC_MAX_N 65536
int lgc_sweep_noalloc(lgc_graph *g, int64_t nnz, const int32_t *d_idx, const double *d_val,
                      int32_t *d_ids, lgc_cluster *out);

/* ---- tracing (deterministic-mode parity tests) ---- */
#define LGC_TRACE_FRONTIERS 1 /* record every round's frontier */
/* lgc_ctx_set_option(ctx, LGC_OPT_TRACE, flags & LGC_TRACE_FRONTIERS): flags
 * 0 turns recording off; other bits are reserved (LGC_EINVAL). */
int lgc_set_trace(lgc_ctx *ctx, int flags);
/* Frontiers of the last diffusion call recorded under LGC_OPT_TRACE:
 * *rounds receives the round count; if sizes != NULL it receives the size of
 * each round's frontier (up to cap_rounds entries); if frontiers != NULL it
 * receives the frontiers concatenated (up to cap_ids ids).  Frontiers are in
 * ascending id in LGC_MODE_DET and in arrival order in LGC_MODE_ATOMIC. */
int lgc_get_trace(lgc_ctx *ctx, int64_t *rounds, int64_t *sizes, int64_t cap_rounds,
                  int32_t *frontiers, int64_t cap_ids);
/* The residual r of the last lgc_prnibble call made under LGC_OPT_TRACE:
 * every key of r's sparse set (the seed and every neighbour of a pushed
 * vertex, Sec. 3.3), zeros included, in a host svec that the caller frees.
 * LGC_ENOTFOUND if there is none.  Tests only. */
int lgc_prnibble_residual(lgc_ctx *ctx, lgc_svec **r);

/* ---- measurement ---- */
/* Kernels launched on this context so far (all of the library's kernels). */
int64_t lgc_launch_count(const lgc_ctx *ctx);
/* Per-kernel timing, recorded with CUDA events on the context's stream
 * around every launch of the named kernel while LGC_OPT_PROFILE is 1.
 * bytes = the algorithmic bytes of those launches (what the method must
 * move: 24 per pushed edge, 24 per frontier vertex staged, 8 per next
 * frontier entry for the edgeMap; 20 per walk step and 4 per walk for the
 * walk kernel; 12 per edge of vol(S_N) plus 24 per swept vertex for the
 * sweep's crossing count). */
enum {
  LGC_PROF_EDGEMAP = 0,    /* atomic-mode edgeMap of push rounds (push scatter, and the
                              device-round kernels) */
  LGC_PROF_VERTEXMAP = 1,  /* vertexMap kernels */
  LGC_PROF_DET_EDGE = 2,   /* deterministic-mode emit + sort + fold + compact, and the
                              deterministic pull gathers */
  LGC_PROF_WALK = 3,       /* rand-HK-PR walk kernel */
  LGC_PROF_SWEEP = 4,      /* sweep crossing-count kernel */
  LGC_PROF_PULL = 5,       /* atomic-mode edgeMap of pull rounds (the light and heavy
                              gathers); same algorithmic bytes as LGC_PROF_EDGEMAP */
  LGC_PROF_COUNT = 6
};
#define LGC_OPT_PROFILE 5
typedef struct {
  int64_t launches;
  double ms;    /* summed event-timed duration */
  double bytes; /* summed algorithmic bytes */
} lgc_kernel_profile;
int lgc_profile_read(lgc_ctx *ctx, int kernel, lgc_kernel_profile *out);
int lgc_profile_reset(lgc_ctx *ctx);

/* ---- request loop (continuous batching) ---- */
enum { LGC_ALGO_PRNIBBLE = 0, LGC_ALGO_NIBBLE = 1, LGC_ALGO_HKPR = 2, LGC_ALGO_RAND_HKPR = 3 };
typedef struct {
  int algo;
  int32_t seed;
  int want_sweep;
  lgc_prnibble_params pr;
  lgc_nibble_params nb;
  lgc_hkpr_params hk;
  lgc_rand_hkpr_params rh;
} lgc_request;
typedef struct {
  int status;            /* LGC_OK or the request's error code */
  lgc_svec *p;           /* host-resident */
  lgc_cluster *cluster;  /* host-resident; NULL unless want_sweep */
  lgc_stats stats;
  double submit_s, start_s, end_s; /* host monotonic clock, seconds */
} lgc_result;
/* Queues one request against graph g (which must outlive it).  The loop
 * batches continuously: PR-Nibble requests (unless LGC_OPT_SERVE_LANE is 0)
 * join one batched lane whose admitted seeds all advance one synchronous
 * round per pass (lgc_prnibble_batch's engine; a request admitted while
 * others run starts at the next round, a finished one leaves with its vector
 * and sweep cut), admitted while the lane's live tables plus the workers'
 * reservations stay within LGC_OPT_SERVE_MEM_BUDGET and at most
 * LGC_OPT_SERVE_LANE seeds are resident.  The other requests run on up to
 * LGC_OPT_SERVE_MAX_BATCH worker contexts side by side with the lane, each
 * admitted when the memory it may need fits the budget; the first queued
 * request that fits goes next, and a request passed over 16 times is
 * admitted before anything behind it.  Each result equals that of the same
 * call made alone (bit for bit in LGC_MODE_DET).  Returns LGC_EBUSY if the
 * queue is full. */
int lgc_submit(lgc_ctx *ctx, lgc_graph *g, const lgc_request *req, uint64_t *ticket);
/* LGC_PENDING while the request runs; LGC_OK and *out when done (the ticket
 * is then released); LGC_ENOTFOUND for an unknown ticket. */
int lgc_poll(lgc_ctx *ctx, uint64_t ticket, lgc_result **out);
/* As lgc_poll, but blocks (without spinning: it sleeps on the loop's
 * condition variable) until the request is done: LGC_OK and *out, or
 * LGC_ENOTFOUND for an unknown or already taken ticket, or when the context
 * is being destroyed.  Thread-safe like lgc_poll; it must not overlap
 * lgc_ctx_destroy of its context. */
int lgc_wait(lgc_ctx *ctx, uint64_t ticket, lgc_result **out);

/* ---- release ---- */
void lgc_svec_free(lgc_svec *p);
void lgc_cluster_free(lgc_cluster *c);
void lgc_result_free(lgc_result *r);
const char *lgc_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* LGC_H_ */

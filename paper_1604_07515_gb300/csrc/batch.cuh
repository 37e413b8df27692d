// The batch engine behind lgc_prnibble_batch and the request loop's
// PR-Nibble lane: many seeds' synchronous PR-Nibble rounds (Sec. 3.3) run
// together, one launch per kernel per round, each seed on its own sparse
// sets with its own parameters.  Seeds occupy slots; seeds can join between
// rounds, and a finished seed's slot is extracted and reused.
#pragma once

#include <vector>

#include "common.cuh"

namespace lgc {

struct SeedParam {
  double alpha, eps, cs, cn;
  int rule;
  int pad;
};

// Per-seed counters of one round, read back by the host once per round.
struct SeedCount {
  int32_t next_size;
  int32_t err;
  int64_t next_edges;
  int64_t inserted;
};

// Table storage: the tables created or grown in one step share one device
// allocation (a slab), cleared by one memset; a slab is freed when none of
// its tables is in use any more.
struct Slabs {
  std::vector<void*> ptr;
  std::vector<int64_t> refs;
  void release(lgc_ctx* ctx, int id) {
    if (id >= 0 && --refs[id] == 0) {
      dfree(ctx, ptr[id]);
      ptr[id] = nullptr;
    }
  }
  void release_all(lgc_ctx* ctx) {
    for (size_t i = 0; i < ptr.size(); i++)
      if (ptr[i]) dfree(ctx, ptr[i]);
    ptr.clear();
    refs.clear();
  }
};

struct Regrow {
  Table from, to;
};

struct BatchEngine {
  enum { kFree = 0, kRunning = 1, kDone = 2 };
  lgc_ctx* ctx = nullptr;
  lgc_graph* g = nullptr;
  int mode = 0;
  bool det = false;
  int64_t n = 0;
  int vbits = 1;
  int64_t handoff_edges = 0;
  int64_t cap = 0;      // slots
  int64_t nf = 0;       // frontier entries of all running seeds
  int64_t running = 0;  // seeds with a frontier
  std::vector<int64_t> done;  // slots finished since the caller last took them
  // per slot
  std::vector<int32_t> seed_of;
  std::vector<int64_t> dseed, count, nfs, edges, rounds, pushes, pushed, max_rounds;
  std::vector<SeedParam> sp;
  std::vector<lgc_prnibble_params> prm;
  std::vector<Table> tabs;
  std::vector<int> slab_of;
  std::vector<int32_t> grown, alive;
  std::vector<int> state, fin_status;
  std::vector<char> alone;
  std::vector<lgc_svec*> p_alone;
  std::vector<lgc_stats> st_alone;
  std::vector<SeedCount> sc_h;
  std::vector<int32_t> cursor_h;
  std::vector<int64_t> free_slots;
  bool tabs_dirty = false, prm_dirty = false;
  Slabs slabs;
  // device
  int32_t* gsize = nullptr;  // frontier size, overflow, rehash error, init error
  DBuf<Table> d_tabs;
  DBuf<SeedParam> d_prm;
  DBuf<SeedCount> d_sc;
  DBuf<int32_t> d_grown, d_alive, d_cursor, d_new;
  DBuf<Regrow> d_rg;
  DBuf<int64_t> d_rgbeg;
  DBuf<int32_t> Fs, Fv, Fslot, Gs, Gv, Gslot, segseed, segv, segslot;
  DBuf<double> share, rv, rv2;
  DBuf<int64_t> cnt, epos, foff, total, flag, segid, segstart, qflag, qpos;
  DBuf<uint64_t> rk, rk2;

  int init(lgc_ctx* c, lgc_graph* gr, int mode);
  int reserve_slots(int64_t want);
  // Seeds k with parameters P (all of this engine's mode) join; they run
  // their first round in the next round().  slots_out (nullable) receives
  // their slots.
  int add(int64_t k, const int32_t* seeds, const lgc_prnibble_params* P, int64_t* slots_out);
  // One synchronous round for every running seed; seeds that finish are
  // appended to `done`.
  int round();
  // Results (and counters) of finished slots; the slots stay occupied until
  // release().
  int extract(const std::vector<int64_t>& which, lgc_svec** outs, lgc_stats* sts);
  void release(int64_t slot);
  int64_t table_bytes_live() const;
  void fini();

 private:
  int upload();
  int compact_alive();
  void finish(int64_t b, int status);
};

int64_t table_bytes(int64_t cap);
// The hand-off threshold of graph g when the context leaves it to the graph:
// its tuned value, else max(2^20, 2m/64).
int64_t batch_handoff_of(const lgc_graph* g);
int autotune_batch(lgc_ctx* ctx, lgc_graph* g);
int run_prnibble_batch(lgc_ctx* ctx, lgc_graph* g, int64_t B, const int32_t* seeds_h,
                       const lgc_prnibble_params* prm_h, lgc_svec** p_out, lgc_stats* st_out);

}  // namespace lgc

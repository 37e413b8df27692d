"""Benchmark: one step = the whole hot path on one seed of the R-MAT scale-22
workload (4.19M vertices, edge factor 16, a=0.57 b=c=0.19, seed 2; seed
vertex = vertex 0's highest-degree neighbour):

  PR-Nibble  (alpha 0.01, eps 1e-7)            + sweep cut
  Nibble     (T 20, eps 1e-7)                  + sweep cut
  HK-PR      (t 10, N 20, eps 1e-7)            + sweep cut
  rand-HK-PR (t 10, K 10, 1e6 walks, Philox 7) + sweep cut

Metric: pushed edges per second (sum over the four diffusions of the
frontier degrees pushed; walk steps for rand-HK-PR), plus clusters/s.
The graph (513 MB of columns) exceeds L2; L2 is also flushed between timed
steps.  Under torchrun each rank runs the same step for its own seed vertex
(independent problems, no collective): weak scaling.

Beside the headline step, on one GPU (rank 0 of a single-rank run):

* ``det_step``: the same step in deterministic mode;
* ``many_seeds``: 1024 PR-Nibble + sweep clusters on R-MAT scale 24 (seed 4),
  eps log-uniform in [1e-8, 1e-5]: one lgc_prnibble_batch + lgc_sweep_batch
  call for all of them, one lgc_prnibble + lgc_sweep per seed, and all of
  them through the request loop;
* ``config3``: PR-Nibble + sweep from 8 seeds of R-MAT scale 26 (seed 3,
  2.1 billion CSR entries), eps 1e-7 and 1e-8, atomic and deterministic;
* ``serving``: open-loop Poisson arrivals of the 80/20 PR-Nibble / HK-PR mix
  on the scale-26 graph at 1k-50k requests/s (and 100/s, below capacity);
* ``cpu_baseline`` and ``cpu_all_cores``: the oracle on the host cores, one
  core on the step, and one process per core on the many-seed and serving
  workloads.

  python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--mode atomic|det]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import queue
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE, GRAPH_SEED = 22, 2
PR = dict(alpha=0.01, eps=1e-7)
NB = dict(T=20, eps=1e-7)
HK = dict(t=10.0, N=20, eps=1e-7)
RH = dict(t=10.0, K=10, n_walks=1_000_000, rng_seed=7)
WORKLOAD = (f"R-MAT scale {SCALE} (ef 16, a=0.57 b=c=0.19, seed {GRAPH_SEED}), one seed: "
            "PR-Nibble a=0.01 eps=1e-7, Nibble T=20 eps=1e-7, HK-PR t=10 N=20 eps=1e-7, "
            "rand-HK-PR t=10 K=10 1e6 walks Philox 7; sweep cut after each")

# 1024 seeds, batched vs one per call (the many-seed workload)
MANY = dict(scale=24, graph_seed=4, seeds=1024, seed_stream=4, alpha=0.01, eps_lo=-8.0,
            eps_hi=-5.0)
# 8 seeds of the 2.1-billion-entry graph, both modes, two eps
C3 = dict(scale=26, graph_seed=3, seeds=8, seed_stream=3, alpha=0.01, eps=(1e-7, 1e-8),
          modes=("atomic", "det"))
# the serving mix on the scale-26 graph
SERVE = dict(scale=26, graph_seed=3, rates=(100, 1000, 5000, 10000, 20000, 50000),
             requests=600, offered_s=2.0, arrival_seed=5, mix_seed=5, hk_eps=1e-7,
             mem_budget=40 << 30, max_batch=32)
CPU_BUDGET_S = dict(step=0.0, many=10.0, serving=15.0)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(off, col, rank):
    """Rank 0 takes vertex 0's highest-degree neighbour; rank r > 0 the r-th
    degree->=2 vertex of the seeded sampler (independent problems)."""
    from paper_1604_07515_gb300 import inputs
    if rank == 0:
        return inputs.config1_seed(off, col)
    return int(inputs.seeds_deg2(off, rank, 2)[rank - 1])


def reduce_ranks(maxed, summed, world, device):
    """Max over ranks of `maxed` (times) and sum over ranks of `summed`
    (work); identity when world == 1."""
    if world == 1:
        return list(maxed), list(summed)
    import torch
    import torch.distributed as dist
    a = torch.tensor(list(maxed), dtype=torch.float64, device=device)
    b = torch.tensor(list(summed), dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.mark = 0  # samples taken before the timed region began

    def start(self, wait_s: float = 5.0):
        """Starts nvidia-smi and returns once its first sample is in (or it
        has exited, or wait_s passed), so that the region timed after this
        call is covered from its start; that first sample is not counted."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while (not self.lines and self.proc.poll() is None
               and time.perf_counter() - t0 < wait_s):
            time.sleep(0.005)
        self.mark = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.mark:]
        in_region = bool(lines)
        if not in_region:  # region shorter than the sampling period: the sample just before it
            lines = self.lines[-1:]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm) if in_region else 0}


ALGOS = ("prnibble", "nibble", "hkpr", "rand_hkpr")


def run_algo(lgc, g, x, name, mode):
    if name == "prnibble":
        return lgc.prnibble(g, x, PR["alpha"], PR["eps"], mode=mode)
    if name == "nibble":
        return lgc.nibble(g, x, NB["T"], NB["eps"], mode=mode)
    if name == "hkpr":
        return lgc.hkpr(g, x, HK["t"], HK["N"], HK["eps"], mode=mode)
    return lgc.rand_hkpr(g, x, RH["t"], RH["K"], RH["n_walks"], RH["rng_seed"])


def one_step(lgc, g, x, mode, events=None):
    """The hot path for one seed; returns (pushed_edges, clusters, d2h_bytes).
    With `events` (a list), records one CUDA event before each diffusion and
    one at the end, for the per-diffusion split."""
    import torch
    pushed, clusters, d2h = 0, 0, 0
    per = []
    for name in STEP_ALGOS:
        if events is not None:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(torch.cuda.current_stream())
            events.append(ev)
        p, st = run_algo(lgc, g, x, name, mode)
        c = lgc.sweep(g, p)
        pushed += st.pushed_edges
        per.append(st.pushed_edges)
        clusters += 1
        d2h += 0 if p.on_device else 12 * p.nnz + 4 * c.size
    if events is not None:
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(torch.cuda.current_stream())
        events.append(ev)
        events.append(per)
    return pushed, clusters, d2h


def hk_terms(t, eps):
    """Taylor degree N for serving HK-PR: the smallest N whose Poisson(t)
    tail P(k > N) is at most eps, capped at ceil(2 t ln(1/eps))."""
    import math
    cap = math.ceil(2.0 * t * math.log(1.0 / eps))
    term = math.exp(-t)
    cdf = term
    k = 0
    while 1.0 - cdf > eps and k < cap:
        k += 1
        term *= t / k
        cdf += term
    return max(1, min(k, cap))


def many_seed_list(inputs, off):
    seeds = inputs.seeds_deg2(off, MANY["seeds"], MANY["seed_stream"])
    eps = inputs.eps_loguniform(MANY["seeds"], MANY["seed_stream"], MANY["eps_lo"],
                                MANY["eps_hi"])
    return seeds, eps


def serving_mix(inputs, off, count):
    """(kind, seed, params) of the serving mix: 80% PR-Nibble (alpha 0.01,
    eps log-uniform [1e-8, 1e-5]), 20% HK-PR (t log-uniform [3, 30], eps
    1e-7, N from the Poisson tail); seeds uniform among degree >= 2."""
    import numpy as np
    s = SERVE["mix_seed"]
    seeds = inputs.seeds_deg2(off, count, s)
    eps = inputs.eps_loguniform(count, s, -8.0, -5.0)
    ts = 10.0 ** (np.log10(3.0) + (np.log10(30.0) - np.log10(3.0)) * inputs.uniform(s + 1, count))
    pr = inputs.uniform(s + 2, count) < 0.8
    out = []
    for i in range(count):
        if pr[i]:
            out.append(("pr", int(seeds[i]), dict(alpha=0.01, eps=float(eps[i]))))
        else:
            t = float(ts[i])
            out.append(("hkpr", int(seeds[i]), dict(t=t, N=hk_terms(t, SERVE["hk_eps"]),
                                                    eps=SERVE["hk_eps"])))
    return out


# ---------------------------------------------------------------------------
# The oracle on the host cores (reported baselines, not targets).  Everything
# here runs before the first CUDA call, so the worker processes are forked
# from a process that has no GPU context; they share the graphs' pages.
# ---------------------------------------------------------------------------
def cpu_oracle_step(off, col, x, k):
    """The oracle on one diffusion (cycled by k) + its sweep; returns pushed edges."""
    import oracle
    which = k % 4
    if which == 0:
        r = oracle.prnibble(off, col, x, PR["alpha"], PR["eps"])
    elif which == 1:
        r = oracle.nibble(off, col, x, NB["T"], NB["eps"])
    elif which == 2:
        r = oracle.hkpr(off, col, x, HK["t"], HK["N"], HK["eps"])
    else:
        r = oracle.rand_hkpr(off, col, x, RH["t"], RH["K"], RH["n_walks"], RH["rng_seed"])
    oracle.sweep(off, col, r.idx, r.val)
    return r.pushed_edges


_SHARED = {}  # graphs and work lists handed to forked workers


def _oracle_worker(kind, k, P, out_q):
    """Worker k of P: runs work items k, k + P, ... of _SHARED[kind] one
    after another and reports each one's (pushed edges, seconds)."""
    import oracle
    off, col, items = _SHARED[kind]
    for i in range(k, len(items), P):
        a, seed, prm = items[i]
        t0 = time.perf_counter()
        if a == "pr":
            r = oracle.prnibble(off, col, seed, prm["alpha"], prm["eps"])
        else:
            r = oracle.hkpr(off, col, seed, prm["t"], prm["N"], prm["eps"])
        oracle.sweep(off, col, r.idx, r.val)
        out_q.put((k, r.pushed_edges, time.perf_counter() - t0))


def cpu_all_cores(kind, budget_s):
    """One forked oracle process per host core over the work list; after
    budget_s seconds the processes still running are stopped and the
    completed clusters counted (aggregate clusters/s over all cores)."""
    P = os.cpu_count() or 1
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(kind, k, P, q), daemon=True)
             for k in range(P)]
    t0 = time.perf_counter()
    for p in procs:
        p.start()
    done = []
    while time.perf_counter() - t0 < budget_s:
        try:
            done.append(q.get(timeout=0.05))
        except queue.Empty:
            if not any(p.is_alive() for p in procs):
                break
    wall = time.perf_counter() - t0
    for p in procs:
        if p.is_alive():
            p.kill()
        p.join()
    while True:  # results that arrived before the stop
        try:
            done.append(q.get_nowait())
        except queue.Empty:
            break
    secs = [d[2] for d in done]
    edges = sum(d[1] for d in done)
    return {"clusters": len(done), "wall_s": wall, "cores": P,
            "clusters_per_s": len(done) / wall, "edges_per_s": edges / wall,
            "per_cluster_s_mean": statistics.mean(secs) if secs else None,
            "per_cluster_s_median": statistics.median(secs) if secs else None,
            "unfinished_workers": sum(1 for k in range(P) if not any(d[0] == k for d in done))}


def host_cpu():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        nproc = int(subprocess.run(["nproc"], capture_output=True, text=True,
                                   timeout=10).stdout.strip())
    except Exception:
        nproc = os.cpu_count()
    return {"lscpu_model": model, "nproc": nproc}


# ---------------------------------------------------------------------------
# GPU measurements beside the headline step
# ---------------------------------------------------------------------------
def measure_many(lgc, inputs, torch, ctx, g, off):
    """1024 PR-Nibble + sweep clusters three ways: one lgc_prnibble_batch +
    lgc_sweep_batch call for all seeds, one lgc_prnibble + lgc_sweep per
    seed, and all at once through the request loop (lgc_submit / lgc_wait,
    host results); device-resident results for the first two."""
    seeds, eps = many_seed_list(inputs, off)
    a = MANY["alpha"]
    B = len(seeds)
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
    # warm-up of both paths: the whole batch once, so that the device pool
    # holds the batch's memory (as in a long-running process) before timing
    ps, _ = lgc.prnibble_batch(g, seeds, a, eps, mode=MODE)
    lgc.sweep_batch(g, ps)
    del ps
    p, _ = lgc.prnibble(g, int(seeds[0]), a, float(eps[0]), mode=MODE)
    lgc.sweep(g, p)
    del p
    torch.cuda.synchronize()

    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    ps, sts = lgc.prnibble_batch(g, seeds, a, eps, mode=MODE)
    cs = lgc.sweep_batch(g, ps)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    e_b = sum(st.pushed_edges for st in sts)
    rounds = [st.rounds for st in sts]
    del ps, cs
    # device memory the pool grew by during the batch (the pool keeps it)
    pool_gb = max(0.0, (free0 - torch.cuda.mem_get_info()[0]) / 1e9)

    t0 = time.perf_counter()
    e_s = 0
    for b in range(B):
        p, st = lgc.prnibble(g, int(seeds[b]), a, float(eps[b]), mode=MODE)
        lgc.sweep(g, p)
        e_s += st.pushed_edges
        del p
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)
    reqs = [lgc.make_request(lgc.ALGO_PRNIBBLE, int(seeds[b]), True, alpha=a, eps=float(eps[b]),
                             mode=MODE) for b in range(B)]
    for tk in [lgc.submit(ctx, g, reqs[b]) for b in range(8)]:  # warm the loop
        lgc.wait(ctx, tk)
    t0 = time.perf_counter()
    pending = [lgc.submit(ctx, g, r) for r in reqs]
    e_q = sum(lgc.wait(ctx, tk)["stats"]["pushed_edges"] for tk in pending)
    tq = time.perf_counter() - t0
    return {"workload": (f"R-MAT scale {MANY['scale']} (seed {MANY['graph_seed']}), {B} PR-Nibble "
                         f"seeds (degree >= 2, stream {MANY['seed_stream']}), alpha {a}, eps "
                         f"log-uniform [1e{int(MANY['eps_lo'])}, 1e{int(MANY['eps_hi'])}], + sweep "
                         f"each; batched: one lgc_prnibble_batch + lgc_sweep_batch call of all "
                         f"{B}, timed after one untimed call of the same batch"),
            "clusters": B, "pushed_edges": e_b, "max_rounds": max(rounds),
            "batched": {"clusters_per_s": B / tb, "edges_per_s": e_b / tb, "s": tb,
                        "device_pool_growth_gb": pool_gb},
            "per_seed": {"clusters_per_s": B / ts, "edges_per_s": e_s / ts, "s": ts},
            "request_loop": {"clusters_per_s": B / tq, "edges_per_s": e_q / tq, "s": tq,
                             "resident": SERVE["max_batch"]},
            "speedup_batched_vs_per_seed": ts / tb}


def measure_config3(lgc, inputs, torch, ctx, g, off):
    """PR-Nibble + sweep from 8 seeds (degree >= 2) of the scale-26 graph,
    eps 1e-7 and 1e-8, atomic and deterministic, device-resident results;
    CUDA events on the context's stream around each mode/eps group."""
    seeds = inputs.seeds_deg2(off, C3["seeds"], C3["seed_stream"])
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
    stream = torch.cuda.current_stream()
    out = {"workload": (f"R-MAT scale {C3['scale']} (seed {C3['graph_seed']}, "
                        f"{len(off) - 1} vertices), {C3['seeds']} PR-Nibble seeds (degree >= 2, "
                        f"stream {C3['seed_stream']}), alpha {C3['alpha']}, + sweep each"),
           "runs": []}
    for mode in C3["modes"]:
        for eps in C3["eps"]:
            p, _ = lgc.prnibble(g, int(seeds[0]), C3["alpha"], eps, mode=mode)  # warm-up
            lgc.sweep(g, p)
            del p
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            edges, rounds = 0, []
            for x in seeds:
                p, st = lgc.prnibble(g, int(x), C3["alpha"], eps, mode=mode)
                lgc.sweep(g, p)
                edges += st.pushed_edges
                rounds.append(st.rounds)
                del p
            b.record(stream)
            b.synchronize()
            s = a.elapsed_time(b) / 1e3
            out["runs"].append({"mode": mode, "eps": eps, "clusters": len(seeds),
                                "pushed_edges": edges, "rounds_max": max(rounds), "s": s,
                                "edges_per_s": edges / s, "clusters_per_s": len(seeds) / s})
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)
    return out


def occupancy(res, t_submit):
    """Queued and admitted requests at each arrival instant, from the
    library's own submission, start and end times."""
    import numpy as np
    sub = np.array([r["submit_s"] for r in res])
    st = np.array([r["start_s"] for r in res])
    en = np.array([r["end_s"] for r in res])
    q, a = [], []
    for t in sub:
        q.append(int(((sub <= t) & (st > t)).sum()))
        a.append(int(((st <= t) & (en > t)).sum()))
    return {"queued_mean": float(np.mean(q)), "queued_max": int(np.max(q)),
            "admitted_mean": float(np.mean(a)), "admitted_max": int(np.max(a)),
            "wait_p50_ms": float(np.percentile(st - sub, 50) * 1e3),
            "service_p50_ms": float(np.percentile(en - st, 50) * 1e3)}


def measure_serving(lgc, inputs, torch, ctx, g, off):
    """Open-loop Poisson arrivals through lgc_submit / lgc_wait of the serving
    mix; latency = completion - submission (library clock)."""
    import numpy as np
    mix = serving_mix(inputs, off, SERVE["requests"])
    reqs = []
    for kind, seed, prm in mix:
        if kind == "pr":
            reqs.append(lgc.make_request(lgc.ALGO_PRNIBBLE, seed, True, mode=MODE, **prm))
        else:
            reqs.append(lgc.make_request(lgc.ALGO_HKPR, seed, True, mode=MODE, **prm))
    ctx.set_option(lgc.OPT_SERVE_MEM_BUDGET, SERVE["mem_budget"])
    try:
        ctx.set_option(lgc.OPT_SERVE_MAX_BATCH, SERVE["max_batch"])
    except lgc.LgcError:
        pass  # the loop is already running with it
    for tk in [lgc.submit(ctx, g, reqs[i]) for i in range(8)]:  # warm the loop
        lgc.wait(ctx, tk)
    out = []
    for rate in SERVE["rates"]:
        # the first R requests of the mix: fewer at rates below capacity so
        # that the offered load lasts about offered_s seconds
        R = min(SERVE["requests"], max(50, int(SERVE["offered_s"] * rate)))
        gaps = -np.log(1.0 - inputs.uniform(SERVE["arrival_seed"] + rate, R)) / rate
        arrive = np.cumsum(gaps)
        # this thread submits at the arrival times; a collector thread takes
        # the results with the blocking lgc_wait
        tickets = queue.Queue()
        res, done_edges = [], [0]

        def collect():
            for _ in range(R):
                r = lgc.wait(ctx, tickets.get())
                res.append(r)
                done_edges[0] += r["stats"]["pushed_edges"]

        th = threading.Thread(target=collect)
        t0 = time.perf_counter()
        th.start()
        for i in range(R):
            dt = arrive[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.put(lgc.submit(ctx, g, reqs[i]))
        th.join()
        wall = time.perf_counter() - t0
        lat_ms = np.sort(np.asarray([r["end_s"] - r["submit_s"] for r in res])) * 1e3
        line = {"rate_per_s": rate, "requests": R, "clusters_per_s": R / wall,
                "edges_per_s": done_edges[0] / wall,
                "p50_ms": float(np.percentile(lat_ms, 50)),
                "p99_ms": float(np.percentile(lat_ms, 99)),
                "offered_s": float(arrive[-1]), "wall_s": wall,
                "failed": sum(1 for r in res if r["status"] != 0)}
        line.update(occupancy(res, arrive))
        out.append(line)
    return {"workload": (f"R-MAT scale {SERVE['scale']} (seed {SERVE['graph_seed']}); Poisson "
                         f"arrivals (seed {SERVE['arrival_seed']}), up to {SERVE['requests']} "
                         f"requests per rate ({SERVE['offered_s']:.0f} s of offered load at low "
                         "rates): 80% PR-Nibble alpha 0.01 eps log-uniform [1e-8, 1e-5], 20% "
                         "HK-PR t log-uniform [3, 30] eps 1e-7 (N from the Poisson tail); sweep "
                         f"each; memory budget {SERVE['mem_budget'] >> 30} GB, "
                         f"{SERVE['max_batch']} resident"),
            "rates": out}


# ---------------------------------------------------------------------------
# Roofline bookkeeping.  DRAM bytes of the atomic pull rounds' gathers
# (pull_light_fx_kernel + pull_heavy_fx_kernel) per pull round of the HK-PR
# diffusion of the step, from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum, -k on those kernels, the first two pull rounds) per
# gather configuration, and the SHA-256 of the gathers' source at capture
# time (the stretches of the sources that make up the two kernels and the
# device code they call: file, first line's text, the text that ends the
# stretch; None = the whole file): when it differs, or the graph's tuned
# configuration was not captured, the figure does not describe the timed
# kernels and `traffic` is null.
# ---------------------------------------------------------------------------
_CSRC = "paper_1604_07515_gb300/csrc/"
PULL_TRAFFIC = {"sources": [
                    (_CSRC + "diffuse.cu", "// Adds every thread's count n into *counter",
                     "__device__ inline void count_inserted("),
                    (_CSRC + "diffuse.cu", "__device__ inline bool pull_member(double s)",
                     "__global__ void pull_scatter_kernel("),
                    (_CSRC + "diffuse.cu", "__device__ inline bool pull_qualifies(",
                     "// Deterministic pull, vertices of degree 1..kPullLight"),
                    (_CSRC + "diffuse.cu", "// Writes a heavy vertex's gathered value",
                     "// The ordered fold acc <- RN(acc + s_k)"),
                    (_CSRC + "diffuse.cu", "__device__ inline int round_scale(",
                     "// edgeMap, deterministic mode."),
                    (_CSRC + "fx128.cuh", None, None),
                    (_CSRC + "common.cuh", "namespace lgc {", "// Host-side objects"),
                    (_CSRC + "common.cuh", "// Work item of a pull round", "struct lgc_graph {"),
                    (_CSRC + "common.cuh", "// A pull round handles vertices of degree",
                     "}  // namespace lgc")],
                "sha256": "d70cee2a7faab3841c6347d5dd646370d3072d1abcb34862fa347cb492d939cc",
                # bytes per pull round (light + heavy gather), by "degree bin, edges per
                # lane per batch, lanes per item, bytes per gathered share"
                "per_round": {"256,16,32,8": 819.3e6, "256,16,16,8": 819.3e6,
                              "256,8,16,8": 820.1e6, "256,8,32,16": 995.2e6,
                              "128,16,32,8": 818.6e6, "128,16,16,8": 818.9e6,
                              "128,8,16,8": 819.6e6, "64,16,32,8": 806.5e6},
                # ncu --set full of one heavy gather launch (bin 256, shape (16, 32, 8 B)):
                # the units that bind it, as fractions of their peaks
                "heavy_gather_full": {"kernel": "pull_heavy_fx_kernel<16, 32, double>",
                                      "duration_us": 327.6, "dram_gb": 0.454,
                                      "dram_frac": 0.175, "lts_throughput_frac": 0.285,
                                      "l1tex_throughput_frac": 0.756, "issue_active_frac": 0.496,
                                      "l2_hit_rate": 0.769}}


def sources_sha(stretches):
    """SHA-256 of the given source stretches (see PULL_TRAFFIC); None if a
    stretch's bounds are not found."""
    h = hashlib.sha256()
    for path, begin, end in stretches:
        with open(os.path.join(ROOT, path), encoding="utf-8") as f:
            text = f.read()
        if begin is not None:
            a = text.find(begin)
            b = text.find(end, a + 1) if a >= 0 else -1
            if a < 0 or b < 0:
                return None
            text = text[a:b]
        h.update(text.encode("utf-8"))
    return h.hexdigest()


# bytes of the per-step inputs handed to the library (seed + parameter structs)
H2D_BYTES_PER_STEP = 4 * 4 + 32 + 24 + 24 + 32


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1604_07515_gb300 import inputs
    off, col = inputs.rmat(SCALE, seed=GRAPH_SEED)
    x = rank_seed(off, col, 0)
    for k in range(args.warmup):
        cpu_oracle_step(off, col, x, k)
    t0 = time.perf_counter()
    pushed = 0
    for k in range(args.steps):
        pushed += cpu_oracle_step(off, col, x, k)
    dt = time.perf_counter() - t0
    v = pushed / dt
    line = {
        "impl": "reference", "metric": "pushed_edges_per_s", "value": v, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": MODE, "l2": "graph > L2"},
        "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": "each step runs one of the four diffusions (cycled) "
                                   "and its sweep cut, single-threaded"},
        "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(lgc, torch, ctx, g, x, mode, steps, flush, stream, barrier):
    """K device-timed steps (L2 flushed before each, not timed); returns
    (total ms, pushed, clusters, per-diffusion split, launches)."""
    step_ms, pushed, clusters = [], 0, 0
    split = {a: {"ms": 0.0, "edges": 0} for a in STEP_ALGOS}
    launches0 = ctx.launch_count()
    for _ in range(steps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        evs = []
        a.record(stream)
        pe, cl, _ = one_step(lgc, g, x, mode, evs)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        pushed += pe
        clusters += cl
        for i, name in enumerate(STEP_ALGOS):
            split[name]["ms"] += evs[i].elapsed_time(evs[i + 1]) / steps
            split[name]["edges"] += evs[-1][i] / steps
    barrier()
    return sum(step_ms), pushed, clusters, split, ctx.launch_count() - launches0


# One named workload, run a given number of times (for ncu captures: the
# capture selects launches with -k / -s / -c; nothing here is timed).
CASES = {
    "batch256_rmat22": "lgc_prnibble_batch of 256 seeds (degree >= 2, stream 4) of R-MAT scale 22 "
                       "(seed 2), eps log-uniform [1e-7, 1e-5], alpha 0.01, atomic",
    "batch1024_rmat24": "lgc_prnibble_batch + lgc_sweep_batch of the 1024 many-seed seeds of R-MAT "
                        "scale 24 (seed 4), atomic",
    "hkpr_serving_rmat26": "the HK-PR request of the serving mix with the largest t, alone, on "
                           "R-MAT scale 26 (seed 3), atomic",
    "hkpr_serving_rmat24": "the HK-PR request with the largest t of the serving mix drawn on "
                           "R-MAT scale 24 (seed 4), alone, atomic",
}


def run_case(name, reps):
    import torch
    from paper_1604_07515_gb300 import inputs, lgc
    if name == "batch256_rmat22":
        off, col = inputs.rmat(22, seed=2)
    elif name in ("batch1024_rmat24", "hkpr_serving_rmat24"):
        off, col = inputs.rmat(MANY["scale"], seed=MANY["graph_seed"])
    else:
        off, col = inputs.rmat(SERVE["scale"], seed=SERVE["graph_seed"])
    ctx = lgc.Context(0, torch.cuda.current_stream())
    g = lgc.Graph(ctx, off, col)
    g.autotune()  # as the bench does before timing
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
    if name.startswith("hkpr_serving"):
        big = max((m for m in serving_mix(inputs, off, SERVE["requests"]) if m[0] == "hkpr"),
                  key=lambda m: m[2]["t"])
    for _ in range(reps):
        t0 = time.perf_counter()
        if name == "batch256_rmat22":
            seeds = inputs.seeds_deg2(off, 256, 4)
            ps, sts = lgc.prnibble_batch(g, seeds, 0.01, inputs.eps_loguniform(256, 4, -7.0, -5.0))
            edges = sum(s.pushed_edges for s in sts)
        elif name == "batch1024_rmat24":
            seeds, eps = many_seed_list(inputs, off)
            ps, sts = lgc.prnibble_batch(g, seeds, MANY["alpha"], eps)
            lgc.sweep_batch(g, ps)
            edges = sum(s.pushed_edges for s in sts)
        else:
            p, st = lgc.hkpr(g, big[1], big[2]["t"], big[2]["N"], big[2]["eps"])
            lgc.sweep(g, p)
            edges = st.pushed_edges
        torch.cuda.synchronize()
        print(f"{name}: {time.perf_counter() - t0:.4f} s, {edges} pushed edges", flush=True)
    g.close()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # default: 80 timed steps (about 1.2 s, several clock samples); the
    # reference arm's oracle, about 10 s per cycle of the four diffusions, 8
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="atomic", choices=["atomic", "det"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-many", action="store_true",
                    help="skip the many-seed, scale-26 and serving measurements")
    ap.add_argument("--no-det", action="store_true", help="skip the deterministic-mode step")
    ap.add_argument("--pull-shape", default="",
                    help="heavy pull gather shape 'batch,lanes,share_bytes[,degree_bin]' "
                         "instead of the graph's autotuned one (e.g. 16,32,8,256)")
    ap.add_argument("--algos", default=",".join(ALGOS),
                    help="comma-separated subset of the step (for profiling one diffusion)")
    ap.add_argument("--case", default="", choices=[""] + list(CASES),
                    help="run one named workload --steps times and exit (for profiling): "
                         + "; ".join(f"{k}: {v}" for k, v in CASES.items()))
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 8 if args.impl == "reference" else 80
    global MODE, STEP_ALGOS
    MODE = args.mode
    STEP_ALGOS = tuple(a for a in args.algos.split(",") if a)
    if not STEP_ALGOS or any(a not in ALGOS for a in STEP_ALGOS):
        ap.error(f"--algos takes a subset of {','.join(ALGOS)}")
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args.case, args.steps)

    rank, world, local = dist_env()
    from paper_1604_07515_gb300 import inputs
    off, col = inputs.rmat(SCALE, seed=GRAPH_SEED)
    x = rank_seed(off, col, rank)
    solo = rank == 0 and world == 1
    big = solo and not args.no_many
    off24 = col24 = off26 = col26 = None
    if big:
        off24, col24 = inputs.rmat(MANY["scale"], seed=MANY["graph_seed"])
        off26, col26 = inputs.rmat(C3["scale"], seed=C3["graph_seed"])

    # ---- the oracle on the host, before any CUDA call (forked workers) ----
    cpu = cpu_all = None
    if solo and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        cp = 0
        for k in range(4):  # one of each diffusion and its sweep
            cp += cpu_oracle_step(off, col, x, k)
        dt = time.perf_counter() - t0
        cpu = {"value": cp / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": "the four diffusions of one step and their sweeps, once each, "
                         "single-threaded on the host"}
        cpu.update(host_cpu())
        if big:
            seeds, eps = many_seed_list(inputs, off24)
            _SHARED["many"] = (off24, col24, [("pr", int(s), dict(alpha=MANY["alpha"], eps=float(e)))
                                              for s, e in zip(seeds, eps)])
            _SHARED["serving"] = (off26, col26, serving_mix(inputs, off26, SERVE["requests"]))
            cpu_all = {"kind": "oracle", **host_cpu(),
                       "many_seeds": cpu_all_cores("many", CPU_BUDGET_S["many"]),
                       "serving": cpu_all_cores("serving", CPU_BUDGET_S["serving"]),
                       "sample": (f"one oracle process per host core over the many-seed list "
                                  f"(scale 24) for {CPU_BUDGET_S['many']:.0f} s and the serving "
                                  f"mix (scale 26) for {CPU_BUDGET_S['serving']:.0f} s; "
                                  "completed PR-Nibble/HK-PR + sweep clusters counted")}
            _SHARED.clear()

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1604_07515_gb300 import lgc

    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ctx = lgc.Context(dev, stream)
    g = lgc.Graph(ctx, off, col)
    if args.pull_shape:
        fixed = tuple(int(v) for v in args.pull_shape.split(","))
        pull_shape = fixed[:3]
        for opt, v in zip((lgc.OPT_PULL_BATCH, lgc.OPT_PULL_GROUP, lgc.OPT_PULL_SHARE),
                          pull_shape):
            ctx.set_option(opt, v)
        if len(fixed) > 3:
            g.set_pull_light(fixed[3])
    else:
        pull_shape = g.autotune()  # launch-shape tuning on this graph, before any timing
    pull_light = g.pull_light()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident results: the kernel-side number ----
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
    for _ in range(args.warmup):
        one_step(lgc, g, x, MODE)
    ctx.set_option(lgc.OPT_PROFILE, 1)
    ctx.profile_reset()
    clocks = ClockSampler(dev)
    barrier()
    clocks.start()
    total_ms, pushed, clusters, split, launches = timed_steps(
        lgc, torch, ctx, g, x, MODE, args.steps, flush, stream, barrier)
    clk = clocks.stop()
    ctx.set_option(lgc.OPT_PROFILE, 0)
    prof = {lgc.PROF_NAMES[k]: ctx.profile(k) for k in lgc.PROF_NAMES}
    (total_ms,), (pushed, clusters) = reduce_ranks([total_ms], [pushed, clusters], world, "cuda")
    value = pushed / (total_ms / 1e3)

    # ---- end to end through the public API with host buffers ----
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)
    one_step(lgc, g, x, MODE)
    barrier()
    e_pushed, d2h, e2e_s = 0, 0, 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        pe, _, db = one_step(lgc, g, x, MODE)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - s0
        e_pushed += pe
        d2h += db
    (e2e_s,), (e_pushed,) = reduce_ranks([e2e_s], [e_pushed], world, "cuda")
    e2e_value = e_pushed / e2e_s

    # ---- the same step in deterministic mode ----
    det = None
    if solo and not args.no_det and MODE == "atomic":
        ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
        kd = max(3, args.steps // 4)
        for _ in range(2):
            one_step(lgc, g, x, "det")
        d_ms, d_pushed, d_cl, d_split, _ = timed_steps(lgc, torch, ctx, g, x, "det", kd, flush,
                                                       stream, barrier)
        det = {"steps": kd, "ms_per_step": d_ms / kd, "edges_per_s": d_pushed / (d_ms / 1e3),
               "clusters_per_s": d_cl / (d_ms / 1e3),
               "per_diffusion_ms": {k: v["ms"] for k, v in d_split.items()}}
        ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)

    # ---- many seeds (scale 24), then the scale-26 graph (rank 0, one GPU) ----
    many = c3 = serving = None
    if big:
        g.close()
        del flush
        gm = lgc.Graph(ctx, off24, col24)
        gm.autotune()
        many = measure_many(lgc, inputs, torch, ctx, gm, off24)
        gm.close()
        torch.cuda.synchronize()
        g26 = lgc.Graph(ctx, off26, col26)
        g26.autotune()
        c3 = measure_config3(lgc, inputs, torch, ctx, g26, off26)
        serving = measure_serving(lgc, inputs, torch, ctx, g26, off26)
        g26.close()

    # ---- roofline of the dominant kernel scope ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    achieved = (d["bytes"] / (d["ms"] / 1e3)) / 1e9 if d["ms"] > 0 else 0.0
    traffic = None
    if (dname == "edgemap_pull" and MODE == "atomic" and STEP_ALGOS == ALGOS
            and PULL_TRAFFIC["sha256"] == sources_sha(PULL_TRAFFIC["sources"])):
        traffic = PULL_TRAFFIC["per_round"].get(
            ",".join(str(v) for v in (pull_light,) + tuple(pull_shape)))
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": traffic, "launches": d["launches"],
                "ncu_units": PULL_TRAFFIC["heavy_gather_full"] if traffic is not None else None,
                "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
                "alg_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "share_of_step": d["ms"] / total_ms if total_ms else None}

    if rank == 0:
        line = {
            "metric": "pushed_edges_per_s", "value": value, "unit": "edges/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if STEP_ALGOS == ALGOS
                       else WORKLOAD + f" (only: {','.join(STEP_ALGOS)})", "mode": MODE,
                       "l2": "inputs larger than L2 and L2 flushed between steps",
                       "parallelism": f"replicas{world}", "pull_shape": list(pull_shape),
                       "pull_light": pull_light},
            "clusters_per_s": clusters / (total_ms / 1e3),
            "pushed_edges_per_step": pushed / args.steps / max(1, world),
            "roofline": roofline, "kernels": prof,
            "per_diffusion": {k: {"ms": v["ms"], "edges": v["edges"],
                                  "edges_per_s": v["edges"] / (v["ms"] / 1e3) if v["ms"] else None}
                              for k, v in split.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "edges/s",
                    "h2d_bytes_per_step": H2D_BYTES_PER_STEP,
                    "d2h_bytes_per_step": d2h // max(1, args.steps)},
            "clocks": clk, "gpu_launches": launches,
            "det_step": det, "many_seeds": many, "config3": c3, "serving": serving,
            "cpu_all_cores": cpu_all,
        }
        print(json.dumps(line), flush=True)
    if not big:
        g.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


MODE = "atomic"
STEP_ALGOS = ALGOS

if __name__ == "__main__":
    sys.exit(main())

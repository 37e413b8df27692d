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

  python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--mode atomic|det]
"""
from __future__ import annotations

import argparse
import json
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


def run_algo(lgc, g, x, name):
    if name == "prnibble":
        return lgc.prnibble(g, x, PR["alpha"], PR["eps"], mode=MODE)
    if name == "nibble":
        return lgc.nibble(g, x, NB["T"], NB["eps"], mode=MODE)
    if name == "hkpr":
        return lgc.hkpr(g, x, HK["t"], HK["N"], HK["eps"], mode=MODE)
    return lgc.rand_hkpr(g, x, RH["t"], RH["K"], RH["n_walks"], RH["rng_seed"])


def one_step(lgc, g, x, events=None):
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
        p, st = run_algo(lgc, g, x, name)
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


# ---------------------------------------------------------------------------
# Batched vs one seed per call (PR-Nibble + sweep), and the request loop.
# Both on R-MAT scale 24 (16.8M vertices, edge factor 16, seed 4) with seeds
# drawn uniformly among degree >= 2 vertices; the serving mix follows the
# paper's serving-style use (many local clusterings on one resident graph).
# ---------------------------------------------------------------------------
MANY = dict(scale=24, graph_seed=4, seeds=1024, seed_stream=4, alpha=0.01, eps_lo=-8.0,
            eps_hi=-5.0, chunk=256)
SERVE = dict(rates=(50, 100, 1000, 5000, 10000, 20000, 50000), requests=1000, offered_s=4.0,
             arrival_seed=5,
             hk_eps=1e-7, mem_budget=40 << 30, max_batch=32)


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


def measure_many(lgc, inputs, torch, ctx, g, off):
    """1024 PR-Nibble + sweep clusters three ways: lgc_prnibble_batch and
    lgc_sweep_batch (in chunks), one seed per call (lgc_prnibble, lgc_sweep),
    and all at once through the request loop (lgc_submit / lgc_wait, host
    results); device-resident results for the first two."""
    seeds = inputs.seeds_deg2(off, MANY["seeds"], MANY["seed_stream"])
    eps = inputs.eps_loguniform(MANY["seeds"], MANY["seed_stream"], MANY["eps_lo"], MANY["eps_hi"])
    a = MANY["alpha"]
    ch = MANY["chunk"]
    # warm-up of both paths
    ps, _ = lgc.prnibble_batch(g, seeds[:8], a, eps[:8], mode=MODE)
    lgc.sweep_batch(g, ps)
    p, _ = lgc.prnibble(g, int(seeds[0]), a, float(eps[0]), mode=MODE)
    lgc.sweep(g, p)
    torch.cuda.synchronize()

    t0 = time.perf_counter()
    e_b = 0
    for i in range(0, len(seeds), ch):
        ps, sts = lgc.prnibble_batch(g, seeds[i:i + ch], a, eps[i:i + ch], mode=MODE)
        lgc.sweep_batch(g, ps)
        e_b += sum(st.pushed_edges for st in sts)
        del ps
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0

    t0 = time.perf_counter()
    e_s = 0
    for b in range(len(seeds)):
        p, st = lgc.prnibble(g, int(seeds[b]), a, float(eps[b]), mode=MODE)
        lgc.sweep(g, p)
        e_s += st.pushed_edges
        del p
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    # all requests at once through the request loop (worker contexts run the
    # single-seed diffusions side by side on their own streams)
    ctx.set_option(lgc.OPT_SERVE_MEM_BUDGET, SERVE["mem_budget"])
    try:
        ctx.set_option(lgc.OPT_SERVE_MAX_BATCH, SERVE["max_batch"])
    except lgc.LgcError:
        pass  # the loop is already running
    reqs = [lgc.make_request(lgc.ALGO_PRNIBBLE, int(seeds[b]), True, alpha=a, eps=float(eps[b]),
                             mode=MODE) for b in range(len(seeds))]
    for tk in [lgc.submit(ctx, g, reqs[b]) for b in range(8)]:  # warm the workers
        lgc.wait(ctx, tk)
    t0 = time.perf_counter()
    pending = [lgc.submit(ctx, g, r) for r in reqs]
    e_q = sum(lgc.wait(ctx, tk)["stats"]["pushed_edges"] for tk in pending)
    tq = time.perf_counter() - t0
    B = len(seeds)
    return {"workload": (f"R-MAT scale {MANY['scale']} (seed {MANY['graph_seed']}), {B} PR-Nibble "
                         f"seeds (degree >= 2, stream {MANY['seed_stream']}), alpha {a}, eps "
                         f"log-uniform [1e{int(MANY['eps_lo'])}, 1e{int(MANY['eps_hi'])}], + sweep "
                         f"each; batched in chunks of {ch}"),
            "clusters": B, "pushed_edges": e_b,
            "batched": {"clusters_per_s": B / tb, "edges_per_s": e_b / tb, "s": tb},
            "per_seed": {"clusters_per_s": B / ts, "edges_per_s": e_s / ts, "s": ts},
            "request_loop": {"clusters_per_s": B / tq, "edges_per_s": e_q / tq, "s": tq,
                             "resident": SERVE["max_batch"]},
            "speedup": ts / tb}


def measure_serving(lgc, inputs, torch, ctx, g, off):
    """Open-loop Poisson arrivals through lgc_submit / lgc_wait: 80% PR-Nibble
    (alpha 0.01, eps log-uniform [1e-8, 1e-5]), 20% HK-PR (t log-uniform
    [3, 30], eps 1e-7), each with its sweep; latency = completion - submission
    (library clock)."""
    import numpy as np
    R = SERVE["requests"]
    seeds = inputs.seeds_deg2(off, R, 5)
    eps = inputs.eps_loguniform(R, 5, -8.0, -5.0)
    ts = 10.0 ** (np.log10(3.0) + (np.log10(30.0) - np.log10(3.0)) * inputs.uniform(6, R))
    kinds = inputs.uniform(7, R) < 0.8
    reqs = []
    for i in range(R):
        if kinds[i]:
            reqs.append(lgc.make_request(lgc.ALGO_PRNIBBLE, int(seeds[i]), True, alpha=0.01,
                                         eps=float(eps[i]), mode=MODE))
        else:
            t = float(ts[i])
            reqs.append(lgc.make_request(lgc.ALGO_HKPR, int(seeds[i]), True, t=t,
                                         N=hk_terms(t, SERVE["hk_eps"]), eps=SERVE["hk_eps"],
                                         mode=MODE))
    ctx.set_option(lgc.OPT_SERVE_MEM_BUDGET, SERVE["mem_budget"])
    try:
        ctx.set_option(lgc.OPT_SERVE_MAX_BATCH, SERVE["max_batch"])
    except lgc.LgcError:
        pass  # the loop is already running with it (set by measure_many)
    # warm the workers
    for tk in [lgc.submit(ctx, g, reqs[i]) for i in range(8)]:
        lgc.wait(ctx, tk)
    out = []
    for rate in SERVE["rates"]:
        # the first R requests of the mix; fewer at rates below capacity so
        # that the offered load lasts about offered_s seconds
        R = min(SERVE["requests"], max(50, int(SERVE["offered_s"] * rate)))
        gaps = -np.log(1.0 - inputs.uniform(SERVE["arrival_seed"] + rate, R)) / rate
        arrive = np.cumsum(gaps)
        # this thread submits at the arrival times; a collector thread takes
        # the results with the blocking lgc_wait (latency is measured on the
        # library's clock, so the order of collection does not matter)
        tickets = queue.Queue()
        lat, done_edges = [], [0]

        def collect():
            for _ in range(R):
                r = lgc.wait(ctx, tickets.get())
                lat.append(r["end_s"] - r["submit_s"])
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
        done_edges = done_edges[0]
        lat_ms = np.sort(np.asarray(lat)) * 1e3
        out.append({"rate_per_s": rate, "requests": R, "clusters_per_s": R / wall,
                    "edges_per_s": done_edges / wall,
                    "p50_ms": float(np.percentile(lat_ms, 50)),
                    "p99_ms": float(np.percentile(lat_ms, 99)),
                    "offered_s": float(arrive[-1]), "wall_s": wall})
    return {"workload": (f"R-MAT scale {MANY['scale']} (seed {MANY['graph_seed']}); Poisson "
                         f"arrivals (seed {SERVE['arrival_seed']}), up to {SERVE['requests']} requests "
                         f"per rate ({SERVE['offered_s']:.0f} s of offered load at low rates): 80% "
                         "PR-Nibble alpha 0.01 eps log-uniform [1e-8, 1e-5], 20% HK-PR t "
                         "log-uniform [3, 30] eps 1e-7 (N from the Poisson tail); sweep each; "
                         f"memory budget {SERVE['mem_budget'] >> 30} GB, "
                         f"{SERVE['max_batch']} resident"),
            "rates": out}


# DRAM read + write bytes of the edge-phase kernels over one step of the
# default workload, by the heavy pull gather's share width (8 or 16 bytes;
# the batch depth and lanes per item move the gathers' DRAM bytes by under
# 2%): ncu dram__bytes_read.sum + dram__bytes_write.sum of emap_atomic_kernel,
# emap_red_kernel, pull_light_fx_kernel, pull_heavy_fx_kernel,
# rounds_prnibble_kernel and rounds_nibble_kernel, summed over one step
# (shapes (8, 32, 8) and (8, 32, 16)).  Re-capture when any of these kernels
# changes.
EDGE_TRAFFIC_PER_STEP = {8: 9.082e9, 16: 10.896e9}
TRAFFIC_SOURCE = "profiles/traffic_edge_phase_rmat22.md"

# bytes of the per-step inputs handed to the library (seed + parameter structs)
H2D_BYTES_PER_STEP = 4 * 4 + 32 + 24 + 24 + 32


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
                    help="skip the batched-vs-per-seed and serving measurements")
    ap.add_argument("--pull-shape", default="",
                    help="heavy pull gather shape 'batch,lanes,share_bytes' instead of the "
                         "graph's autotuned one (e.g. 8,32,8)")
    ap.add_argument("--algos", default=",".join(ALGOS),
                    help="comma-separated subset of the step (for profiling one diffusion)")
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

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1604_07515_gb300 import inputs, lgc

    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    off, col = inputs.rmat(SCALE, seed=GRAPH_SEED)
    x = rank_seed(off, col, rank)
    stream = torch.cuda.current_stream()
    ctx = lgc.Context(dev, stream)
    g = lgc.Graph(ctx, off, col)
    if args.pull_shape:
        pull_shape = tuple(int(v) for v in args.pull_shape.split(","))
        for opt, v in zip((lgc.OPT_PULL_BATCH, lgc.OPT_PULL_GROUP, lgc.OPT_PULL_SHARE),
                          pull_shape):
            ctx.set_option(opt, v)
    else:
        pull_shape = g.autotune()  # launch-shape tuning on this graph, before any timing
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident results: the kernel-side number ----
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
    for _ in range(args.warmup):
        one_step(lgc, g, x)
    ctx.set_option(lgc.OPT_PROFILE, 1)
    ctx.profile_reset()
    clocks = ClockSampler(dev)
    barrier()
    clocks.start()
    launches0 = ctx.launch_count()
    step_ms, pushed, clusters = [], 0, 0
    split = {a: {"ms": 0.0, "edges": 0} for a in STEP_ALGOS}
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (not timed)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        evs = []
        a.record(stream)
        pe, cl, _ = one_step(lgc, g, x, evs)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        pushed += pe
        clusters += cl
        for i, name in enumerate(STEP_ALGOS):
            split[name]["ms"] += evs[i].elapsed_time(evs[i + 1]) / args.steps
            split[name]["edges"] += evs[-1][i] / args.steps  # mean over the steps
    barrier()
    launches = ctx.launch_count() - launches0
    clk = clocks.stop()
    ctx.set_option(lgc.OPT_PROFILE, 0)
    prof = {lgc.PROF_NAMES[k]: ctx.profile(k) for k in lgc.PROF_NAMES}
    (total_ms,), (pushed, clusters) = reduce_ranks([sum(step_ms)], [pushed, clusters], world,
                                                    "cuda")
    value = pushed / (total_ms / 1e3)

    # ---- end to end through the public API with host buffers ----
    ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)
    one_step(lgc, g, x)
    barrier()
    e_pushed, d2h, e2e_s = 0, 0, 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        pe, _, db = one_step(lgc, g, x)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - s0
        e_pushed += pe
        d2h += db
    (e2e_s,), (e_pushed,) = reduce_ranks([e2e_s], [e_pushed], world, "cuda")
    e2e_value = e_pushed / e2e_s

    # ---- batched vs per-seed, and serving (rank 0, one GPU) ----
    many = serving = None
    if rank == 0 and world == 1 and not args.no_many:
        g.close()
        del flush
        offm, colm = inputs.rmat(MANY["scale"], seed=MANY["graph_seed"])
        gm = lgc.Graph(ctx, offm, colm)
        gm.autotune()
        del colm
        ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 1)
        many = measure_many(lgc, inputs, torch, ctx, gm, offm)
        ctx.set_option(lgc.OPT_RESULT_ON_DEVICE, 0)
        serving = measure_serving(lgc, inputs, torch, ctx, gm, offm)
        gm.close()

    # ---- roofline of the dominant kernel ----
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
    # DRAM bytes of the edge phase per launch, from the ncu capture of this
    # workload and pull shape (null for any other workload or shape)
    traffic = None
    share_bytes = pull_shape[2]
    if (dname == "edgemap_atomic" and MODE == "atomic" and STEP_ALGOS == ALGOS
            and share_bytes in EDGE_TRAFFIC_PER_STEP and d["launches"] > 0):
        per_step = d["launches"] / args.steps
        traffic = EDGE_TRAFFIC_PER_STEP[share_bytes] / per_step
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": traffic, "traffic_source": TRAFFIC_SOURCE if traffic else None,
                "launches": d["launches"],
                "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
                "alg_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "share_of_step": d["ms"] / total_ms if total_ms else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        cp = 0
        k = 0
        while k < 4:  # one of each diffusion, about 20 s of single-threaded work
            cp += cpu_oracle_step(off, col, x, k)
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": cp / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": "the four diffusions of one step and their sweeps, once each, "
                         "single-threaded on the host"}

    if rank == 0:
        line = {
            "metric": "pushed_edges_per_s", "value": value, "unit": "edges/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if STEP_ALGOS == ALGOS
                       else WORKLOAD + f" (only: {','.join(STEP_ALGOS)})", "mode": MODE,
                       "l2": "inputs larger than L2 and L2 flushed between steps",
                       "parallelism": f"replicas{world}", "pull_shape": list(pull_shape)},
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
            "many_seeds": many, "serving": serving,
        }
        print(json.dumps(line), flush=True)
    g.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


MODE = "atomic"
STEP_ALGOS = ALGOS

if __name__ == "__main__":
    sys.exit(main())

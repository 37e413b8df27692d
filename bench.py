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

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

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
        for ln in self.lines:
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
                "samples": len(sm)}


def one_step(lgc, g, x):
    """The hot path for one seed; returns (pushed_edges, clusters, d2h_bytes)."""
    pushed, clusters, d2h = 0, 0, 0
    p, st = lgc.prnibble(g, x, PR["alpha"], PR["eps"], mode=MODE)
    c = lgc.sweep(g, p)
    pushed += st.pushed_edges
    clusters += 1
    d2h += 0 if p.on_device else 12 * p.nnz + 4 * c.size
    p, st = lgc.nibble(g, x, NB["T"], NB["eps"], mode=MODE)
    c = lgc.sweep(g, p)
    pushed += st.pushed_edges
    clusters += 1
    d2h += 0 if p.on_device else 12 * p.nnz + 4 * c.size
    p, st = lgc.hkpr(g, x, HK["t"], HK["N"], HK["eps"], mode=MODE)
    c = lgc.sweep(g, p)
    pushed += st.pushed_edges
    clusters += 1
    d2h += 0 if p.on_device else 12 * p.nnz + 4 * c.size
    p, st = lgc.rand_hkpr(g, x, RH["t"], RH["K"], RH["n_walks"], RH["rng_seed"])
    c = lgc.sweep(g, p)
    pushed += st.pushed_edges
    clusters += 1
    d2h += 0 if p.on_device else 12 * p.nnz + 4 * c.size
    return pushed, clusters, d2h


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
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="atomic", choices=["atomic", "det"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    global MODE
    MODE = args.mode
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
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (not timed)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pe, cl, _ = one_step(lgc, g, x)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        pushed += pe
        clusters += cl
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
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": None, "launches": d["launches"],
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
            "config": {"workload": WORKLOAD, "mode": MODE,
                       "l2": "inputs larger than L2 and L2 flushed between steps",
                       "parallelism": f"replicas{world}"},
            "clusters_per_s": clusters / (total_ms / 1e3),
            "pushed_edges_per_step": pushed / args.steps / max(1, world),
            "roofline": roofline, "kernels": prof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "edges/s",
                    "h2d_bytes_per_step": H2D_BYTES_PER_STEP,
                    "d2h_bytes_per_step": d2h // max(1, args.steps)},
            "clocks": clk, "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    g.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


MODE = "atomic"

if __name__ == "__main__":
    sys.exit(main())

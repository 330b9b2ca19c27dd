"""Benchmark of the phase-parallel Dijkstra hot path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1..5]
                    [--criterion C] [--form auto|single|batched] [--impl ours|reference]

Default workload: directed G(n, m) with n = 2^24 vertices and m = 2^28 edges,
uint32 costs uniform in [0, 2^24), 8 seeded random sources.  A step is one pass
of the whole hot path over that input: all 8 solves (threshold reduce,
selection, relaxation in every phase, until F is empty), by default as one
batched persistent launch (captured in a CUDA graph, blocks per solve from the
library's autotuner) in which every phase picks its criterion variant and
frontier representation with the learned policy (trained in this run by the
library's own FP32 kernels on small seeded graphs, none of them the benchmark
graph).  Single-source workloads time one solve per step.  Graph preprocessing
is timed once and reported separately (``prep_ms``); the end-to-end number
(``e2e``) includes it, together with the host->device copy of the CSR graph
from pinned memory and the device->host read of every distance array.

Metric: GTEPS = (sum over solves of the out-degrees of the settled vertices,
i.e. every edge relaxed once) / time.  Phases and queries/s are reported
alongside.  Beside the headline form the same solves are timed as plain
single solves with the fixed IN-STATIC | OUT-STATIC criterion (``plain``), and,
for the learned policy, with each of its four fixed arms in the headline's
form (``fixed_arms``: the fastest of them is the policy's judge).  Rank 0
prints one JSON line.

Under torchrun (N>1) every rank runs an independent replica of the workload (the
method has no exchange step on one GPU), value = all ranks' edges / max time.
``--impl reference`` times the CPU oracle's binary-heap Dijkstra instead (rank 0
only) on the same workload and metric, each step a bounded sample of a solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SSSP GTEPS & phases (learned/batched vs plain IN+OUT, 1 GB300); queries/s"
L2_BYTES = 129 * 2**20
DEFAULT_WORKLOAD = 5  # G(2^24, 2^28), 8 sources: the largest workload that fits one GPU


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", type=int, default=DEFAULT_WORKLOAD)
    ap.add_argument("--shrink", type=int, default=0,
                    help="a smaller member of the workload's family (sizes / 2^shrink), for profiling captures")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--criterion", default="learned", choices=["in_out", "simple", "learned", "full_weak", "approx4"],
                    help="learned = per-phase policy over the IN-STATIC/IN-SIMPLE x sparse/dense arms (fallback "
                         "IN-STATIC | OUT-STATIC); full_weak = IN (full) | OUT-WEAK; approx4 = approximate minima "
                         "recomputed every 4th phase")
    ap.add_argument("--form", default="auto", choices=["auto", "single", "batched"],
                    help="batched = all solves of a step in one prepared launch; auto = batched when the workload "
                         "has more than one solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain single-solve IN+OUT leg")
    ap.add_argument("--no-arms", action="store_true", help="skip timing the policy's fixed arms")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--batch-sources", type=int, default=0,
                    help="single-source workloads: also time this many seeded sources in one batched launch")
    return ap.parse_args()


# DRAM bytes (read + write) of one solve launch, from one ncu capture of this
# bench's own command (the summaries under profiles/ give the command), keyed by
# workload name and criterion, with a hash of the engine sources the capture ran
# on: once the kernel changes the figure no longer applies and is reported null.
MEASURED_TRAFFIC = {
    # one timed launch of the default step (8 solves of G(2^24, 2^28), 152 blocks)
    ("gnm_n16777216_m268435456", "learned", "k_solve_batch"): (471704877312 + 42709658368, "5d86847cefe8b298"),
}
ENGINE_SOURCES = ("engine.cu", "engine.h", "common.cuh", "policy.cuh")


def engine_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        with open(os.path.join(ROOT, "paper_1903_12085_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, criterion: str, kernel: str):
    t = MEASURED_TRAFFIC.get((workload, criterion, kernel))
    if t is None or t[1] != engine_hash():
        return None
    return t[0]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"clocks_rank{index}_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.f.close()

    def summary(self):
        if not self.proc:
            if os.path.exists(self.path):
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(dist, device, total_ms: float, counts: dict) -> tuple:
    """Whole-job figures of a timed region run by every rank of ``dist``.

    Returns (max over ranks of total_ms, {key: sum over ranks}).  The time is
    the slowest rank's (the job ends when it does); the counts (edges, solves,
    phases, ...) add up because every rank processed its own units.  With
    ``dist`` None (one process) the inputs come back unchanged.
    """
    if dist is None:
        return total_ms, dict(counts)
    import torch
    keys = sorted(counts)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    c = torch.tensor([int(counts[k]) for k in keys], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), {k: int(v) for k, v in zip(keys, c.tolist())}


def rank_solve(solves: list, rank: int, k: int):
    """Solve of step k on this rank: ranks start at different sources."""
    return solves[(k + rank) % len(solves)]


def build_workload(k: int, shrink: int = 0):
    import graphgen as gg
    return gg.workload(k, shrink=shrink)


def crit_value(sp, name):
    return {"in_out": sp.IN_OUT, "simple": sp.SIMPLE, "learned": sp.IN_OUT | sp.POLICY_LEARNED,
            "full_weak": sp.IN_FULL | sp.OUT_WEAK, "approx4": sp.approx(4)}[name]


def oracle_sample(g, s: int, max_settled: int):
    """One timed run of the oracle's binary-heap Dijkstra from s, stopped
    after max_settled settled vertices (the whole solve when max_settled >= n).
    Returns (settled, edges scanned = their out-degrees, seconds)."""
    import oracle
    t0 = time.perf_counter()
    settled, scanned = oracle.dijkstra_prefix(g, s, max_settled)
    return settled, scanned, time.perf_counter() - t0


def calibrate_sample(g, s: int, budget_s: float) -> int:
    """Settled-vertex count of a Dijkstra prefix from s that takes about
    budget_s on this host (the whole solve if that is faster)."""
    probe = min(g.n, 1 << 18)
    settled, _, dt = oracle_sample(g, s, probe)
    if settled < probe:  # the whole reachable part took dt
        return g.n
    return int(min(g.n, max(probe, probe * budget_s / max(dt, 1e-6))))


def sample_desc(wl, settled: int, n: int, runs: int, seconds: float) -> str:
    what = "whole solves" if settled >= n else f"prefixes of the first {settled} settled vertices (of {n})"
    return (f"{runs} binary-heap Dijkstra {what} of {wl.name}, source of its first solve "
            f"({seconds:.1f} s, 1 thread)")


def run_reference(args, wl):
    """CPU oracle (binary-heap Dijkstra, one host core) on the same workload:
    every step a bounded sample (a Dijkstra prefix of about 8 s, or the whole
    solve if shorter) from the source of the workload's first solve."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    gi, s = wl.solves[0]
    g = wl.graphs[gi]
    max_settled = calibrate_sample(g, s, budget_s=8.0)
    times, edges, settled = [], 0, 0
    for step in range(args.warmup + args.steps):
        st, sc, dt = oracle_sample(g, s, max_settled)
        if step >= args.warmup:
            times.append(dt)
            edges += sc
            settled = st
    total = sum(times)
    value = edges / total / 1e9
    desc = sample_desc(wl, settled, g.n, args.steps, total)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "solver": "oracle binary-heap Dijkstra, 1 host core",
                   "sample": desc},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": desc,
                         **host_info()},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(wl, budget_s=12.0):
    """Oracle Dijkstra on one host core: a bounded sample (a prefix of about
    budget_s, or whole solves while they fit) from the first solve's source."""
    gi, s = wl.solves[0]
    g = wl.graphs[gi]
    max_settled = calibrate_sample(g, s, budget_s=budget_s / 2)
    edges, t, runs, settled = 0, 0.0, 0, 0
    while t < budget_s / 2 and runs < 64:
        st, sc, dt = oracle_sample(g, s, max_settled)
        edges += sc
        t += dt
        runs += 1
        settled = st
    return {"value": edges / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": sample_desc(wl, settled, g.n, runs, t), **host_info()}


def host_info():
    """The host the CPU baseline ran on (it uses one of these cores)."""
    import platform
    return {"host_cpus": os.cpu_count(), "host_arch": platform.machine()}


def trace_totals(tr) -> dict:
    """Counts of one solve from its per-phase records."""
    return {"phases": len(tr), "edges_relaxed": int(tr["deg_settled"].astype(np.int64).sum()),
            "settled": int(tr["settled"].astype(np.int64).sum()),
            "sum_frontier": int(tr["frontier"].astype(np.int64).sum()),
            "sum_queued": int(tr["queued"].astype(np.int64).sum())}


def timed_steps(torch, stream, flush, fn, steps: int):
    """CUDA-event times (ms) of `steps` calls of fn on `stream`, with the L2
    flushed before each (outside the events)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        fn(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


class Form:
    """The solves of one step, run either as one prepared batch or as single
    solves back to back, with per-solve counts from traced runs."""

    def __init__(self, sp, torch, G, solves, crit, batched: bool, bpg=None, autotune=True):
        self.sp, self.torch, self.solves, self.crit, self.batched = sp, torch, solves, crit, batched
        self.graphs = [G[gi] for gi, _ in solves]
        self.sources = [s for _, s in solves]
        self.bpg = None
        if batched:
            if bpg is not None:
                sp.set_tuning(batch_blocks_per_solve=bpg)
            self.B = sp.Batch(self.graphs, self.sources, crit)
            if bpg is not None:
                sp.set_tuning(batch_blocks_per_solve=0)
                self.bpg = bpg
            elif autotune:
                self.bpg, _ = self.B.autotune()
            cap = min(max(g.n for g in self.graphs) + 1, 1 << 16)
            for i in range(len(self.graphs)):
                self.B.attach_trace(i, trace_cap=cap)
            self.B.launch()
            torch.cuda.synchronize()
            self.stats = []
            for i in range(len(self.graphs)):
                _, tr = self.B.trace_of(i)
                assert len(tr) == int(self.B.phases[i].item()), "trace capacity below the phase count"
                self.stats.append(trace_totals(tr))
            for i in range(len(self.graphs)):
                self.B.detach_trace(i)
        else:
            self.outs = {}
            self.stats = []
            for G_, s in zip(self.graphs, self.sources):
                if id(G_) not in self.outs:
                    self.outs[id(G_)] = torch.empty(G_.n, dtype=torch.int64, device="cuda")
                _, _, _, tr = sp.solve_trace(G_, s, crit, out=self.outs[id(G_)], settle=False,
                                             trace_cap=min(G_.n + 1, 1 << 21))
                self.stats.append(trace_totals(tr))

    def run(self, k=0):
        if self.batched:
            self.B.launch()
        else:
            for G_, s in zip(self.graphs, self.sources):
                self.sp.solve(G_, s, self.crit, out=self.outs[id(G_)])

    def launches(self) -> int:
        return 1 if self.batched else len(self.graphs)

    def total(self, key: str) -> int:
        return sum(st[key] for st in self.stats)

    def close(self):
        if self.batched:
            self.B.close()


def main():
    args = parse()
    ws, rank, local = dist_env()
    wl = build_workload(args.workload, args.shrink)
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    import paper_1903_12085_gb300 as sp

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    crit = crit_value(sp, args.criterion)
    learned = args.criterion == "learned"
    reverse = args.criterion != "in_out"  # the policy's IN-SIMPLE arms need the reverse CSR
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()
    batched = args.form == "batched" or (args.form == "auto" and len(wl.solves) > 1)
    # the solves of one step on this rank (replicas start at different sources)
    solves = [rank_solve(wl.solves, rank, k) for k in range(len(wl.solves))] if batched or len(wl.solves) == 1 \
        else [rank_solve(wl.solves, rank, 0)]

    # ---- device-resident graphs (prep timed once)
    t0 = time.perf_counter()
    G = [sp.Graph.from_csr(g, reverse=reverse) for g in wl.graphs]
    torch.cuda.synchronize()
    prep_ms = 1e3 * (time.perf_counter() - t0)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    train = None
    if learned:  # the policy network, trained here by the library's own kernels
        from paper_1903_12085_gb300 import policy as pol
        t0 = time.perf_counter()
        _, hist = pol.fit_and_load()
        train = {"train_s": round(time.perf_counter() - t0, 2), "final_train_loss": hist[-1][1] if hist else None}

    # ---- headline form
    head = Form(sp, torch, G, solves, crit, batched)
    for k in range(args.warmup):
        head.run(k)
    if pg:
        pg.barrier()
    with ClockSampler(local) as clk:
        step_ms = timed_steps(torch, stream, flush, head.run, args.steps)
    if pg:
        pg.barrier()
    local_ms = sum(step_ms)
    per = {key: head.total(key) for key in ("edges_relaxed", "phases", "settled", "sum_frontier", "sum_queued")}
    nsolves = len(solves) * args.steps
    total_ms, tot = combine_ranks(pg, "cuda", local_ms,
                                  {"edges": per["edges_relaxed"] * args.steps, "phases": per["phases"] * args.steps,
                                   "sum_f": per["sum_frontier"] * args.steps, "sum_q": per["sum_queued"] * args.steps,
                                   "solves": nsolves})
    value = tot["edges"] / (total_ms * 1e-3) / 1e9
    step_avg_ms = local_ms / args.steps

    # roofline of the solve kernel: algorithmic bytes per step / step time.
    # Per solve: 16 B per relaxed edge (8 B edge + 8 B distance word) + 16 B
    # per settled vertex + 16 B per queue entry a phase scans (the paper's
    # identification work, sum of |F| over phases, less the far part of F that
    # the near/far split leaves untouched).
    alg_bytes = 16 * (per["edges_relaxed"] + per["settled"] + per["sum_queued"])
    achieved = alg_bytes / (step_avg_ms * 1e-3) / 1e9
    edge_only = 16 * per["edges_relaxed"] / (step_avg_ms * 1e-3) / 1e9
    kernel = "k_solve_batch" if batched else "k_solve_grid"
    traffic = measured_traffic(wl.name, args.criterion, kernel)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": kernel, "launches_per_step": head.launches(),
                "alg_bytes_per_step": alg_bytes, "edge_only_frac": edge_only / hbm,
                # DRAM bytes the launch really moved (ncu) over the same step time
                "dram_frac": None if traffic is None else traffic / (step_avg_ms * 1e-3) / 1e9 / hbm}
    if learned:
        train["arms_used"] = "per-phase choice logged in the trace records"

    # ---- the same solves as plain single solves with the fixed IN+OUT criterion
    plain = None
    if not args.no_plain and (batched or learned or args.criterion != "in_out"):
        pf = Form(sp, torch, G, solves, sp.IN_OUT, batched=False)
        pf.run()
        reps = max(1, min(args.steps, 3))
        pms = timed_steps(torch, stream, flush, pf.run, reps)
        pmed = statistics.median(pms)
        plain = {"criterion": "in_out", "form": "single", "ms_per_step": pmed,
                 "value": pf.total("edges_relaxed") / (pmed * 1e-3) / 1e9, "unit": "GTEPS",
                 "phases_per_solve": pf.total("phases") / len(solves),
                 "speedup_of_headline": pmed / statistics.median(step_ms)}
        pf.close()

    # ---- the policy's judge: each fixed arm in the headline's form
    arms = None
    if learned and not args.no_arms:
        names = ["in_out_sparse", "in_out_dense", "insimple_out_sparse", "insimple_out_dense"]
        masks = [sp.IN_OUT, sp.IN_OUT | sp.FRONTIER_DENSE, sp.IN_SIMPLE | sp.OUT_STATIC,
                 sp.IN_SIMPLE | sp.OUT_STATIC | sp.FRONTIER_DENSE]
        arms = {}
        for name, mask in zip(names, masks):
            fa = Form(sp, torch, G, solves, mask, batched, bpg=head.bpg)
            fa.run()
            reps = max(1, min(args.steps, 3))
            ams = statistics.median(timed_steps(torch, stream, flush, fa.run, reps))
            arms[name] = {"ms_per_step": ams, "phases_per_solve": fa.total("phases") / len(solves)}
            fa.close()
        fastest = min(arms, key=lambda a: arms[a]["ms_per_step"])
        arms["fastest_fixed"] = fastest
        arms["speedup_vs_fastest_fixed"] = arms[fastest]["ms_per_step"] / statistics.median(step_ms)
        arms["speedup_vs_in_out_same_form"] = arms["in_out_sparse"]["ms_per_step"] / statistics.median(step_ms)

    # ---- single-source workloads: many seeded sources in one batched launch
    extra_batch = None
    if not batched and args.batch_sources > 0:
        import graphgen as gg
        gi0 = wl.solves[0][0]
        g0 = wl.graphs[gi0]
        src = [int(gg.splitmix64_nth(0x5EED0B, i) >> 32) * g0.n >> 32 for i in range(args.batch_sources)]
        src[0] = wl.solves[0][1]
        t0 = time.perf_counter()
        fb = Form(sp, torch, G, [(gi0, s) for s in src], crit, batched=True)
        tune_s = time.perf_counter() - t0
        for k in range(args.warmup):
            fb.run(k)
        bms = statistics.median(timed_steps(torch, stream, flush, fb.run, max(1, min(args.steps, 5))))
        extra_batch = {"sources": len(src), "ms_per_launch": bms, "blocks_per_solve": fb.bpg,
                       "setup_s": round(tune_s, 2), "queries_per_s": len(src) / (bms * 1e-3),
                       "value": fb.total("edges_relaxed") / (bms * 1e-3) / 1e9, "unit": "GTEPS",
                       "speedup_queries_vs_single": (len(src) / bms) / (nsolves / local_ms)}
        fb.close()
    head.close()

    # ---- end to end through the public API: graphs from pinned host CSR,
    # the step's solves, every distance array read back to pinned host memory
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        used = sorted({gi for gi, _ in solves})
        hcsr = {gi: (wl.graphs[gi].n, pin(wl.graphs[gi].row_off), pin(wl.graphs[gi].col), pin(wl.graphs[gi].w))
                for gi in used}
        sizes = [wl.graphs[gi].n for gi, _ in solves]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        dist_h = torch.empty(int(offs[-1]), dtype=torch.int64).pin_memory()
        ph_h = torch.empty(len(solves), dtype=torch.int64).pin_memory()
        e2e_t = 0.0
        reps = max(1, min(args.steps, 3))
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Gh = {gi: sp.Graph(n, ro, col, w, reverse=reverse) for gi, (n, ro, col, w) in hcsr.items()}
            if batched:
                Bh = sp.Batch([Gh[gi] for gi, _ in solves], [s for _, s in solves], crit)
                Bh.launch()
                for k, o in enumerate(Bh.outs):
                    dist_h[offs[k]:offs[k + 1]].copy_(o, non_blocking=True)
                ph_h.copy_(Bh.phases, non_blocking=True)
                torch.cuda.synchronize()
                Bh.close()
            else:
                dv = dist_h.numpy().view(np.uint64)
                for k, (gi, s) in enumerate(solves):
                    _, ph = sp.solve(Gh[gi], s, crit, out=dv[offs[k]:offs[k + 1]])
            for gh in Gh.values():
                gh.close()
            dt = time.perf_counter() - t0
            if r > 0:
                e2e_t += dt
        e2e_ms, etot = combine_ranks(pg, "cuda", 1e3 * e2e_t, {"edges": per["edges_relaxed"] * reps})
        e2e = {"value": etot["edges"] / (e2e_ms * 1e-3) / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": int(sum(ro.nbytes + col.nbytes + w.nbytes for _, ro, col, w in hcsr.values())),
               "d2h_bytes_per_step": int(dist_h.numel() * 8 + (ph_h.numel() * 8 if batched else 0)),
               "includes": "graphs created from pinned host CSR (H2D + preprocessing)"
                           + (" + batch prepared and launched" if batched else " + solves") + " + distances D2H"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl.name, "criterion": args.criterion, "form": "batched" if batched else "single",
                       "solves_per_step": len(solves), "blocks_per_solve": head.bpg,
                       "phases_per_solve": tot["phases"] / tot["solves"],
                       "queries_per_s": tot["solves"] / (total_ms * 1e-3),
                       "us_per_phase": 1e3 * local_ms / (per["phases"] * args.steps),
                       "sum_frontier_per_solve": tot["sum_f"] / tot["solves"],
                       "sum_queued_per_solve": tot["sum_q"] / tot["solves"],
                       "median_ms_per_step_rank0": statistics.median(step_ms),
                       "prep_ms": prep_ms, "l2": "flushed between steps (2x L2 buffer written)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "policy": train, "plain": plain, "fixed_arms": arms, "batched_sources": extra_batch,
            "gpu_launches": args.steps * head.launches(), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()

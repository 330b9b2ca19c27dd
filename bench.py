"""Benchmark of the phase-parallel Dijkstra hot path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1..5] [--impl ours|reference]

A step is one pass of the whole hot path over the workload: for a single-graph
workload one solve (threshold reduce, selection, relaxation in every phase, until
F is empty) from the workload's source (sources rotate for multi-source
workloads); for the batched workload one launch of all its solves.  Graph
preprocessing is timed once and reported separately (``prep_ms``); the
end-to-end number (``e2e``) includes it, together with the host->device copy of
the CSR graph from pinned memory and the device->host read of the distances.

Metric: GTEPS = (sum over solves of the out-degrees of the settled vertices,
i.e. every edge relaxed once) / solve time.  Phases and queries/s are reported
alongside.  Rank 0 prints one JSON line.

Under torchrun (N>1) every rank runs an independent replica of the workload (the
method has no exchange step on one GPU), value = all ranks' edges / max time.
``--impl reference`` times the CPU oracle's binary-heap Dijkstra instead (rank 0
only) on the same workload and metric.
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
DEFAULT_WORKLOAD = 2  # the 1024x1024 grid: the second workload of the study


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", type=int, default=DEFAULT_WORKLOAD)
    ap.add_argument("--shrink", type=int, default=0,
                    help="a smaller member of the workload's family (sizes / 2^shrink), for profiling captures")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--criterion", default="in_out", choices=["in_out", "simple", "learned", "full_weak", "approx4"],
                    help="full_weak = IN (full) | OUT-WEAK; approx4 = approximate minima recomputed every 4th phase")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-policy", action="store_true", help="skip training/timing the learned policy")
    ap.add_argument("--batch-sources", type=int, default=152,
                    help="sources of the batched leg (one persistent launch), 0 to skip")
    return ap.parse_args()


# DRAM bytes (read + write) of one solve launch, from one ncu capture of this
# bench's own command (the summaries under profiles/ give the command), keyed by
# workload name and criterion, with a hash of the engine sources the capture ran
# on: once the kernel changes the figure no longer applies and is reported null.
MEASURED_TRAFFIC = {
    ("grid_1024x1024", "in_out"): (52220672 + 7912192, "9afd8ba9ec29eacd"),
}
ENGINE_SOURCES = ("engine.cu", "engine.h", "common.cuh", "policy.cuh")


def engine_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ENGINE_SOURCES:
        with open(os.path.join(ROOT, "paper_1903_12085_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, criterion: str):
    t = MEASURED_TRAFFIC.get((workload, criterion))
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


def run_reference(args, wl):
    """CPU oracle (binary-heap Dijkstra, one host core) on the same workload."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    solves = wl.solves
    times, edges = [], 0
    for step in range(args.warmup + args.steps):
        gi, s = solves[step % len(solves)]
        g = wl.graphs[gi]
        t0 = time.perf_counter()
        d = oracle.dijkstra(g, s)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            edges += int(g.outdeg()[d != oracle.INF].sum())
    total = sum(times)
    value = edges / total / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl.name, "solver": "oracle binary-heap Dijkstra, 1 host core"},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} whole solves of {wl.name}", **host_info()},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(wl, budget_s=12.0):
    """Oracle Dijkstra on the host: whole solves until ~budget_s of CPU time."""
    import oracle
    edges, t, count = 0, 0.0, 0
    while t < budget_s and count < 64:
        gi, s = wl.solves[count % len(wl.solves)]
        g = wl.graphs[gi]
        t0 = time.perf_counter()
        d = oracle.dijkstra(g, s)
        t += time.perf_counter() - t0
        edges += int(g.outdeg()[d != oracle.INF].sum())
        count += 1
    return {"value": edges / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{count} whole binary-heap Dijkstra solves of {wl.name} ({t:.1f} s, 1 thread)",
            **host_info()}


def host_info():
    """The host the CPU baseline ran on (it uses one of these cores)."""
    import platform
    return {"host_cpus": os.cpu_count(), "host_arch": platform.machine()}


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
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()

    # ---- device-resident graphs (prep timed once)
    t0 = time.perf_counter()
    G = [sp.Graph.from_csr(g, reverse=(args.criterion != "in_out")) for g in wl.graphs]
    torch.cuda.synchronize()
    prep_ms = 1e3 * (time.perf_counter() - t0)
    batched = args.workload == 4
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    batch_tune = None
    if batched:
        B = sp.Batch([G[i] for i, _ in wl.solves], [s for _, s in wl.solves], crit)
        bpg, _ = B.autotune()
        batch_tune = {"blocks_per_solve": bpg}
        edges_per_step = None

        def step(k):
            B.launch()
    else:
        outs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for g in wl.graphs]

        def step(k):
            gi, s = rank_solve(wl.solves, rank, k)
            return sp.solve_trace(G[gi], s, crit, out=outs[gi], settle=False)

    # edges / phases / frontier work per step (deterministic: from one traced
    # pass per solve), indexed like step(k)
    # (the trace gives the queue entries each phase scanned: with the near/far
    # split the far part of F is not touched)
    per_solve = []
    for k in range(len(wl.solves)):
        gi, s = rank_solve(wl.solves, rank, k)
        _, stats, _, tr = sp.solve_trace(G[gi], s, crit, settle=False, trace_cap=min(1 << 21, G[gi].n + 1))
        stats["sum_queued"] = int(tr["queued"].astype(np.int64).sum())
        per_solve.append(stats)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    edges = phases = settled = sum_f = sum_q = 0
    nsolves = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            step(k)
            ev[k][1].record(stream)
            if batched:
                for st in per_solve:
                    edges += st["edges_relaxed"]; phases += st["phases"]
                    settled += st["settled"]; sum_f += st["sum_frontier"]; sum_q += st["sum_queued"]
                nsolves += len(per_solve)
            else:
                st = per_solve[k % len(per_solve)]
                edges += st["edges_relaxed"]; phases += st["phases"]
                settled += st["settled"]; sum_f += st["sum_frontier"]; sum_q += st["sum_queued"]
                nsolves += 1
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    local_ms = sum(step_ms)
    local_edges = edges
    total_ms, tot = combine_ranks(pg, "cuda", local_ms,
                                  {"edges": edges, "phases": phases, "settled": settled,
                                   "sum_f": sum_f, "sum_q": sum_q, "solves": nsolves})
    value = tot["edges"] / (total_ms * 1e-3) / 1e9
    kernel_ms = local_ms / args.steps

    # roofline of the solve kernel: algorithmic bytes per launch / launch time
    # per solve: 16 B per relaxed edge (8 B edge + 8 B distance word) + 16 B per
    # settled vertex + 16 B per queue entry a phase scans (the paper's
    # identification work, sum of |F| over phases, less the far part of F that
    # the near/far split leaves untouched)
    alg_bytes = (16 * local_edges + 16 * settled + 16 * sum_q) / args.steps
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    edge_only = 16 * local_edges / args.steps / (kernel_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None if batched else measured_traffic(wl.name, args.criterion),
                "peak_kind": peak_kind, "kernel": "k_solve_grid" if not batched else "k_solve_batch",
                "edge_only_frac": edge_only / hbm}

    # ---- learned per-phase policy (trained here on small graphs, by the
    # library's own FP32 kernels), same workload and timing rules
    learned = None
    if not batched and not args.no_policy and args.criterion == "in_out":
        from paper_1903_12085_gb300 import policy as pol
        t0 = time.perf_counter()
        _, hist = pol.fit_and_load()
        train_s = time.perf_counter() - t0
        Gr = [sp.Graph.from_csr(g, reverse=True) for g in wl.graphs]
        lcrit = sp.IN_OUT | sp.POLICY_LEARNED
        lstats = []
        for k in range(len(wl.solves)):
            gi, s = rank_solve(wl.solves, rank, k)
            _, st, _, _ = sp.solve_trace(Gr[gi], s, lcrit, settle=False)
            lstats.append(st)
        for k in range(args.warmup):
            gi, s = rank_solve(wl.solves, rank, k)
            sp.solve(Gr[gi], s, lcrit, out=outs[gi])
        lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        ledges = lphases = 0
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            gi, s = rank_solve(wl.solves, rank, k)
            lev[k][0].record(stream)
            sp.solve(Gr[gi], s, lcrit, out=outs[gi])
            lev[k][1].record(stream)
            ledges += lstats[k % len(lstats)]["edges_relaxed"]
            lphases += lstats[k % len(lstats)]["phases"]
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        lms_local = sum(a.elapsed_time(b) for a, b in lev)
        lms, ltot = combine_ranks(pg, "cuda", lms_local, {"edges": ledges})
        learned = {"value": ltot["edges"] / (lms * 1e-3) / 1e9, "unit": "GTEPS", "ms_per_step": lms / args.steps,
                   "phases_per_solve": lphases / args.steps, "speedup_vs_in_out": local_ms / lms_local,
                   "train_s": round(train_s, 2), "final_train_loss": hist[-1][1] if hist else None}
        sp.policy_clear()

    # ---- batched: many sources on the same graph(s) in one persistent launch
    # captured in a CUDA graph (groups of blocks per solve chosen by the library)
    batched_leg = None
    if not batched and args.batch_sources > 0:
        import graphgen as gg
        gi0 = wl.solves[0][0]
        g0 = wl.graphs[gi0]
        rng_src = [int(gg.splitmix64_nth(0x5EED0B, i) >> 32) * g0.n >> 32 for i in range(args.batch_sources)]
        rng_src[0] = wl.solves[0][1]
        B = sp.Batch([G[gi0]] * len(rng_src), rng_src, crit)
        t0 = time.perf_counter()
        bpg, tuned_ms = B.autotune()  # the library's autotuner picks blocks per solve
        tune_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            B.launch()
        torch.cuda.synchronize()
        # edges relaxed by each solve = out-degrees of the vertices it reached
        deg_t = torch.from_numpy(g0.outdeg()).cuda()
        bedges = int(sum(int(deg_t[o != -1].sum().item()) for o in B.outs))
        bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            bev[k][0].record(stream)
            B.launch()
            bev[k][1].record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        bms_local = sum(a.elapsed_time(b) for a, b in bev) / args.steps
        bms, btot = combine_ranks(pg, "cuda", bms_local, {"edges": bedges, "sources": len(rng_src)})
        batched_leg = {"sources": len(rng_src), "ms_per_launch": bms, "blocks_per_solve": bpg,
                       "autotune_s": round(tune_s, 2),
                       "queries_per_s": btot["sources"] / (bms * 1e-3),
                       "value": btot["edges"] / (bms * 1e-3) / 1e9, "unit": "GTEPS",
                       "speedup_queries_vs_single": (len(rng_src) / bms_local) / (nsolves / local_ms)}
        B.close()

    # ---- end to end through the public API with host buffers
    e2e = None
    if not batched:
        gi, s = rank_solve(wl.solves, rank, 0)
        g = wl.graphs[gi]
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        ro, col, w = pin(g.row_off), pin(g.col), pin(g.w)
        dist_h = torch.empty(g.n, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        e2e_t, e2e_edges = 0.0, 0
        reps = max(1, min(args.steps, 5))
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Gh = sp.Graph(g.n, ro, col, w, reverse=(args.criterion != "in_out"))
            _, ph = sp.solve(Gh, s, crit, out=dist_h)
            Gh.close()
            dt = time.perf_counter() - t0
            if r > 0:
                e2e_t += dt
                e2e_edges += per_solve[0]["edges_relaxed"]
        if pg:
            pg.barrier()
        e2e_ms, etot = combine_ranks(pg, "cuda", 1e3 * e2e_t, {"edges": e2e_edges})
        e2e = {"value": etot["edges"] / (e2e_ms * 1e-3) / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": int(ro.nbytes + col.nbytes + w.nbytes),
               "d2h_bytes_per_step": int(dist_h.nbytes + 8), "includes": "graph create (H2D + preprocessing) + solve + D2H"}
    else:
        # every step: all graphs created from pinned host CSR, the batch
        # prepared (workspaces, CUDA graph capture) and launched, every
        # solve's distances read back into pinned host memory
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        hcsr = [(g.n, pin(g.row_off), pin(g.col), pin(g.w)) for g in wl.graphs]
        sizes = [wl.graphs[i].n for i, _ in wl.solves]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        dist_h = torch.empty(int(offs[-1]), dtype=torch.int64).pin_memory()
        e2e_t, e2e_edges = 0.0, 0
        reps = max(1, min(args.steps, 3))
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Gh = [sp.Graph(n, ro, col, w, reverse=(args.criterion != "in_out")) for n, ro, col, w in hcsr]
            Bh = sp.Batch([Gh[i] for i, _ in wl.solves], [s for _, s in wl.solves], crit)
            Bh.launch()
            for k, o in enumerate(Bh.outs):
                dist_h[offs[k]:offs[k + 1]].copy_(o, non_blocking=True)
            ph_h = Bh.phases.cpu()
            torch.cuda.synchronize()
            Bh.close()
            for gh in Gh:
                gh.close()
            dt = time.perf_counter() - t0
            if r > 0:
                e2e_t += dt
                e2e_edges += sum(st["edges_relaxed"] for st in per_solve)
        if pg:
            pg.barrier()
        e2e_ms, etot = combine_ranks(pg, "cuda", 1e3 * e2e_t, {"edges": e2e_edges})
        e2e = {"value": etot["edges"] / (e2e_ms * 1e-3) / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": int(sum(ro.nbytes + col.nbytes + w.nbytes for _, ro, col, w in hcsr)),
               "d2h_bytes_per_step": int(dist_h.numel() * 8 + ph_h.numel() * 8),
               "includes": "all graphs created (H2D + preprocessing) + batch prepared and launched + D2H"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": wl.name, "criterion": args.criterion, "solves_per_step": nsolves // args.steps,
                       "phases_per_solve": tot["phases"] / tot["solves"],
                       "queries_per_s": tot["solves"] / (total_ms * 1e-3),
                       "us_per_phase": 1e3 * local_ms / phases, "sum_frontier_per_solve": tot["sum_f"] / tot["solves"],
                       "sum_queued_per_solve": tot["sum_q"] / tot["solves"],
                       "median_ms_per_step_rank0": statistics.median(step_ms),
                       "prep_ms": prep_ms, "l2": "flushed between steps (2x L2 buffer written)",
                       "parallelism": f"replicas x{ws}", "batch_autotune": batch_tune},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "learned_policy": learned, "batched": batched_leg,
            "gpu_launches": args.steps, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()

"""Writes fullsize_<criterion>.json: the oracle's results on the full-size workloads.

    python tests/golden/make_fullsize.py [--criterion C] [--workloads 2,3,4,5] [--solves5 N] [--jobs J]

Every solve is run through the CPU oracle only: binary-heap Dijkstra for the
distances and the phase simulator (the generic phased algorithm of Section 3)
for the phase-by-phase settled sets, with one criterion mask:

    in_out     IN-STATIC | OUT-STATIC          (eqs. crit:instatic, crit:outstatic)
    simple     IN-SIMPLE | OUT-SIMPLE          (eqs. crit:insimple, crit:outsimple)
    full_weak  IN (full) | OUT-WEAK            (eqs. crit:in, crit:outweak)
    approx4    APPROX(4): approximate IN (full) / OUT-WEAK minima recomputed in
               every 4th phase (the closing remark of Section 3)

Workloads: 2 (1024 x 1024 grid), 3 (R-MAT scale 22), 4 (the batch of 256
graphs, 1024 solves; in_out only) and 5 (G(2^24, 2^28), 8 sources; the
dynamic criteria cost the simulator about an hour per solve there, so only the
first --solves5 sources are run for them).  Stored per solve: phases, sum of
|F|, settled and relaxed counts, and SHA-256 digests of the uint64 distance
array (UINT64_MAX = unreachable) and of the uint32 settle-phase array.  Rows of
workloads not re-run are kept from the existing file.  The GPU tests compare
the library's outputs with these values; nothing here touches the GPU path.
Workloads come from graphgen's integer-only generators, so the graphs are the
same on every host.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CRITERIA = ("in_out", "simple", "full_weak", "approx4")


def out_path(criterion: str) -> str:
    return os.path.join(HERE, f"fullsize_{criterion}.json")


def crit_bits(criterion: str) -> int:
    sys.path.insert(0, ROOT)
    import oracle
    return {"in_out": oracle.IN_STATIC | oracle.OUT_STATIC, "simple": oracle.IN_SIMPLE | oracle.OUT_SIMPLE,
            "full_weak": oracle.IN_FULL | oracle.OUT_WEAK, "approx4": oracle.approx(4)}[criterion]


def digest(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()[:32]


def _jobs(criterion: str, workloads, solves5: int):
    """(criterion, workload, [solve indices]) units of work (each unit
    generates its workload once)."""
    units = []
    for k in workloads:
        if k == 4:  # 1024 solves, 4 per graph, in 6 units
            units += [(criterion, 4, list(range(lo, min(lo + 172, 1024)))) for lo in range(0, 1024, 172)]
        elif k == 5:
            units += [(criterion, 5, [j]) for j in range(solves5)]
        else:
            units.append((criterion, k, [0]))
    return units


def _run(unit):
    criterion, k, js = unit
    sys.path.insert(0, ROOT)
    import graphgen as gg
    import oracle
    wl = gg.workload(k)
    crit = crit_bits(criterion)
    rows = []
    for j in js:
        gi, s = wl.solves[j]
        g = wl.graphs[gi]
        t0 = time.time()
        d = oracle.dijkstra(g, s)
        sim = oracle.simulate(g, s, crit, dist_ref=d)
        assert (sim.d == d).all()
        rows.append({"workload": k, "solve": j, "graph": gi, "source": s, "n": g.n, "m": int(g.m),
                     "phases": sim.phases, "sum_f": sim.sum_f, "settled": sim.settled, "relaxed": sim.relaxed,
                     "dist_sha256": digest(d), "settle_sha256": digest(sim.settle_phase),
                     "oracle_s": round(time.time() - t0, 1)})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--criterion", default="in_out", choices=CRITERIA)
    ap.add_argument("--workloads", default=None, help="comma-separated workload numbers (default: all that apply)")
    ap.add_argument("--solves5", type=int, default=None,
                    help="sources of workload 5 to run (default 8 for in_out, 1 otherwise)")
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    default_wl = (2, 3, 4, 5) if args.criterion == "in_out" else (2, 3, 5)
    workloads = default_wl if args.workloads is None else tuple(int(x) for x in args.workloads.split(","))
    if args.criterion != "in_out" and 4 in workloads:
        ap.error("the batch workload is stored for in_out only")
    solves5 = args.solves5 if args.solves5 is not None else (8 if args.criterion == "in_out" else 1)
    units = _jobs(args.criterion, workloads, solves5)
    # big units first so the pool stays busy
    units.sort(key=lambda u: {5: 0, 3: 1, 2: 2, 4: 3}[u[1]])
    rows = []
    with mp.get_context("spawn").Pool(min(args.jobs, len(units))) as pool:
        for r in pool.imap_unordered(_run, units):
            rows += r
            print(f"{len(rows)} solves done", flush=True)
    path = out_path(args.criterion)
    if os.path.exists(path):  # keep the rows of workloads not re-run
        with open(path) as f:
            old = json.load(f)["solves"]
        rows += [r for r in old if r["workload"] not in workloads]
    rows.sort(key=lambda r: (r["workload"], r["solve"]))
    out = {"criterion": args.criterion, "criterion_bits": crit_bits(args.criterion),
           "generator": "tests/golden/make_fullsize.py (oracle only)", "solves": rows}
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    main()

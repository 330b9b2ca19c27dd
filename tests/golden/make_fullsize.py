"""Writes fullsize_in_out.json: the oracle's results on the full-size workloads.

    python tests/golden/make_fullsize.py [--jobs J]

For workloads 2 (1024 x 1024 grid), 3 (R-MAT scale 22), 4 (the batch of 256
graphs, 1024 solves) and 5 (G(2^24, 2^28), 8 sources), every solve is run
through the CPU oracle only: binary-heap Dijkstra for the distances and the
phase simulator with IN-STATIC | OUT-STATIC (Section 3's IN and OUT criteria
with static minima) for the phase-by-phase settled sets.  Stored per solve:
phases, sum of |F|, settled and relaxed counts, and SHA-256 digests of the
uint64 distance array (UINT64_MAX = unreachable) and of the uint32
settle-phase array.  The GPU tests compare the library's outputs with these
values; nothing here touches the GPU path.  Workloads come from graphgen's
integer-only generators, so the graphs are the same on every host.
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
OUT = os.path.join(HERE, "fullsize_in_out.json")
WORKLOADS = (2, 3, 4, 5)


def digest(a) -> str:
    return hashlib.sha256(a.tobytes()).hexdigest()[:32]


def _jobs():
    """(workload, [solve indices]) units of work (each unit generates its
    workload once)."""
    units = []
    for k in WORKLOADS:
        if k == 4:  # 1024 solves, 4 per graph, in 6 units
            units += [(4, list(range(lo, min(lo + 172, 1024)))) for lo in range(0, 1024, 172)]
        elif k == 5:
            units += [(5, [j]) for j in range(8)]
        else:
            units.append((k, [0]))
    return units


def _run(unit):
    k, js = unit
    sys.path.insert(0, ROOT)
    import graphgen as gg
    import oracle
    wl = gg.workload(k)
    crit = oracle.IN_STATIC | oracle.OUT_STATIC
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
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()
    units = _jobs()
    # big units first so the pool stays busy
    units.sort(key=lambda u: {5: 0, 3: 1, 2: 2, 4: 3}[u[0]])
    rows = []
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        for r in pool.imap_unordered(_run, units):
            rows += r
            print(f"{len(rows)} solves done", flush=True)
    rows.sort(key=lambda r: (r["workload"], r["solve"]))
    out = {"criterion": "IN_STATIC|OUT_STATIC", "generator": "tests/golden/make_fullsize.py (oracle only)",
           "solves": rows}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", OUT)


if __name__ == "__main__":
    main()

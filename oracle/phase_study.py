"""Phase-count study with the CPU oracle (analysis; test infrastructure only).

    python oracle/phase_study.py [--samples S] [--jobs J] [--approx]

The paper's simulation section counts, for every criterion, the phases the
generic algorithm needs to settle all reachable vertices and the sum of |F|
over those phases, on two families, and fits a + b n^c (a + b log2 n for
ORACLE) to the means:
  - uniform random graphs with mean out-degree 10 (G(n, p), p = 10/(n-1));
  - Kronecker graphs sampled from the initiator 2.5 (0.57 0.19; 0.19 0.05),
    2^k vertices and about 2.5^k edges, k = 7..16.
Stand-ins here (seeded, integer): G(n, m) with m = 10 n (endpoints uniform, no
self-loops) for sizes 2^7 .. 2^16 in steps of sqrt(2); R-MAT edge sampling with
the same quadrant probabilities and round(2.5^k) edges; weights uniform in
[0, 2^24) (the paper's are real in [0, 1]); source 0 for uniform graphs, the
vertex of largest out-degree for R-MAT.  Every count comes from
oracle.simulate (phases and sum of |F|); ORACLE uses oracle.dijkstra's
distances.  Writes oracle/phase_study.json and prints a markdown table.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "phase_study.json")
SEED = 0x1903120850 + 1000

# criterion masks of the oracle (oracle/__init__.py): name -> mask
CRITERIA = [
    ("OUT-STATIC", 2), ("IN-STATIC", 1), ("IN-STATIC|OUT-STATIC", 3),
    ("OUT-SIMPLE", 8), ("IN-SIMPLE", 4), ("IN-SIMPLE|OUT-SIMPLE", 12),
    ("OUT", 256), ("IN", 16), ("IN|OUT", 272),
    ("ORACLE", 128),
]


def uniform_sizes():
    return [int(round(2 ** (7 + h / 2))) for h in range(0, 19)]  # 128 .. 65536


def kron_scales():
    return list(range(7, 17))


def _graph(family: str, size: int, sample: int):
    sys.path.insert(0, ROOT)
    import graphgen as gg
    seed = (SEED + (0 if family == "uniform" else 1 << 40) + size * 1000 + sample) & ((1 << 64) - 1)
    if family == "uniform":
        g = gg.gnm(size, 10 * size, 0, 1 << 24, seed)
        return g, 0
    m = int(round(2.5 ** size))
    g = gg.rmat(size, 0, 0.57, 0.19, 0.19, 0, 1 << 24, seed, m=m)
    return g, gg.max_outdeg_vertex(g)


def _run(task):
    family, size, sample = task
    sys.path.insert(0, ROOT)
    import oracle
    g, s = _graph(family, size, sample)
    d = oracle.dijkstra(g, s)
    out = {"family": family, "size": size, "n": g.n, "sample": sample}
    for name, mask in CRITERIA:
        sim = oracle.simulate(g, s, mask, dist_ref=d)
        out[name] = (sim.phases, sim.sum_f)
    return out


def fit(ns, ys, log_form: bool):
    """Least-squares fit of a + b n^c (or a + b log2 n); returns (a, b, c)."""
    import numpy as np
    from scipy.optimize import curve_fit
    ns = np.asarray(ns, float)
    ys = np.asarray(ys, float)
    if log_form:
        A = np.vstack([np.ones_like(ns), np.log2(ns)]).T
        (a, b), *_ = np.linalg.lstsq(A, ys, rcond=None)
        return float(a), float(b), None
    c0 = math.log(ys[-1] / ys[0]) / math.log(ns[-1] / ns[0])
    b0 = ys[-1] / ns[-1] ** c0
    (a, b, c), _ = curve_fit(lambda x, a, b, c: a + b * x ** c, ns, ys, p0=(0.0, b0, c0), maxfev=20000)
    return float(a), float(b), float(c)


# APPROX(k) sweep (the approximate minima of Section 3's closing remark): the
# static criteria, APPROX(k) for growing k, and IN (full) | OUT-WEAK, which
# APPROX(1) equals; uniform family only.
APPROX_KS = [1, 2, 4, 8, 16, 32]
APPROX_OUT = os.path.join(HERE, "approx_study.json")


def _run_approx(task):
    size, sample = task
    sys.path.insert(0, ROOT)
    import oracle
    g, s = _graph("uniform", size, sample)
    d = oracle.dijkstra(g, s)
    out = {"size": size, "n": g.n, "sample": sample}
    crits = [("IN-STATIC|OUT-STATIC", 3), ("IN|OUT-WEAK", 16 | 32)] + [(f"APPROX({k})", oracle.approx(k))
                                                                        for k in APPROX_KS]
    for name, mask in crits:
        sim = oracle.simulate(g, s, mask, dist_ref=d)
        out[name] = (sim.phases, sim.sum_f)
    return out


def approx_main(samples: int, jobs: int):
    sizes = [1 << e for e in range(10, 19)]
    tasks = sorted([(z, s) for z in sizes for s in range(samples)], key=lambda t: -t[0])
    with mp.get_context("spawn").Pool(jobs) as pool:
        rows = list(pool.imap_unordered(_run_approx, tasks))
    names = ["IN-STATIC|OUT-STATIC"] + [f"APPROX({k})" for k in reversed(APPROX_KS)] + ["IN|OUT-WEAK"]
    result = {"samples": samples, "rows": rows, "fits": {}}
    ns = [sum(r["n"] for r in rows if r["size"] == z) / samples for z in sizes]
    for name in names:
        ph = [sum(r[name][0] for r in rows if r["size"] == z) / samples for z in sizes]
        result["fits"][name] = {"phases": fit(ns, ph, False), "mean_phases": ph, "n": ns}
    with open(APPROX_OUT, "w") as f:
        json.dump(result, f, indent=1)
    print("| criterion | phases fit | mean phases at n = 2^10 | at n = 2^18 |")
    print("|---|---|---:|---:|")
    for name in names:
        a, b, c = result["fits"][name]["phases"]
        ph = result["fits"][name]["mean_phases"]
        print(f"| {name} | {b:.2f} n^{c:.2f} | {ph[0]:.1f} | {ph[-1]:.1f} |")
    print("wrote", APPROX_OUT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=10)
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--approx", action="store_true", help="run the APPROX(k) sweep instead")
    args = ap.parse_args()
    if args.approx:
        approx_main(args.samples, args.jobs)
        return
    tasks = [("uniform", n, s) for n in uniform_sizes() for s in range(args.samples)]
    tasks += [("kronecker", k, s) for k in kron_scales() for s in range(args.samples)]
    tasks.sort(key=lambda t: -(t[1] if t[0] == "uniform" else 2 ** t[1]))
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rows = list(pool.imap_unordered(_run, tasks))
    result = {"samples": args.samples, "rows": rows, "fits": {}}
    for family in ("uniform", "kronecker"):
        fr = [r for r in rows if r["family"] == family]
        sizes = sorted({r["size"] for r in fr})
        ns = [sum(r["n"] for r in fr if r["size"] == z) / args.samples for z in sizes]
        result["fits"][family] = {}
        for name, _ in CRITERIA:
            ph = [sum(r[name][0] for r in fr if r["size"] == z) / args.samples for z in sizes]
            sf = [sum(r[name][1] for r in fr if r["size"] == z) / args.samples for z in sizes]
            result["fits"][family][name] = {
                "phases": fit(ns, ph, name == "ORACLE"), "sum_f": fit(ns, sf, False),
                "n": ns, "mean_phases": ph, "mean_sum_f": sf}
    with open(OUT, "w") as f:
        json.dump(result, f, indent=1)
    print("| criterion | uniform phases | Kronecker phases | uniform sum|F| | Kronecker sum|F| |")
    print("|---|---|---|---|---|")
    for name, _ in CRITERIA:
        cells = []
        for key in ("phases", "sum_f"):
            for family in ("uniform", "kronecker"):
                a, b, c = result["fits"][family][name][key]
                cells.append(f"{b:.2f} log2(n)" if c is None else f"{b:.2f} n^{c:.2f}")
        print(f"| {name} | {cells[0]} | {cells[1]} | {cells[2]} | {cells[3]} |")
    print("wrote", OUT)


if __name__ == "__main__":
    main()

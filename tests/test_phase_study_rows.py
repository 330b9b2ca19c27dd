"""The phase-count study's stored counts (oracle/phase_study.json, written by
oracle/phase_study.py from the oracle alone) against the oracle re-run on the
same seeded graphs (CPU) and against the GPU engine's traces (GPU).

The study reproduces the paper's simulation section (phases and sum of |F|
per criterion on uniform and Kronecker-shaped graphs).  On the GPU every
criterion it implements must give the same phase count and the same sum of
|F| as the simulator on every graph of the subset below.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import phase_study as ps

STUDY = os.path.join(os.path.dirname(oracle.__file__), "phase_study.json")
GPU_MASK = 1 | 2 | 4 | 8 | 16  # IN/OUT static, IN/OUT simple, IN (full)


def _rows(max_uniform, max_kron, samples):
    with open(STUDY) as f:
        rows = json.load(f)["rows"]
    keep = [r for r in rows if r["sample"] < samples and
            ((r["family"] == "uniform" and r["size"] <= max_uniform) or
             (r["family"] == "kronecker" and r["size"] <= max_kron))]
    return sorted(keep, key=lambda r: (r["family"], r["size"], r["sample"]))


def test_stored_rows_are_the_oracles():
    """A few stored rows re-computed by the oracle on graphs rebuilt from the
    study's seeds: every criterion's (phases, sum of |F|) is identical."""
    rows = _rows(512, 9, 1)
    assert len(rows) >= 8
    for r in rows:
        g, s = ps._graph(r["family"], r["size"], r["sample"])
        assert g.n == r["n"]
        d = oracle.dijkstra(g, s)
        for name, mask in ps.CRITERIA:
            sim = oracle.simulate(g, s, mask, dist_ref=d)
            assert [sim.phases, sim.sum_f] == r[name], (r["family"], r["size"], name)


@pytest.mark.gpu
def test_gpu_traces_reproduce_the_study():
    import paper_1903_12085_gb300 as sp

    rows = _rows(4096, 12, 2)
    assert len(rows) >= 30
    checked = 0
    for r in rows:
        g, s = ps._graph(r["family"], r["size"], r["sample"])
        G = sp.Graph.from_csr(g, reverse=True)
        for name, mask in ps.CRITERIA:
            if mask & ~GPU_MASK:
                continue  # ORACLE and OUT (full) exist in the simulator only
            _, st, _, _ = sp.solve_trace(G, s, mask, settle=False)
            assert [st["phases"], st["sum_frontier"]] == r[name], (r["family"], r["size"], r["sample"], name)
            checked += 1
        G.close()
    assert checked == 7 * len(rows)


def test_stored_approx_rows_are_the_oracles():
    """The APPROX(k) sweep (oracle/approx_study.json): stored rows re-computed
    by the oracle; on every row APPROX(1) equals IN (full) | OUT-WEAK; the mean
    phase count never falls as k grows and stays at most the static one."""
    with open(os.path.join(os.path.dirname(oracle.__file__), "approx_study.json")) as f:
        study = json.load(f)
    rows = study["rows"]
    for r in rows:
        assert r["APPROX(1)"] == r["IN|OUT-WEAK"], r["size"]
    for r in [r for r in rows if r["size"] <= 2048 and r["sample"] < 2]:
        g, s = ps._graph("uniform", r["size"], r["sample"])
        d = oracle.dijkstra(g, s)
        for k in ps.APPROX_KS:
            sim = oracle.simulate(g, s, oracle.approx(k), dist_ref=d)
            assert [sim.phases, sim.sum_f] == r[f"APPROX({k})"], (r["size"], k)
    means = [np.mean([r[f"APPROX({k})"][0] for r in rows]) for k in ps.APPROX_KS]
    static = np.mean([r["IN-STATIC|OUT-STATIC"][0] for r in rows])
    assert all(a <= b for a, b in zip(means, means[1:])) and means[-1] <= static

"""Full-size workloads, in the launch configuration bench.py times (default
tuning, one persistent launch per solve or per batch).

Expected values come from tests/golden/fullsize_<criterion>.json, written by
tests/golden/make_fullsize.py from the CPU oracle alone (Dijkstra distances and
the phase simulator's per-vertex settle phases, as SHA-256 digests, plus the
phase and frontier counts), for IN-STATIC | OUT-STATIC on every workload and for
IN-SIMPLE | OUT-SIMPLE, IN (full) | OUT-WEAK and APPROX(4) on the grid, R-MAT
and large G(n, m) workloads.  The cheap single-source workloads are also
compared element by element with a fresh oracle run on this host.  A policy
network trained here switches arms phase by phase on the full grid and on the
large G(n, m) family at a quarter of its size; its logged schedule is
replayed by the simulator.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_1903_12085_gb300")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _gold(criterion="in_out"):
    path = os.path.join(GOLDEN, f"fullsize_{criterion}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def _rows(k, criterion="in_out"):
    return [r for r in _gold(criterion)["solves"] if r["workload"] == k]


def _digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:32]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    sp.set_wait_limit_ns(2_000_000_000)
    sp.set_tuning()
    yield
    sp.set_tuning()


@pytest.mark.parametrize("k", [2, 3, 5], ids=["grid1024", "rmat22", "gnm2p24"])
def test_fullsize_single_source(k):
    wl = gg.workload(k)
    rows = _rows(k)
    assert len(rows) == len(wl.solves)
    g = wl.graphs[0]
    G = sp.Graph.from_csr(g, reverse=False)
    out = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for r in rows:
        gi, s = wl.solves[r["solve"]]
        assert (gi, s, g.n) == (r["graph"], r["source"], r["n"])
        dist, st, settle, _ = sp.solve_trace(G, s, sp.IN_OUT, out=out)
        d = sp.as_uint64(dist)
        assert _digest(d) == r["dist_sha256"], "distances differ from the oracle's"
        assert _digest(settle.astype(np.uint32)) == r["settle_sha256"], "settle phases differ"
        assert (st["phases"], st["sum_frontier"], st["settled"], st["edges_relaxed"]) == \
            (r["phases"], r["sum_f"], r["settled"], r["relaxed"])
        if k in (2, 3):  # element by element against a fresh oracle run
            assert (d == oracle.dijkstra(g, s)).all()
    G.close()


def test_fullsize_batch_one_launch():
    """All 1024 solves of the batch workload in one captured persistent launch."""
    wl = gg.workload(4)
    rows = _rows(4)
    assert len(rows) == len(wl.solves) == 1024
    G = [sp.Graph.from_csr(g, reverse=False) for g in wl.graphs]
    B = sp.Batch([G[i] for i, _ in wl.solves], [s for _, s in wl.solves], sp.IN_OUT)
    B.launch()
    torch.cuda.synchronize()
    phases = B.phases.cpu().numpy()
    for r in rows:
        j = r["solve"]
        assert _digest(sp.as_uint64(B.outs[j])) == r["dist_sha256"], f"solve {j}"
        assert int(phases[j]) == r["phases"], f"solve {j}"
    B.launch()  # a replay gives the same results
    torch.cuda.synchronize()
    assert (B.phases.cpu().numpy() == phases).all()
    B.close()
    for x in G:
        x.close()


def test_fullsize_learned_policy_rmat22():
    """A seeded random network switches arms phase by phase on the full R-MAT
    graph; distances equal Dijkstra's and the simulator, replaying the logged
    per-phase criteria, reproduces every phase's settled set."""
    from oracle import mlp as omlp
    wl = gg.workload(3)
    g = wl.graphs[0]
    _, s = wl.solves[0]
    G = sp.Graph.from_csr(g, reverse=True)
    sp.policy_load(omlp.init(7, scale=1.0).astype(np.float32))
    try:
        dist, st, settle, tr = sp.solve_trace(G, s, sp.IN_OUT | sp.POLICY_LEARNED, trace_cap=1 << 20)
    finally:
        sp.policy_clear()
    ref = oracle.dijkstra(g, s)
    assert (sp.as_uint64(dist) == ref).all()
    sched = tr["criterion"].astype(np.uint32)
    assert set(np.unique(sched)) <= {sp.IN_OUT, sp.IN_SIMPLE | sp.OUT_STATIC}
    sim = oracle.simulate(g, s, sp.IN_OUT, schedule=sched, dist_ref=ref)
    assert sim.phases == st["phases"]
    assert (settle == sim.settle_phase).all()
    G.close()


STRONGER = [(c, k) for c in ("simple", "full_weak", "approx4") for k in (2, 3, 5)]


@pytest.mark.parametrize("criterion,k", STRONGER, ids=[f"{c}-w{k}" for c, k in STRONGER])
def test_fullsize_stronger_criteria(criterion, k):
    """IN-SIMPLE | OUT-SIMPLE, IN (full) | OUT-WEAK and APPROX(4) at full size:
    distances, per-vertex settle phases, phase and frontier counts equal the
    oracle's (every stored solve of the workload)."""
    gold = _gold(criterion)
    if gold is None:
        pytest.skip(f"tests/golden/fullsize_{criterion}.json not generated")
    rows = _rows(k, criterion)
    if not rows:
        pytest.skip(f"no stored solve of workload {k} for {criterion}")
    crit = gold["criterion_bits"]
    wl = gg.workload(k)
    g = wl.graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    out = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for r in rows:
        gi, s = wl.solves[r["solve"]]
        assert (gi, s, g.n) == (r["graph"], r["source"], r["n"])
        dist, st, settle, _ = sp.solve_trace(G, s, crit, out=out)
        d = sp.as_uint64(dist)
        assert _digest(d) == r["dist_sha256"], "distances differ from the oracle's"
        assert _digest(settle.astype(np.uint32)) == r["settle_sha256"], "settle phases differ"
        assert (st["phases"], st["sum_frontier"], st["settled"], st["edges_relaxed"]) == \
            (r["phases"], r["sum_f"], r["settled"], r["relaxed"])
        if k == 2:
            assert (d == oracle.dijkstra(g, s)).all()
    G.close()


@pytest.fixture(scope="module")
def trained_policy():
    """A policy network trained on this GPU by the library's own kernels (on
    the small seeded training graphs, none of them a benchmark graph)."""
    from paper_1903_12085_gb300 import policy as pol
    w, _ = pol.fit_and_load()
    sp.policy_clear()
    return w


@pytest.mark.parametrize("k,shrink", [(2, 0), (5, 2)], ids=["grid1024", "gnm2p22"])
def test_fullsize_trained_policy_replay(k, shrink, trained_policy):
    """The trained network picks each phase's arm on the full 1024 x 1024 grid
    and on G(2^22, 2^26) (the large G(n, m) family at a quarter of its size:
    the simulator's replay of a schedule costs minutes per solve at full
    size).  Distances equal Dijkstra's; the logged per-phase criteria,
    replayed by the simulator, settle the same vertices in every phase."""
    wl = gg.workload(k, shrink=shrink)
    g = wl.graphs[0]
    _, s = wl.solves[0]
    G = sp.Graph.from_csr(g, reverse=True)
    sp.policy_load(trained_policy)
    try:
        dist, st, settle, tr = sp.solve_trace(G, s, sp.IN_OUT | sp.POLICY_LEARNED, trace_cap=1 << 20)
    finally:
        sp.policy_clear()
    G.close()
    assert len(tr) == st["phases"]
    d = sp.as_uint64(dist)
    sched = tr["criterion"].astype(np.uint32)
    assert set(np.unique(sched)) <= {sp.IN_OUT, sp.IN_SIMPLE | sp.OUT_STATIC}
    assert ((tr["arm"] & 0x80) != 0).all()  # every phase logged the policy's choice
    ref = oracle.dijkstra(g, s)
    assert (d == ref).all()
    sim = oracle.simulate(g, s, sp.IN_OUT, schedule=sched, dist_ref=ref)
    assert sim.phases == st["phases"]
    assert (settle == sim.settle_phase).all()
    assert sim.sum_f == st["sum_frontier"]

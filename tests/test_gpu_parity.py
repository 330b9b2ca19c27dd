"""GPU parity: the CUDA phase engine against the CPU oracle, bit for bit.

Distances must equal Dijkstra's; the phase count, the per-vertex settle phase
(i.e. every per-phase settled set S') and the counters must equal the
simulator's for the same criterion.  All inputs are seeded and synthetic."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import oracle_pins as P

sp = pytest.importorskip("paper_1903_12085_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CRITS = [sp.IN_STATIC, sp.OUT_STATIC, sp.IN_OUT, sp.IN_SIMPLE, sp.OUT_SIMPLE, sp.SIMPLE,
         sp.IN_STATIC | sp.OUT_SIMPLE, sp.IN_SIMPLE | sp.OUT_STATIC,
         sp.IN_FULL, sp.OUT_WEAK, sp.IN_FULL | sp.OUT_WEAK, sp.IN_FULL | sp.OUT_STATIC,
         sp.approx(1), sp.approx(3), sp.approx(8) | sp.DIJK]
MODES = [0, sp.FRONTIER_DENSE, sp.FRONTIER_AUTO]


# execution tunings that must not change any result (fields of sssp_tuning; the
# near/far ones force the split on small fringes and a refill every few phases)
TUNINGS = {
    "default": {},
    "grid_only_3blk": dict(solo_max_frontier=0, grid_blocks=3, solo_max_edges=0),
    "solo_3blk": dict(solo_max_frontier=8, grid_blocks=3, solo_max_edges=4096),
    "solo_edges_3blk": dict(solo_max_frontier=4096, grid_blocks=3, solo_max_edges=24),
    "one_block": dict(solo_max_frontier=0, grid_blocks=1, solo_max_edges=0),
    "one_block_solo": dict(solo_max_frontier=4096, grid_blocks=1, solo_max_edges=1 << 30),
    "nearfar_grid_3blk": dict(solo_max_frontier=0, grid_blocks=3, nearfar_min_frontier=4, nearfar_target=6,
                              nearfar_min_share=0),
    "nearfar_solo_3blk": dict(solo_max_frontier=4096, grid_blocks=3, solo_max_edges=64,
                              nearfar_min_frontier=8, nearfar_target=40, nearfar_min_share=0),
    "nearfar_one_block": dict(solo_max_frontier=0, grid_blocks=1, nearfar_min_frontier=1, nearfar_target=1,
                              nearfar_min_share=0),
    "nearfar_auto_target": dict(nearfar_min_frontier=32, nearfar_target=0, nearfar_min_share=8),
}


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    sp.set_wait_limit_ns(2_000_000_000)
    sp.set_tuning()
    yield
    sp.set_tuning()


@pytest.fixture(params=list(TUNINGS), ids=list(TUNINGS))
def tuning(request):
    sp.set_tuning()
    sp.set_tuning(**TUNINGS[request.param])
    yield request.param
    sp.set_tuning()


def check(g, G, s, crit, ref=None, mode=0):
    ref = oracle.dijkstra(g, s) if ref is None else ref
    sim = oracle.simulate(g, s, crit, dist_ref=ref)
    dist, stats, settle, _ = sp.solve_trace(G, s, crit | mode)
    d = sp.as_uint64(dist)
    assert (d == ref).all(), f"distances differ at {np.nonzero(d != ref)[0][:10]}"
    assert stats["phases"] == sim.phases, (stats["phases"], sim.phases)
    assert (settle == sim.settle_phase).all(), f"settle phase differs at {np.nonzero(settle != sim.settle_phase)[0][:10]}"
    assert stats["sum_frontier"] == sim.sum_f
    assert stats["settled"] == sim.settled
    assert stats["edges_relaxed"] == sim.relaxed
    return stats


def test_golden_examples_on_gpu():
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")) as f:
        data = json.load(f)
    for ex in data["examples"]:
        g = gg.from_edges(ex["n"], ex["edges"])
        G = sp.Graph.from_csr(g, reverse=True)
        for run in ex["runs"]:
            if run["crit"] & ~(sp.IN_STATIC | sp.OUT_STATIC | sp.IN_SIMPLE | sp.OUT_SIMPLE | sp.IN_FULL |
                               sp.OUT_WEAK | sp.DIJK):
                continue
            dist, stats, settle, _ = sp.solve_trace(G, 0, run["crit"])
            assert sp.as_uint64(dist).tolist() == [int(x) for x in ex["dist"]], ex["name"]
            assert stats["phases"] == run["phases"], (ex["name"], run)
            assert settle.tolist() == run["settle_phase"], (ex["name"], run)
            assert stats["sum_frontier"] == run["sum_f"], (ex["name"], run)


@pytest.mark.parametrize("mode", MODES, ids=["sparse", "dense", "auto"])
def test_fuzz_tiny_graphs(mode, tuning):
    rng = np.random.default_rng(1234 + mode % 7)
    for case in range(40):
        g = P.random_tiny_graph(rng, n_max=40, w_max=int(rng.choice([0, 3, 50, 2**31])))
        s = int(rng.integers(0, g.n))
        G = sp.Graph.from_csr(g, reverse=True)
        ref = oracle.dijkstra(g, s)
        for crit in CRITS + [sp.DIJK]:
            check(g, G, s, crit, ref, mode)
        G.close()


@pytest.mark.parametrize("crit", CRITS, ids=lambda c: f"crit{c}")
def test_workload1_full(crit, tuning):
    """G(16384, 131072), the full first workload, every criterion."""
    g = gg.workload(1).graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    ref = oracle.dijkstra(g, 0)
    for mode in MODES:
        check(g, G, 0, crit, ref, mode)


def test_workload_shapes_small(tuning):
    """Smaller members of every workload family (several tiles, ragged tails)."""
    cases = [gg.workload(2, shrink=6), gg.workload(3, shrink=8), gg.workload(5, shrink=8)]
    for wl in cases:
        g = wl.graphs[0]
        G = sp.Graph.from_csr(g, reverse=True)
        for _, s in wl.solves[:2]:
            ref = oracle.dijkstra(g, s)
            for crit in [sp.IN_OUT, sp.SIMPLE, sp.IN_FULL | sp.OUT_WEAK, sp.approx(4)]:
                for mode in MODES:
                    check(g, G, s, crit, ref, mode)


def _d2h(ptr, count, dtype):
    """Copy `count` elements from a raw device pointer (the library's own
    libcudart is already loaded, so dlopen returns it by soname)."""
    import ctypes
    cudart = ctypes.CDLL("libcudart.so.13")
    out = np.empty(count, dtype)
    rc = cudart.cudaMemcpy(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(ptr), ctypes.c_size_t(out.nbytes), 2)
    assert rc == 0
    return out


def test_preprocessing_matches_definitions():
    """Rows sorted by (cost, target); static minima equal their definitions;
    the in-edge CSR holds every edge once, rows sorted by (cost, source)."""
    g = gg.workload(3, shrink=10).graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    arr = G.device_arrays()
    m, n = g.m, g.n
    edges = _d2h(arr["edges"], 2 * m, np.uint32).reshape(m, 2)
    out_min = _d2h(arr["out_min"], n, np.uint32)
    in_min = _d2h(arr["in_min"], n, np.uint32)
    rro = _d2h(arr["rrow_off"], n + 1, np.uint64).astype(np.int64)
    redges = _d2h(arr["redges"], 2 * m, np.uint32).reshape(m, 2)
    ro = g.row_off.astype(np.int64)
    src = np.repeat(np.arange(n), np.diff(ro))
    for u in range(n):
        row = edges[ro[u]:ro[u + 1]]
        ref_row = sorted(zip(g.w[ro[u]:ro[u + 1]].tolist(), g.col[ro[u]:ro[u + 1]].tolist()))
        assert [(int(b), int(a)) for a, b in row] == ref_row
        assert out_min[u] == (min(g.w[ro[u]:ro[u + 1]]) if ro[u + 1] > ro[u] else 0xFFFFFFFF)
    ref_in = np.full(n, 0xFFFFFFFF, np.uint64)
    np.minimum.at(ref_in, g.col.astype(np.int64), g.w.astype(np.uint64))
    assert (in_min.astype(np.uint64) == ref_in).all()
    indeg = np.bincount(g.col.astype(np.int64), minlength=n)
    assert (np.diff(rro) == indeg).all() and rro[0] == 0
    order = np.lexsort((src, g.w, g.col))  # by target, then cost, then source
    ref_rev = np.stack([src[order], g.w[order]], axis=1)
    assert (redges.astype(np.int64) == ref_rev.astype(np.int64)).all()


def test_long_rows_sorted():
    """Rows longer than one block's sort (merge passes) come out sorted."""
    rng = np.random.default_rng(7)
    n = 3000
    edges = [(0, int(rng.integers(0, n)), int(rng.integers(0, 1000))) for _ in range(20000)]
    edges += [(1, int(rng.integers(0, n)), int(rng.integers(0, 10))) for _ in range(9000)]
    edges += [(u, (u * 7 + 1) % n, int(rng.integers(0, 99))) for u in range(2, n)]
    g = gg.from_edges(n, edges)
    G = sp.Graph.from_csr(g, reverse=True)
    for s in (0, 1, 5):
        ref = oracle.dijkstra(g, s)
        for crit in (sp.IN_OUT, sp.SIMPLE):
            check(g, G, s, crit, ref)


def test_device_inputs_equal_host_inputs():
    g = gg.workload(1, shrink=2).graphs[0]
    ro = torch.from_numpy(g.row_off.view(np.int64)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    w = torch.from_numpy(g.w.view(np.int32)).cuda()
    Gd = sp.Graph(g.n, ro, col, w, reverse=True)
    Gh = sp.Graph.from_csr(g, reverse=True)
    for crit in (sp.IN_OUT, sp.SIMPLE):
        a, pa = sp.solve(Gd, 0, crit)
        b, pb = sp.solve(Gh, 0, crit)
        assert (sp.as_uint64(a) == sp.as_uint64(b)).all() and pa == pb


def test_host_dist_buffer():
    g = gg.workload(1, shrink=2).graphs[0]
    G = sp.Graph.from_csr(g)
    out = np.zeros(g.n, np.uint64)
    _, phases = sp.solve(G, 0, sp.IN_OUT, out=out)
    assert (out == oracle.dijkstra(g, 0)).all()
    assert phases == oracle.simulate(g, 0, sp.IN_OUT).phases


def test_edge_cases():
    # single vertex, no edges
    g = gg.from_edges(1, [])
    G = sp.Graph.from_csr(g, reverse=True)
    dist, stats, settle, _ = sp.solve_trace(G, 0, sp.IN_OUT)
    assert sp.as_uint64(dist).tolist() == [0] and stats["phases"] == 1 and settle.tolist() == [1]
    # source without out-edges, others unreachable
    g = gg.from_edges(4, [(1, 2, 3), (2, 3, 4)])
    G = sp.Graph.from_csr(g, reverse=True)
    for crit in CRITS:
        check(g, G, 0, crit)
    # largest costs: distances near 2^33 per edge, sums exact in uint64
    big = 0xFFFFFFFE
    g = gg.from_edges(5, [(0, 1, big), (1, 2, big), (2, 3, big), (0, 3, big), (3, 4, 0), (4, 4, big)])
    G = sp.Graph.from_csr(g, reverse=True)
    for crit in CRITS:
        check(g, G, 0, crit)


def test_invalid_arguments_are_rejected():
    g = gg.from_edges(3, [(0, 1, 1), (1, 2, 2)])
    with pytest.raises(sp.SsspError) as e:
        sp.Graph(3, g.row_off, g.col, np.array([1, 0xFFFFFFFF], np.uint32))
    assert e.value.status == 1
    with pytest.raises(sp.SsspError) as e:
        sp.Graph(3, g.row_off, np.array([1, 7], np.uint32), g.w)
    assert e.value.status == 1
    with pytest.raises(sp.SsspError) as e:
        sp.Graph(3, np.array([0, 2, 1, 2], np.uint64), g.col, g.w)
    assert e.value.status == 1
    # device-side validation of device inputs
    with pytest.raises(sp.SsspError) as e:
        sp.Graph(3, torch.tensor([0, 1, 2, 2], dtype=torch.int64, device="cuda"),
                 torch.tensor([1, 9], dtype=torch.int32, device="cuda"),
                 torch.tensor([1, 1], dtype=torch.int32, device="cuda"))
    assert e.value.status == 1
    G = sp.Graph.from_csr(g)  # no reverse CSR
    with pytest.raises(sp.SsspError) as e:
        sp.solve(G, 5, sp.IN_OUT)
    assert e.value.status == 1
    with pytest.raises(sp.SsspError) as e:
        sp.solve(G, 0, 0)
    assert e.value.status == 1
    with pytest.raises(sp.SsspError) as e:
        sp.solve(G, 0, sp.IN_SIMPLE)
    assert e.value.status == 6
    # the handle still works after the rejected calls
    d, ph = sp.solve(G, 0, sp.IN_OUT)
    assert sp.as_uint64(d).tolist() == [0, 1, 3]


def test_bounded_wait_runs_out_and_context_survives():
    """A device wait on a flag that nothing sets gives up after its limit with
    SSSP_ERR_TIMEOUT (no trap, no hang); the context stays usable."""
    import time
    t0 = time.perf_counter()
    assert sp.selftest_wait(50_000_000) == 4
    assert time.perf_counter() - t0 < 10
    g = gg.workload(1).graphs[0]
    G = sp.Graph.from_csr(g)
    d, phases = sp.solve(G, 0, sp.IN_OUT)
    assert (sp.as_uint64(d) == oracle.dijkstra(g, 0)).all()


def test_zero_wait_limit_solve_ends_cleanly():
    """With a 0 ns barrier limit a multi-block solve either finishes or stops
    with SSSP_ERR_TIMEOUT; either way the next solve is exact."""
    g = gg.workload(1).graphs[0]
    G = sp.Graph.from_csr(g)
    sp.set_wait_limit_ns(0)
    try:
        try:
            d, _ = sp.solve(G, 0, sp.IN_OUT)
            assert (sp.as_uint64(d) == oracle.dijkstra(g, 0)).all()
        except sp.SsspError as e:
            assert e.status == 4
    finally:
        sp.set_wait_limit_ns(2_000_000_000)
    d, phases = sp.solve(G, 0, sp.IN_OUT)
    assert (sp.as_uint64(d) == oracle.dijkstra(g, 0)).all()


def test_batch_matches_oracle():
    wl = gg.workload(4, shrink=4)
    Gs = [sp.Graph.from_csr(g, reverse=True) for g in wl.graphs]
    graphs = [Gs[i] for i, _ in wl.solves]
    sources = [s for _, s in wl.solves]
    for crit in (sp.IN_OUT, sp.SIMPLE):
        outs, phases = sp.solve_batch(graphs, sources, crit)
        for k, (i, s) in enumerate(wl.solves):
            g = wl.graphs[i]
            ref = oracle.dijkstra(g, s)
            assert (sp.as_uint64(outs[k]) == ref).all(), k
            assert phases[k] == oracle.simulate(g, s, crit).phases, k


def test_prepared_batch_replays():
    wl = gg.workload(4, shrink=5)
    Gs = [sp.Graph.from_csr(g) for g in wl.graphs]
    B = sp.Batch([Gs[i] for i, _ in wl.solves], [s for _, s in wl.solves], sp.IN_OUT)
    for rep in range(3):
        for o in B.outs:
            o.fill_(0)
        B.launch()
        torch.cuda.synchronize()
        ph = B.phases.cpu().numpy()
        for k, (i, s) in enumerate(wl.solves):
            g = wl.graphs[i]
            assert (sp.as_uint64(B.outs[k]) == oracle.dijkstra(g, s)).all()
            assert ph[k] == oracle.simulate(g, s, sp.IN_OUT).phases
    B.close()


def test_batch_autotune_keeps_results():
    """The autotuner walks the blocks-per-solve ladder and re-captures the launch
    with the fastest candidate it timed; the replayed batch still gives the
    oracle's output."""
    wl = gg.workload(4, shrink=5)
    Gs = [sp.Graph.from_csr(g) for g in wl.graphs]
    B = sp.Batch([Gs[i] for i, _ in wl.solves], [s for _, s in wl.solves], sp.IN_OUT)
    bpg, ms = B.autotune()
    assert ms > 0 and bpg >= 1 and (bpg & (bpg - 1) == 0 or bpg >= 128)
    for o in B.outs:
        o.fill_(0)
    B.launch()
    torch.cuda.synchronize()
    ph = B.phases.cpu().numpy()
    for k, (i, s) in enumerate(wl.solves):
        g = wl.graphs[i]
        assert (sp.as_uint64(B.outs[k]) == oracle.dijkstra(g, s)).all()
        assert ph[k] == oracle.simulate(g, s, sp.IN_OUT).phases
    B.close()


@pytest.mark.parametrize("crit", [sp.IN_OUT, sp.IN_STATIC, sp.OUT_STATIC], ids=["in_out", "in", "out"])
def test_nearfar_split_runs_and_changes_nothing(crit):
    """With a small split threshold the fringe is split and its bound raised
    many times (trace arm bits 2: split active, 3: full refill, 4: pull from the
    far-vertex bucket lists); every per-phase figure still equals the oracle's."""
    g = gg.workload(1).graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    ref = oracle.dijkstra(g, 0)
    sim = oracle.simulate(g, 0, crit, dist_ref=ref, trace=True)
    refills = pulls = 0
    try:
        for tune in ["nearfar_grid_3blk", "nearfar_solo_3blk", "nearfar_auto_target"]:
            sp.set_tuning()
            sp.set_tuning(**TUNINGS[tune])
            check(g, G, 0, crit, ref)
            _, st, _, tr = sp.solve_trace(G, 0, crit, trace_cap=1 << 20)
            arm = tr["arm"].astype(np.uint32)
            assert (arm & 4).any() and ((arm & 24) != 0).sum() >= 2, tune
            refills += int(((arm & 8) != 0).sum())
            pulls += int(((arm & 16) != 0).sum())
            q, f = tr["queued"], tr["frontier"]
            assert (q <= f).all() and (q[(arm & 4) == 0] == f[(arm & 4) == 0]).all()
            assert (q < f).any()  # some phases scanned only the near part
            assert (tr["frontier"] == sim.trace[:, 0]).all()
            assert (tr["settled"] == sim.trace[:, 1]).all()
            assert (tr["min_d"] == sim.trace[:, 2]).all()  # thresholds exact after every refill
            if crit & sp.OUT_STATIC:
                assert (tr["min_out"] == sim.trace[:, 3]).all()
        assert refills >= 1 and pulls >= 1, (refills, pulls)  # both ways of raising B ran
        sp.set_tuning()
        sp.set_tuning(**TUNINGS["nearfar_grid_3blk"])
        _, _, _, tr = sp.solve_trace(G, 0, sp.SIMPLE, trace_cap=1 << 20)
        assert not (tr["arm"].astype(np.uint32) & 28).any()  # dynamic IN: never split
    finally:
        sp.set_tuning()


def test_trace_timestamps_are_ordered(tuning):
    """Every phase record's interval lies after the previous one's (solo
    episodes, hand-offs to the group, near/far refills included)."""
    g = gg.workload(1).graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    for crit in [sp.IN_OUT, sp.SIMPLE]:
        _, st, _, tr = sp.solve_trace(G, 0, crit, trace_cap=1 << 20)
        t0 = tr["t_start_ns"].astype(np.int64)
        t1 = tr["t_end_ns"].astype(np.int64)
        assert len(tr) == st["phases"] and (t0 > 0).all()
        assert (t1 >= t0).all()
        assert (t0[1:] >= t1[:-1]).all()
        assert (tr["select_ns"].astype(np.int64) <= t1 - t0).all()

"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each ``pin_*`` function takes the oracle module and raises AssertionError when
the oracle disagrees with something derived independently of it: worked
examples computed by hand (tests/golden), closed forms, brute force, or
theorems about the phased algorithm of Section 3.  ``test_oracle.py`` runs them
on the real oracle; ``test_oracle_mutations.py`` runs them on deliberately
broken copies of the oracle to show that plausible mistakes are caught.
"""
from __future__ import annotations

import json
import os
from collections import deque

import numpy as np

import graphgen as gg

INF = 0xFFFFFFFFFFFFFFFF
HERE = os.path.dirname(os.path.abspath(__file__))

# criterion masks used throughout (interface values)
IN_STATIC, OUT_STATIC, IN_SIMPLE, OUT_SIMPLE = 1, 2, 4, 8
IN_FULL, OUT_WEAK, DIJK, ORACLE, OUT_FULL = 16, 32, 64, 128, 256
SOUND_COMPLETE = [
    IN_STATIC, OUT_STATIC, IN_STATIC | OUT_STATIC, IN_SIMPLE, OUT_SIMPLE, IN_SIMPLE | OUT_SIMPLE,
    IN_FULL, OUT_WEAK, IN_FULL | OUT_WEAK, OUT_FULL, IN_FULL | OUT_FULL, DIJK, ORACLE,
]


def random_tiny_graph(rng, n_max=12, w_max=6, p_self=0.1):
    """Tiny random multigraph: zero weights, self-loops, parallel edges and
    unreachable vertices all occur."""
    n = int(rng.integers(1, n_max + 1))
    m = int(rng.integers(0, 3 * n + 1))
    edges = []
    for _ in range(m):
        u = int(rng.integers(0, n))
        v = u if rng.random() < p_self else int(rng.integers(0, n))
        edges.append((u, v, int(rng.integers(0, w_max + 1))))
    return gg.from_edges(n, edges)


def edges_of(g):
    deg = np.diff(g.row_off.astype(np.int64))
    src = np.repeat(np.arange(g.n), deg)
    return src, g.col.astype(np.int64), g.w.astype(np.int64)


def bfs_reachable(g, s):
    seen = np.zeros(g.n, bool)
    seen[s] = True
    q = deque([s])
    while q:
        u = q.popleft()
        for e in range(int(g.row_off[u]), int(g.row_off[u + 1])):
            t = int(g.col[e])
            if not seen[t]:
                seen[t] = True
                q.append(t)
    return seen


def all_paths_dist(g, s):
    """Minimum cost over all simple paths, by enumeration (n <= 7)."""
    adj = [[] for _ in range(g.n)]
    for e_u, e_v, e_w in zip(*edges_of(g)):
        adj[e_u].append((int(e_v), int(e_w)))
    best = [INF] * g.n
    best[s] = 0

    def walk(u, cost, onpath):
        for v, c in adj[u]:
            if v in onpath:
                continue
            if cost + c < best[v]:
                best[v] = cost + c
            onpath.add(v)
            walk(v, cost + c, onpath)
            onpath.discard(v)

    walk(s, 0, {s})
    return np.array(best, dtype=np.uint64)


def min_hops_on_shortest_paths(g, dist, s):
    """BFS over tight edges (dist[u] + c == dist[v]): the least number of edges
    on any shortest path to each vertex (-1 if unreachable)."""
    h = np.full(g.n, -1, np.int64)
    h[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for e in range(int(g.row_off[u]), int(g.row_off[u + 1])):
            t = int(g.col[e])
            if h[t] < 0 and int(dist[u]) + int(g.w[e]) == int(dist[t]):
                h[t] = h[u] + 1
                q.append(t)
    return h


# ---------------------------------------------------------------------------
# pins

def pin_golden_examples(O):
    """Hand-derived phase sets of tests/golden/hand_examples.json."""
    with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
        data = json.load(f)
    for ex in data["examples"]:
        g = gg.from_edges(ex["n"], ex["edges"])
        dist = np.array(ex["dist"], np.uint64)
        assert (O.dijkstra(g, 0) == dist).all(), ex["name"]
        for run in ex["runs"]:
            r = O.simulate(g, 0, run["crit"], dist_ref=dist)
            tag = f'{ex["name"]} crit={run["crit"]}'
            assert r.phases == run["phases"], (tag, r.phases)
            assert r.sum_f == run["sum_f"], (tag, r.sum_f)
            assert r.settle_phase.tolist() == run["settle_phase"], (tag, r.settle_phase.tolist())
            assert (r.d == dist).all(), tag


def pin_bellman_ford_fuzz(O, cases=10000, seed=11):
    """Dijkstra equals Bellman-Ford on random tiny multigraphs."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        g = random_tiny_graph(rng)
        s = int(rng.integers(0, g.n))
        a = O.dijkstra(g, s)
        b = O.bellman_ford(g, s)
        assert (a == b).all(), (g.row_off, g.col, g.w, s, a, b)


def pin_path_enumeration(O, cases=300, seed=12):
    """Dijkstra and Bellman-Ford equal the minimum over all simple paths."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=6, w_max=9)
        s = int(rng.integers(0, g.n))
        ref = all_paths_dist(g, s)
        assert (O.dijkstra(g, s) == ref).all()
        assert (O.bellman_ford(g, s) == ref).all()


def pin_unit_grid(O, rows=7, cols=11):
    """Unit-weight grid from a corner: d = Manhattan distance; every criterion
    that settles all vertices of minimum d needs rows+cols-1 phases (one
    anti-diagonal per phase); DIJK needs rows*cols."""
    g = gg.grid(rows, cols, 1, 2, 5)
    r_, c_ = np.divmod(np.arange(rows * cols), cols)
    manhattan = (r_ + c_).astype(np.uint64)
    assert (O.dijkstra(g, 0) == manhattan).all()
    for crit in [IN_STATIC, OUT_STATIC, IN_STATIC | OUT_STATIC, IN_SIMPLE, OUT_SIMPLE,
                 IN_SIMPLE | OUT_SIMPLE, IN_FULL | OUT_WEAK, ORACLE]:
        r = O.simulate(g, 0, crit, dist_ref=manhattan)
        assert r.phases == rows + cols - 1, (crit, r.phases)
        assert (r.settle_phase.astype(np.int64) == manhattan.astype(np.int64) + 1).all(), crit
        assert r.sum_f == rows * cols, crit
    assert O.simulate(g, 0, DIJK, dist_ref=manhattan).phases == rows * cols


def pin_path_graph(O, n=40, seed=13):
    """Directed path 0->1->...->n-1: prefix sums; one vertex per phase."""
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 1000, n - 1)
    g = gg.from_edges(n, [(i, i + 1, int(w[i])) for i in range(n - 1)])
    pref = np.concatenate([[0], np.cumsum(w)]).astype(np.uint64)
    assert (O.dijkstra(g, 0) == pref).all()
    for crit in SOUND_COMPLETE:
        r = O.simulate(g, 0, crit, dist_ref=pref)
        assert r.phases == n and (r.d == pref).all(), crit
        assert r.settle_phase.tolist() == list(range(1, n + 1)), crit


def pin_out_star(O, leaves=25, seed=14):
    """Out-star from the centre: d(leaf) = its edge cost; IN and OUT settle
    all leaves in phase 2 (a leaf's only in-edge is its own, and leaves have
    no out-edges); DIJK settles one leaf per phase."""
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 50, leaves)
    g = gg.from_edges(leaves + 1, [(0, i + 1, int(w[i])) for i in range(leaves)])
    ref = np.concatenate([[0], w]).astype(np.uint64)
    assert (O.dijkstra(g, 0) == ref).all()
    for crit in [IN_STATIC, OUT_STATIC, IN_SIMPLE, OUT_SIMPLE, IN_FULL, OUT_WEAK, ORACLE]:
        r = O.simulate(g, 0, crit, dist_ref=ref)
        assert r.phases == 2, (crit, r.phases)
    assert O.simulate(g, 0, DIJK, dist_ref=ref).phases == leaves + 1


def pin_oracle_hops(O, cases=150, seed=15):
    """ORACLE settles v exactly in phase 1 + (least number of edges on a
    shortest path to v), so phases(ORACLE) = 1 + max over reached v."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=40, w_max=3)
        s = int(rng.integers(0, g.n))
        dist = O.bellman_ford(g, s)
        h = min_hops_on_shortest_paths(g, dist, s)
        r = O.simulate(g, s, ORACLE, dist_ref=dist)
        reached = h >= 0
        assert (r.settle_phase[reached].astype(np.int64) == h[reached] + 1).all()
        assert (r.settle_phase[~reached] == 0).all()
        assert r.phases == 1 + int(h.max())


def pin_distance_invariants(O, seed=16):
    """On sampled workload-shaped graphs: d(v) <= d(u)+c(u,v) on every edge
    out of a reached u, a tight in-edge for every reached v != s, and the
    reached set equals BFS reachability."""
    graphs = [(gg.workload(1, shrink=2).graphs[0], 0), (gg.workload(2, shrink=8).graphs[0], 0),
              (gg.workload(3, shrink=12).graphs[0], None)]
    for g, s in graphs:
        if s is None:
            s = gg.max_outdeg_vertex(g)
        d = O.dijkstra(g, s)
        src, dst, w = edges_of(g)
        du = d[src].astype(object)
        dv = d[dst].astype(object)
        fin = d[src] != INF
        assert all(dv[fin] <= du[fin] + w[fin].astype(object))
        tight = fin & (d[src] + w.astype(np.uint64) == d[dst])
        has_tight = np.zeros(g.n, bool)
        has_tight[dst[tight]] = True
        reached = d != INF
        reached_ns = reached.copy()
        reached_ns[s] = False
        assert has_tight[reached_ns].all()
        assert (reached == bfs_reachable(g, s)).all()


def pin_soundness_fuzz(O, cases=400, seed=17):
    """Every criterion of Section 3 is sound and complete (Lemmas 1-2 and the
    weakenings): on random graphs the simulator never settles an incorrect
    vertex, never stalls, and ends with Dijkstra's distances; phases lie
    between ORACLE's and the number of reachable vertices."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=30, w_max=int(rng.choice([0, 2, 10, 1000])))
        s = int(rng.integers(0, g.n))
        dist = O.bellman_ford(g, s)
        nreach = int((dist != INF).sum())
        lo = O.simulate(g, s, ORACLE, dist_ref=dist).phases
        for crit in SOUND_COMPLETE:
            r = O.simulate(g, s, crit, dist_ref=dist)
            assert (r.d == dist).all(), crit
            assert lo <= r.phases <= nreach, (crit, lo, r.phases, nreach)
            assert r.settled == nreach
        assert O.simulate(g, s, DIJK, dist_ref=dist).phases == nreach


def pin_strength_chain(O, cases=40, seed=18):
    """On the same state (same schedule prefix), the settled sets nest:
    DIJK <= IN-STATIC <= IN-SIMPLE <= IN and OUT-STATIC <= OUT-SIMPLE <=
    OUT-WEAK <= OUT (the implication chain of Section 3)."""
    rng = np.random.default_rng(seed)
    chains = [[DIJK, IN_STATIC, IN_SIMPLE, IN_FULL], [OUT_STATIC, OUT_SIMPLE, OUT_WEAK, OUT_FULL]]
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=25, w_max=20)
        s = int(rng.integers(0, g.n))
        dist = O.bellman_ford(g, s)
        base = O.simulate(g, s, IN_STATIC | OUT_STATIC, dist_ref=dist)
        for k in range(base.phases):
            prefix = [IN_STATIC | OUT_STATIC] * k
            for chain in chains:
                prev = None
                for crit in chain:
                    r = O.simulate(g, s, crit, schedule=prefix + [crit], dist_ref=dist)
                    cur = set(np.nonzero(r.settle_phase == k + 1)[0].tolist())
                    if prev is not None:
                        assert prev <= cur, (k, crit, prev, cur)
                    prev = cur


def pin_trace_accounting(O, seed=19):
    """Per-phase trace sums to the totals; |S'| >= 1; minD is non-decreasing."""
    g = gg.workload(1, shrink=3).graphs[0]
    dist = O.dijkstra(g, 0)
    for crit in [IN_STATIC | OUT_STATIC, IN_SIMPLE | OUT_SIMPLE, IN_FULL | OUT_WEAK]:
        r = O.simulate(g, 0, crit, dist_ref=dist, trace=True)
        t = r.trace
        assert int(t[:, 0].sum()) == r.sum_f
        assert int(t[:, 1].sum()) == r.settled == int((dist != INF).sum())
        assert int(t[:, 4].sum()) == r.relaxed == int(g.outdeg()[dist != INF].sum())
        assert (t[:, 1] >= 1).all()
        assert (np.diff(t[:, 2].astype(np.float64)) >= 0).all()
        assert all(int(t[i, 5]) == crit for i in range(len(t)))


def pin_approx_k1_is_full_weak(O, cases=120, seed=20):
    """APPROX(1) recomputes the exact IN (full) / OUT-WEAK terms in every
    phase, so it must settle exactly what IN (full) | OUT-WEAK settles."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=30, w_max=int(rng.choice([3, 50, 2**20])))
        s = int(rng.integers(0, g.n))
        ref = O.dijkstra(g, s)
        a = O.simulate(g, s, O.APPROX | (1 << 10), dist_ref=ref)
        b = O.simulate(g, s, O.IN_FULL | O.OUT_WEAK, dist_ref=ref)
        assert a.phases == b.phases and (a.settle_phase == b.settle_phase).all()


def pin_approx_sound_between(O, cases=80, seed=21):
    """APPROX(k) is sound (the simulator checks against Dijkstra) and, on the
    same state, selects at least what the static criteria select and at most
    what IN (full) | OUT-WEAK selects; its OUT threshold lies between the
    static one and the exact OUT-WEAK one (every value between the static
    minimum and the exact term)."""
    rng = np.random.default_rng(seed)
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=30, w_max=int(rng.choice([3, 50, 2**20])))
        s = int(rng.integers(0, g.n))
        ref = O.dijkstra(g, s)
        for k in (2, 3, 8):
            crit = O.APPROX | (k << 10)
            base = O.simulate(g, s, crit, dist_ref=ref)
            for p in range(1, base.phases):
                sets, thr = [], []
                for last in (O.IN_STATIC | O.OUT_STATIC, crit, O.IN_FULL | O.OUT_WEAK):
                    sched = np.array([crit] * p + [last], np.uint32)
                    sim = O.simulate(g, s, crit, schedule=sched, dist_ref=ref, trace=True)
                    sets.append(set(np.nonzero(sim.settle_phase == p + 1)[0].tolist()))
                    thr.append(int(sim.trace[p, 3]))
                assert sets[0] <= sets[1] <= sets[2]
                assert thr[0] <= thr[1] <= thr[2], (p, thr)


def pin_dijkstra_prefix(O, cases=300, seed=22):
    """A Dijkstra run stopped after k settled vertices has settled the k
    reachable vertices of least distance (distances from Bellman-Ford, the
    reachable set from BFS): its settled count is min(k, reachable) and its
    scanned-edge count is the sum of their out-degrees (graphs whose k-th and
    (k+1)-th distances tie are skipped: either vertex may come first)."""
    rng = np.random.default_rng(seed)
    checked = 0
    for _ in range(cases):
        g = random_tiny_graph(rng, n_max=14, w_max=1000)
        s = int(rng.integers(0, g.n))
        bf = O.bellman_ford(g, s)
        reach = bfs_reachable(g, s)
        deg = np.diff(g.row_off.astype(np.int64))
        order = sorted(np.flatnonzero(reach), key=lambda v: int(bf[v]))
        for k in range(0, g.n + 2):
            settled, scanned = O.dijkstra_prefix(g, s, k)
            kk = min(k, len(order))
            assert settled == kk, (k, settled, kk)
            if 0 < kk < len(order) and bf[order[kk - 1]] == bf[order[kk]]:
                continue
            assert scanned == int(deg[order[:kk]].sum()), (k, scanned)
            checked += 1
    assert checked > 1000


ALL_PINS = [pin_golden_examples, pin_bellman_ford_fuzz, pin_path_enumeration, pin_unit_grid,
            pin_path_graph, pin_out_star, pin_oracle_hops, pin_distance_invariants,
            pin_soundness_fuzz, pin_strength_chain, pin_trace_accounting,
            pin_approx_k1_is_full_weak, pin_approx_sound_between, pin_dijkstra_prefix]

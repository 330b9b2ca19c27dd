"""Per-phase policy network on the GPU: the FP32 training kernels against the
float64 oracle, exactness of solves that switch arms every phase (the
simulator replays the logged schedule), and what a trained network gains."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import mlp as omlp

sp = pytest.importorskip("paper_1903_12085_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield
    sp.policy_clear()
    sp.set_tuning()


def _batch(seed, B=777):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=(B, 8)).astype(np.float32)
    t = rng.normal(0, 2, size=B).astype(np.float32)
    a = rng.integers(0, 4, size=B).astype(np.uint32)
    return x, t, a


def _cuda(a):
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_forward_matches_oracle():
    w = omlp.init(1).astype(np.float32)
    x, _, _ = _batch(2)
    y = sp.mlp_forward(_cuda(w), _cuda(x)).cpu().numpy()
    ref, _ = omlp.forward(w.astype(np.float64), x.astype(np.float64))
    assert np.allclose(y, ref, rtol=1e-4, atol=1e-5)


def test_backward_matches_oracle():
    w = omlp.init(3).astype(np.float32)
    x, t, a = _batch(4)
    g, loss = sp.mlp_backward(_cuda(w), _cuda(x), _cuda(t), _cuda(a))
    g = g.cpu().numpy()
    L, gref = omlp.backward(w.astype(np.float64), x.astype(np.float64), t.astype(np.float64), a)
    assert np.isclose(float(loss.item()), L, rtol=1e-4)
    scale = np.abs(gref).max()
    assert np.abs(g - gref).max() <= 1e-4 * scale, np.abs(g - gref).max() / scale
    # deterministic: a second call gives the same bits
    g2, _ = sp.mlp_backward(_cuda(w), _cuda(x), _cuda(t), _cuda(a))
    assert np.array_equal(g, g2.cpu().numpy())


def test_adam_step_matches_formula():
    rng = np.random.default_rng(5)
    w = rng.normal(size=1476).astype(np.float32)
    g = rng.normal(size=1476).astype(np.float32)
    m1 = rng.normal(size=1476).astype(np.float32) * 0.1
    m2 = np.abs(rng.normal(size=1476)).astype(np.float32) * 0.1
    W, G, M1, M2 = (_cuda(v.copy()) for v in (w, g, m1, m2))
    sp.mlp_adam(W, G, M1, M2, lr=0.01, step=3)
    b1, b2, eps = 0.9, 0.999, 1e-8
    a = b1 * m1.astype(np.float64) + (1 - b1) * g
    b = b2 * m2.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    ref = w - 0.01 * (a / (1 - b1 ** 3)) / (np.sqrt(b / (1 - b2 ** 3)) + eps)
    assert np.allclose(W.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


TUNINGS = [(4096, 0, 2048), (0, 3, 0), (8, 3, 24)]


@pytest.mark.parametrize("tune", TUNINGS, ids=["default", "grid3", "solo3_handoff"])
def test_policy_solves_are_exact_and_replayable(tune):
    """A random network switches arms from phase to phase; distances equal
    Dijkstra's and the simulator, fed the logged per-phase criteria, settles
    exactly the same vertices in every phase."""
    sp.set_tuning(solo_max_frontier=tune[0], grid_blocks=tune[1], solo_max_edges=tune[2])
    try:
        for seed in range(3):
            sp.policy_load(omlp.init(100 + seed, scale=1.0).astype(np.float32))
            for wl in [gg.workload(1, shrink=2), gg.workload(3, shrink=12), gg.workload(2, shrink=10)]:
                gi, s = wl.solves[0]
                g = wl.graphs[gi]
                G = sp.Graph.from_csr(g, reverse=True)
                d, st, settle, tr = sp.solve_trace(G, s, sp.IN_OUT | sp.POLICY_LEARNED, trace_cap=1 << 20)
                ref = oracle.dijkstra(g, s)
                assert (sp.as_uint64(d) == ref).all()
                sched = tr["criterion"].astype(np.uint32)
                assert set(np.unique(sched)) <= {sp.IN_OUT, sp.IN_SIMPLE | sp.OUT_STATIC}
                assert ((tr["arm"] & 0x80) != 0).all()
                sim = oracle.simulate(g, s, sp.IN_OUT, schedule=sched, dist_ref=ref)
                assert st["phases"] == sim.phases
                assert (settle == sim.settle_phase).all()
                assert st["sum_frontier"] == sim.sum_f
    finally:
        sp.set_tuning()


@pytest.mark.parametrize("bpg", [1, 3], ids=["bpg1", "bpg3"])
def test_batched_policy_solves_are_exact_and_replayable(bpg):
    """The learned policy inside one batched persistent launch: graphs of
    three families with two sources each, a random network switching arms
    phase by phase in every group.  Every solve's distances equal Dijkstra's;
    for traced solves the simulator, fed the logged per-phase criteria,
    settles the same vertices in every phase (soundness of switching: any
    disjunction of sound criteria is sound, Section 3)."""
    sp.set_tuning(batch_blocks_per_solve=bpg)
    try:
        sp.policy_load(omlp.init(211, scale=1.0).astype(np.float32))
        wls = [gg.workload(1, shrink=2), gg.workload(3, shrink=12), gg.workload(2, shrink=10),
               gg.workload(5, shrink=11)]
        graphs, Gs, srcs = [], [], []
        for wl in wls:
            g = wl.graphs[0]
            G = sp.Graph.from_csr(g, reverse=True)
            for j in range(2):
                s = wl.solves[0][1] if j == 0 else (wl.solves[0][1] + g.n // 3) % g.n
                graphs.append(g)
                Gs.append(G)
                srcs.append(s)
        B = sp.Batch(Gs, srcs, sp.IN_OUT | sp.POLICY_LEARNED)
        sp.policy_clear()  # the batch keeps its own copy of the network
        traced = list(range(0, len(Gs), 2))
        for i in traced:
            B.attach_trace(i)
        for rep in range(2):  # a replay of the captured launch gives the same results
            B.launch()
            torch.cuda.synchronize()
            phases = B.phases.cpu().numpy()
            for i, (g, s) in enumerate(zip(graphs, srcs)):
                ref = oracle.dijkstra(g, s)
                assert (sp.as_uint64(B.outs[i]) == ref).all(), f"solve {i}"
                if i in traced:
                    settle, tr = B.trace_of(i)
                    assert len(tr) == phases[i]
                    sched = tr["criterion"].astype(np.uint32)
                    assert set(np.unique(sched)) <= {sp.IN_OUT, sp.IN_SIMPLE | sp.OUT_STATIC}
                    assert ((tr["arm"] & 0x80) != 0).all()
                    sim = oracle.simulate(g, s, sp.IN_OUT, schedule=sched, dist_ref=ref)
                    assert sim.phases == phases[i]
                    assert (settle == sim.settle_phase).all(), f"solve {i}"
        B.close()
    finally:
        sp.policy_clear()
        sp.set_tuning()


def test_policy_requires_a_loaded_network_and_the_fallback_criterion():
    g = gg.workload(1, shrink=4).graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    sp.policy_clear()
    with pytest.raises(sp.SsspError) as e:
        sp.solve(G, 0, sp.IN_OUT | sp.POLICY_LEARNED)
    assert e.value.status == 6
    sp.policy_load(omlp.init(1).astype(np.float32))
    with pytest.raises(sp.SsspError) as e:
        sp.solve(G, 0, sp.SIMPLE | sp.POLICY_LEARNED)
    assert e.value.status == 1


def _time(G, s, crit, reps=5):
    out = torch.empty(G.n, dtype=torch.int64, device="cuda")
    sp.solve(G, s, crit, out=out)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, ph = sp.solve(G, s, crit, out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), ph


def test_trained_policy_gain(capsys):
    """Train on small graphs of every family, evaluate on larger held-out ones.
    The judge is the fastest fixed policy: each of the network's four arms run
    on its own for the whole solve.  In total over the held-out graphs the
    trained network is no slower than the fixed IN+OUT method (2 % allowed for
    timing noise) and within 10 % of choosing the fastest fixed arm per graph
    in hindsight; on some graph it beats IN+OUT by at least 5 %."""
    from paper_1903_12085_gb300 import policy as pol

    w, hist = pol.fit_and_load()
    assert hist[-1][1] < hist[0][1]  # training lowers the loss
    rows = []
    # held out: none of these graphs is among the training graphs (the third
    # has the first workload's shape, drawn with another seed)
    held_out = [gg.workload(3, shrink=4), gg.workload(5, shrink=4),
                gg.Workload("gnm_n16384_m131072_seed2", [gg.gnm(16384, 131072, 0, 1 << 24, gg.SEED_BASE + 101)],
                            [(0, 0)]),
                gg.workload(2, shrink=4)]
    for wl in held_out:
        gi, s = wl.solves[0]
        G = sp.Graph.from_csr(wl.graphs[gi], reverse=True)
        arms = [_time(G, s, crit)[0] for crit in pol.ARMS]
        t_learn, p_learn = _time(G, s, sp.IN_OUT | sp.POLICY_LEARNED)
        rows.append((wl.name, arms, t_learn, p_learn))
    with capsys.disabled():
        print("\npolicy vs fixed arms (held-out graphs, ms): name, IN+OUT sparse/dense, IN-SIMPLE|OUT sparse/dense,"
              " learned (phases), speedup vs IN+OUT, vs fastest arm")
        for name, arms, tl, pl in rows:
            print(f"  {name:24s} " + " ".join(f"{a:9.3f}" for a in arms) +
                  f" {tl:9.3f} ({pl:6d}) {arms[0] / tl:5.2f}x {min(arms) / tl:5.2f}x")
    total_learn = sum(r[2] for r in rows)
    total_in_out = sum(r[1][0] for r in rows)
    total_best = sum(min(r[1]) for r in rows)
    with capsys.disabled():
        print(f"  total: learned {total_learn:.3f} ms, IN+OUT {total_in_out:.3f} ms, "
              f"fastest arm per graph {total_best:.3f} ms")
    assert total_learn <= 1.02 * total_in_out
    assert total_learn <= 1.10 * total_best
    assert max(r[1][0] / r[2] for r in rows) >= 1.05

"""The APPROX(k) criterion of the simulator (approximate IN (full) / OUT-WEAK
minima recomputed every k-th phase, Section 3's closing remark), on CPU.

Pins: with k = 1 the values are exact in every phase, so APPROX must settle
exactly what IN (full) | OUT-WEAK settles; for any k the criterion must be
sound and complete (the simulator checks every settled vertex against
Dijkstra and fails on an empty phase); and on one and the same state its
selection lies between the static criteria's and the full/weak criteria's,
because every value lies between the static minimum and the exact term.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle_pins import random_tiny_graph

STATIC = oracle.IN_STATIC | oracle.OUT_STATIC
FULLWEAK = oracle.IN_FULL | oracle.OUT_WEAK


def _graphs(count, seed, n_max=40):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        g = random_tiny_graph(rng, n_max=n_max, w_max=int(rng.choice([0, 3, 50, 2**20])))
        out.append((g, int(rng.integers(0, g.n))))
    return out


def test_k1_equals_in_full_or_out_weak():
    for g, s in _graphs(300, 11):
        ref = oracle.dijkstra(g, s)
        a = oracle.simulate(g, s, oracle.approx(1), dist_ref=ref, trace=True)
        b = oracle.simulate(g, s, FULLWEAK, dist_ref=ref, trace=True)
        assert a.phases == b.phases
        assert (a.settle_phase == b.settle_phase).all()
        assert (a.trace[:, :4] == b.trace[:, :4]).all()  # |F|, |S'|, minD, minOut


@pytest.mark.parametrize("k", [2, 3, 5, 8, 63])
def test_sound_and_complete(k):
    for g, s in _graphs(200, 100 + k):
        ref = oracle.dijkstra(g, s)
        for crit in [oracle.approx(k), oracle.approx(k) | oracle.DIJK]:
            sim = oracle.simulate(g, s, crit, dist_ref=ref)  # raises if unsound or incomplete
            assert (sim.d == ref).all()


@pytest.mark.parametrize("k", [2, 3, 8])
def test_selection_between_static_and_full_on_the_same_state(k):
    """Phases 1..p run APPROX(k) in all three runs; phase p+1 then runs the
    static criteria, APPROX(k) or IN (full) | OUT-WEAK on the same state."""
    checked = 0
    for g, s in _graphs(120, 200 + k, n_max=60):
        ref = oracle.dijkstra(g, s)
        base = oracle.simulate(g, s, oracle.approx(k), dist_ref=ref)
        for p in range(1, base.phases):
            sets = []
            for last in [STATIC, oracle.approx(k), FULLWEAK]:
                sched = np.array([oracle.approx(k)] * p + [last], np.uint32)
                sim = oracle.simulate(g, s, oracle.approx(k), schedule=sched, dist_ref=ref)
                sets.append(set(np.nonzero(sim.settle_phase == p + 1)[0].tolist()))
            assert sets[0] <= sets[1] <= sets[2], (p, sets)
            checked += 1
    assert checked > 100


def test_phase_counts_order_on_uniform_graphs():
    """Averaged over seeds: IN (full) | OUT-WEAK needs the fewest phases,
    the static criteria the most, APPROX(k) in between and more as k grows."""
    tot = {}
    crits = {"static": STATIC, "a2": oracle.approx(2), "a8": oracle.approx(8), "full": FULLWEAK}
    for k in range(4):
        g = gg.gnm(2048, 10 * 2048, 0, 1 << 24, 0x5EED + k)
        for name, c in crits.items():
            tot[name] = tot.get(name, 0) + oracle.simulate(g, 0, c).phases
    assert tot["full"] <= tot["a2"] <= tot["a8"] <= tot["static"]
    assert tot["full"] < tot["static"]

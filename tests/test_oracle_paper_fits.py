"""The simulator against the paper's own curve fits (CPU).

The paper's simulation section prints, for uniform random graphs with mean
out-degree 10, fits b * n^c of the number of phases and of the sum of |F| for
every criterion (the constant term of the fit dropped), and b * log2(n) for
ORACLE.  On our seeded stand-in (G(n, m), m = 10 n, weights uniform) the
simulator's means must land near those printed curves; a dropped term, a wrong
comparison or a swapped minimum in any criterion moves a count by far more than
the tolerance.  Sizes and samples are small enough for the CPU suite; the full
study (oracle/phase_study.py) fits the exponents themselves.
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

# The paper's fits for uniform graphs (phases; sum of |F|): (b, c), c None for b*log2(n).
PAPER_UNIFORM = {
    "OUT-STATIC": (oracle.OUT_STATIC, (2.48, 0.5), (0.79, 1.50)),
    "IN-STATIC": (oracle.IN_STATIC, (2.28, 0.5), (0.73, 1.50)),
    "IN-STATIC|OUT-STATIC": (oracle.IN_STATIC | oracle.OUT_STATIC, (3.97, 0.34), (1.17, 1.33)),
    "OUT-SIMPLE": (oracle.OUT_SIMPLE, (1.66, 0.5), (0.64, 1.50)),
    "IN-SIMPLE": (oracle.IN_SIMPLE, (1.43, 0.46), (0.39, 1.49)),
    "IN-SIMPLE|OUT-SIMPLE": (oracle.IN_SIMPLE | oracle.OUT_SIMPLE, (3.75, 0.29), (0.95, 1.31)),
    "OUT": (oracle.OUT_FULL, (1.62, 0.48), (0.58, 1.49)),
    "IN": (oracle.IN_FULL, (1.47, 0.43), (0.35, 1.49)),
    "IN|OUT": (oracle.IN_FULL | oracle.OUT_FULL, (4.60, 0.26), (0.96, 1.29)),
    "ORACLE": (oracle.ORACLE, (1.69, None), (2.49, 1.05)),
}


@pytest.fixture(scope="module")
def means():
    n, samples = 1 << 14, 3
    acc = {name: [0.0, 0.0] for name in PAPER_UNIFORM}
    for k in range(samples):
        g = gg.gnm(n, 10 * n, 0, 1 << 24, 0x1903120850 + 777 + k)
        d = oracle.dijkstra(g, 0)
        for name, (mask, _, _) in PAPER_UNIFORM.items():
            sim = oracle.simulate(g, 0, mask, dist_ref=d)
            acc[name][0] += sim.phases / samples
            acc[name][1] += sim.sum_f / samples
    return n, acc


@pytest.mark.parametrize("name", list(PAPER_UNIFORM))
def test_phases_follow_the_papers_fit(means, name):
    n, acc = means
    b, c = PAPER_UNIFORM[name][1]
    ref = b * (math.log2(n) if c is None else n ** c)
    assert 0.85 <= acc[name][0] / ref <= 1.15, (acc[name][0], ref)


@pytest.mark.parametrize("name", list(PAPER_UNIFORM))
def test_sum_f_follows_the_papers_fit(means, name):
    n, acc = means
    b, c = PAPER_UNIFORM[name][2]
    ref = b * n ** c
    assert 0.8 <= acc[name][1] / ref <= 1.2, (acc[name][1], ref)


def test_strength_order_on_uniform_graphs(means):
    """The orderings the paper reports: each disjunction needs fewer phases than
    its parts, the simple and full variants fewer than the static ones, and
    ORACLE the fewest."""
    _, acc = means
    ph = {k: v[0] for k, v in acc.items()}
    assert ph["IN-STATIC|OUT-STATIC"] < min(ph["IN-STATIC"], ph["OUT-STATIC"])
    assert ph["IN-SIMPLE|OUT-SIMPLE"] < ph["IN-STATIC|OUT-STATIC"]
    assert ph["IN|OUT"] < ph["IN-SIMPLE|OUT-SIMPLE"]
    assert ph["ORACLE"] < ph["IN|OUT"]
    assert np.isfinite(list(ph.values())).all()

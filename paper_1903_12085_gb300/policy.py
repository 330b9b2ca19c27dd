"""Training of the per-phase policy network on traces the solver itself produces.

For every training graph and every arm (IN-STATIC|OUT-STATIC or
IN-SIMPLE|OUT-STATIC, sparse queue or dense scan), one traced solve records each
phase's fringe size, settled vertices, relaxed edges and device time.  Each phase
becomes a sample: the features of its start state (sssp_policy_features) ->
log2(phase time / settled vertices) for the arm it ran with.  The network is fit
with the library's FP32 backward and Adam kernels (masked mean squared error on
the arm taken) and loaded with sssp_policy_load; a solve with
SSSP_POLICY_LEARNED then runs every phase with the arm of lowest predicted cost
per settled vertex.
"""
from __future__ import annotations

import numpy as np

from . import (FRONTIER_DENSE, IN_SIMPLE, IN_STATIC, OUT_STATIC, POLICY_WEIGHTS, Graph, mlp_adam, mlp_backward,
               policy_features, policy_load, solve_trace)

ARMS = [IN_STATIC | OUT_STATIC, IN_STATIC | OUT_STATIC | FRONTIER_DENSE,
        IN_SIMPLE | OUT_STATIC, IN_SIMPLE | OUT_STATIC | FRONTIER_DENSE]


def phase_samples(trace, n: int, m: int, arm: int):
    """Features, targets and arm labels of the phases of one traced solve."""
    X, T, A = [], [], []
    prev_e = prev_s = prev_f = 0
    for k, r in enumerate(trace, start=1):
        X.append(policy_features(r["frontier"], n, m, k, prev_e, prev_s, prev_f))
        dt = max(int(r["t_end_ns"]) - int(r["t_start_ns"]), 32)
        T.append(np.log2(dt / max(int(r["settled"]), 1)))
        A.append(arm)
        prev_e, prev_s, prev_f = int(r["deg_settled"]), int(r["settled"]), int(r["frontier"])
    return X, T, A


def collect(cases, arms=None, repeats: int = 3):
    """cases: list of (Graph built with reverse=True, source).  Runs every arm
    `repeats` times (the first run of each warms up) and returns X [N,8]
    float32, T [N] float32, A [N] uint32."""
    arms = list(range(len(ARMS))) if arms is None else arms
    X, T, A = [], [], []
    for G, s in cases:
        for a in arms:
            for rep in range(repeats):
                _, st, _, tr = solve_trace(G, s, ARMS[a], trace_cap=1 << 20, settle=False)
                if rep == 0 and repeats > 1:
                    continue
                x, t, lab = phase_samples(tr, G.n, G.m, a)
                X += x
                T += t
                A += lab
    return np.asarray(X, np.float32), np.asarray(T, np.float32), np.asarray(A, np.uint32)


def init_weights(seed: int = 0, arm_means=None) -> np.ndarray:
    """He-style uniform hidden layers, a near-zero output layer, and output
    biases at the mean target of each arm, so training starts at the per-arm
    mean cost."""
    rng = np.random.default_rng(seed)
    lim1, lim2 = np.sqrt(6.0 / 8), np.sqrt(6.0 / 32)
    b3 = np.zeros(4) if arm_means is None else np.asarray(arm_means, dtype=np.float64)
    parts = [rng.uniform(-lim1, lim1, 8 * 32), np.full(32, 0.01), rng.uniform(-lim2, lim2, 32 * 32),
             np.full(32, 0.01), rng.uniform(-0.01, 0.01, 32 * 4), b3]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == POLICY_WEIGHTS
    return w


def train(X, T, A, epochs: int = 2000, lr: float = 1e-2, seed: int = 0, log_every: int = 0):
    """Full-batch Adam on the GPU with the library's kernels (the learning
    rate decays linearly to lr/10).  Returns the weights (numpy float32) and
    the loss history [(step, loss)]."""
    import torch

    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(T)).to(dev)
    a = torch.from_numpy(np.ascontiguousarray(A).view(np.int32)).to(dev)
    means = [float(np.mean(T[A == k])) if np.any(A == k) else float(np.mean(T)) for k in range(4)]
    w = torch.from_numpy(init_weights(seed, means)).to(dev)
    m1 = torch.zeros_like(w)
    m2 = torch.zeros_like(w)
    grad = torch.empty_like(w)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    hist = []
    for step in range(1, epochs + 1):
        mlp_backward(w, x, t, a, grad=grad, loss=loss)
        mlp_adam(w, grad, m1, m2, lr * (1.0 - 0.9 * (step - 1) / max(epochs - 1, 1)), step)
        if log_every and (step % log_every == 0 or step == 1):
            hist.append((step, float(loss.item())))
    torch.cuda.synchronize()
    return w.cpu().numpy(), hist


def training_cases(shrink_base: int = 0):
    """Seeded training graphs of every family, none of them a benchmark or
    held-out test graph: uniform G(n,m) from 2^13 to 2^22 vertices (the
    2^14-vertex one drawn with its own seed, not the benchmark's), R-MAT from
    scale 12 to 20 and grids (sources from their own recipes)."""
    import graphgen as gg

    g14 = gg.gnm(16384, 131072, 0, 1 << 24, gg.SEED_BASE + 201)
    wls = [gg.Workload(g14.name, [g14], [(0, 0)]), gg.workload(1, shrink=1), gg.workload(3, shrink=2 + shrink_base),
           gg.workload(5, shrink=2 + shrink_base), gg.workload(3, shrink=8 + shrink_base),
           gg.workload(3, shrink=10 + shrink_base), gg.workload(5, shrink=5 + shrink_base),
           gg.workload(5, shrink=6 + shrink_base),
           gg.workload(5, shrink=8 + shrink_base), gg.workload(5, shrink=10 + shrink_base),
           gg.workload(2, shrink=6 + shrink_base), gg.workload(2, shrink=8 + shrink_base)]
    cases = []
    for wl in wls:
        gi, s = wl.solves[0]
        cases.append((Graph.from_csr(wl.graphs[gi], reverse=True), s))
    return cases


def fit_and_load(cases=None, epochs: int = 2000, lr: float = 1e-2, seed: int = 0):
    """Collect traces, train, load the network; returns (weights, loss history)."""
    cases = training_cases() if cases is None else cases
    X, T, A = collect(cases)
    w, hist = train(X, T, A, epochs=epochs, lr=lr, seed=seed, log_every=100)
    policy_load(w)
    return w, hist

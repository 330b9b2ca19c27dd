"""Out-of-memory injection on the host: a cap on the library's device memory
(sssp_set_device_memory_limit) makes an allocation fail at every point of
graph creation, of a solve's set-up, of a traced solve's temporaries, of batch
creation and of policy loading.  Every failing call must return
SSSP_ERR_OUT_OF_MEMORY, free everything it took (the library's count of live
device bytes returns to where it was) and leave the library usable.  No GPU
fault is involved: the refusal happens before cudaMalloc is called."""
import numpy as np
import pytest

import graphgen as gg
import oracle

sp = pytest.importorskip("paper_1903_12085_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    sp.set_device_memory_limit(0)
    yield
    sp.set_device_memory_limit(0)


def _caps(base, need, points=48):
    """Caps from `base` (nothing more may be taken) to just below base + need,
    evenly spread, so that every allocation of the call is refused by some of
    them."""
    caps = sorted({base + (need * i) // points for i in range(points)} | {base + need - 1})
    # a cap of 0 means "no cap": with nothing held yet, 1 byte stands for it
    return [max(c, 1) for c in caps if base <= c < base + need]


def _expect_oom(call, base):
    with pytest.raises(sp.SsspError) as e:
        call()
    assert e.value.status == 2, e.value
    assert sp.device_memory_in_use() == base, "a failing call left device memory allocated"


def test_graph_create_out_of_memory_frees_everything():
    g = gg.workload(3, shrink=10).graphs[0]  # R-MAT rows long enough for merge passes
    base = sp.device_memory_in_use()
    G = sp.Graph.from_csr(g, reverse=True)
    torch.cuda.synchronize()
    need = sp.device_memory_in_use() - base
    G.close()
    assert need > 0 and sp.device_memory_in_use() == base
    for cap in _caps(base, need):
        sp.set_device_memory_limit(cap)
        try:
            _expect_oom(lambda: sp.Graph.from_csr(g, reverse=True), base)
        finally:
            sp.set_device_memory_limit(0)
    # device inputs (validation temporaries) as well
    ro = torch.from_numpy(g.row_off.view(np.int64)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    w = torch.from_numpy(g.w.view(np.int32)).cuda()
    for cap in _caps(base, need, points=16):
        sp.set_device_memory_limit(cap)
        try:
            _expect_oom(lambda: sp.Graph(g.n, ro, col, w, reverse=True), base)
        finally:
            sp.set_device_memory_limit(0)
    G = sp.Graph.from_csr(g, reverse=True)  # usable afterwards
    s = int(g.outdeg().argmax())
    d, _ = sp.solve(G, s, sp.SIMPLE)
    assert (sp.as_uint64(d) == oracle.dijkstra(g, s)).all()
    G.close()


def test_first_solve_and_traced_solve_out_of_memory():
    g = gg.workload(1, shrink=2).graphs[0]
    G = sp.Graph.from_csr(g, reverse=True)
    out = torch.empty(g.n, dtype=torch.int64, device="cuda")
    base = sp.device_memory_in_use()
    sp.solve(G, 0, sp.IN_OUT, out=out)  # allocates the handle's workspace
    need = sp.device_memory_in_use() - base
    G.close()
    G = sp.Graph.from_csr(g, reverse=True)
    base = sp.device_memory_in_use()
    for cap in _caps(base, need):
        sp.set_device_memory_limit(cap)
        try:
            _expect_oom(lambda: sp.solve(G, 0, sp.IN_OUT, out=out), base)
        finally:
            sp.set_device_memory_limit(0)
    ref = oracle.dijkstra(g, 0)
    d, ph = sp.solve(G, 0, sp.IN_OUT, out=out)
    assert (sp.as_uint64(d) == ref).all()
    # a traced solve with host outputs takes two temporaries on top of the workspace
    base = sp.device_memory_in_use()
    for extra in (0, g.n * 4 - 1, g.n * 4 + 64 * (1 << 12) - 1):  # the settle buffer, then the trace buffer
        sp.set_device_memory_limit(base + extra)
        try:
            _expect_oom(lambda: sp.solve_trace(G, 0, sp.IN_OUT, out=out, trace_cap=1 << 12), base)
        finally:
            sp.set_device_memory_limit(0)
    _, st, settle, tr = sp.solve_trace(G, 0, sp.IN_OUT, out=out, trace_cap=1 << 12)
    sim = oracle.simulate(g, 0, sp.IN_OUT, dist_ref=ref)
    assert st["phases"] == sim.phases == ph and (settle == sim.settle_phase).all()
    assert sp.device_memory_in_use() == base
    G.close()


def test_batch_create_out_of_memory_frees_everything():
    wl = gg.workload(4, shrink=5)
    Gs = [sp.Graph.from_csr(g) for g in wl.graphs]
    graphs = [Gs[i] for i, _ in wl.solves]
    sources = [s for _, s in wl.solves]
    outs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for g in graphs]
    base = sp.device_memory_in_use()
    B = sp.Batch(graphs, sources, sp.IN_OUT, outs=outs)
    need = sp.device_memory_in_use() - base
    B.close()
    assert sp.device_memory_in_use() == base
    for cap in _caps(base, need, points=24):
        sp.set_device_memory_limit(cap)
        try:
            _expect_oom(lambda: sp.Batch(graphs, sources, sp.IN_OUT, outs=outs), base)
            _expect_oom(lambda: sp.solve_batch(graphs, sources, sp.IN_OUT, outs=outs), base)
        finally:
            sp.set_device_memory_limit(0)
    res, ph = sp.solve_batch(graphs, sources, sp.IN_OUT, outs=outs)
    for k, (i, s) in enumerate(wl.solves):
        assert (sp.as_uint64(res[k]) == oracle.dijkstra(wl.graphs[i], s)).all()
    for G in Gs:
        G.close()


def test_policy_load_out_of_memory():
    from oracle import mlp as omlp
    sp.policy_clear()
    base = sp.device_memory_in_use()
    sp.set_device_memory_limit(max(base, 1))  # (a cap of 0 means "no cap")
    try:
        _expect_oom(lambda: sp.policy_load(omlp.init(1).astype(np.float32)), base)
    finally:
        sp.set_device_memory_limit(0)
    sp.policy_load(omlp.init(1).astype(np.float32))
    assert sp.device_memory_in_use() == base + 4 * sp.POLICY_WEIGHTS
    sp.policy_clear()
    assert sp.device_memory_in_use() == base

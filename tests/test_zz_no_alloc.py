"""sssp_solve_noalloc, the entry point for callers that cannot allocate
device memory at solve time (their allocator owns the device, or their request
path cannot take cudaMalloc's device synchronisation).  Its scratch lives in a
fixed file-scope device array, so it is checked here against the regular
sssp_solve on the same graphs, bit for bit, on two calls in a row (the second
call reuses whatever the first left in the array), and against the CPU oracle
(Dijkstra's distances, the simulator's phase count).  That it allocates nothing
is checked twice: under a device-memory cap with no headroom left for the
library, and by the device's free memory, unchanged across a call.  This file
is collected last on purpose."""
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


def _device_csr(g):
    ro = torch.from_numpy(g.row_off.view(np.int64)).cuda()
    pairs = np.empty((g.m, 2), np.uint32)
    pairs[:, 0] = g.col
    pairs[:, 1] = g.w
    edges = torch.from_numpy(pairs.reshape(-1).view(np.int32)).cuda()
    return ro, edges


CRITS = [sp.IN_OUT, sp.IN_STATIC, sp.OUT_STATIC, sp.IN_OUT | sp.FRONTIER_DENSE, sp.IN_OUT | sp.FRONTIER_AUTO,
         sp.DIJK, sp.IN_STATIC | sp.DIJK]


@pytest.mark.parametrize("crit", CRITS, ids=["in_out", "in", "out", "dense", "auto", "dijk", "in_dijk"])
def test_noalloc_matches_regular_solve_and_oracle_twice(crit):
    cases = [(gg.workload(1).graphs[0], [0, 77]), (gg.workload(2, shrink=4).graphs[0], [0, 5])]
    if crit & sp.DIJK:  # one vertex per phase: the smaller graphs keep the phase count modest
        cases = [(gg.workload(1, shrink=2).graphs[0], [0, 77]), (gg.workload(2, shrink=8).graphs[0], [0, 5])]
    for g, sources in cases:
        G = sp.Graph.from_csr(g)
        ro, edges = _device_csr(g)
        out = torch.empty(g.n, dtype=torch.int64, device="cuda")
        for s in sources:  # two calls in a row, different sources
            ref, ref_phases = sp.solve(G, s, crit)
            out.fill_(-1)
            d, phases = sp.solve_noalloc(g.n, ro, edges, s, crit, out=out)
            torch.cuda.synchronize()
            assert phases == ref_phases
            assert torch.equal(d, ref)
            dist = oracle.dijkstra(g, s)
            assert (sp.as_uint64(d) == dist).all()
            assert phases == oracle.simulate(g, s, crit & 0xFFFF, dist_ref=dist).phases
        G.close()


def test_noalloc_allocates_nothing():
    g = gg.workload(1).graphs[0]
    ro, edges = _device_csr(g)
    out = torch.empty(g.n, dtype=torch.int64, device="cuda")
    ref = oracle.dijkstra(g, 0)
    sp.solve_noalloc(g.n, ro, edges, 0, sp.IN_OUT, out=out)  # first call on the device: set-up
    torch.cuda.synchronize()
    sp.set_device_memory_limit(max(sp.device_memory_in_use(), 1))  # no headroom for the library
    try:
        free0, _ = torch.cuda.mem_get_info()
        for s in (0, 0):
            out.fill_(-1)
            d, _ = sp.solve_noalloc(g.n, ro, edges, s, sp.IN_OUT, out=out)
            torch.cuda.synchronize()
            assert (sp.as_uint64(d) == ref).all()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
    finally:
        sp.set_device_memory_limit(0)


def test_noalloc_rejects_sizes_beyond_its_maximum_and_bad_input():
    n = sp.NOALLOC_MAX_VERTICES + 1
    ro = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    edges = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(sp.SsspError) as e:
        sp.solve_noalloc(n, ro, edges[:0], 0, sp.IN_OUT, out=out)
    assert e.value.status == 1
    with pytest.raises(sp.SsspError) as e:
        sp.solve_noalloc(4, ro[:5], edges[:0], 0, sp.SIMPLE, out=out[:4])
    assert e.value.status == 6
    # a small in-bounds CSR whose edge points past the last vertex
    bad_ro = torch.tensor([0, 1, 1, 1], dtype=torch.int64, device="cuda")
    bad_edges = torch.tensor([7, 3], dtype=torch.int32, device="cuda")
    with pytest.raises(sp.SsspError) as e:
        sp.solve_noalloc(3, bad_ro, bad_edges, 0, sp.IN_OUT, out=out[:3])
    assert e.value.status == 1
    # an edge array sliced one 4-byte word off its 8-byte boundary
    with pytest.raises(sp.SsspError) as e:
        sp.solve_noalloc(3, bad_ro, edges[1:3], 0, sp.IN_OUT, out=out[:3])
    assert e.value.status == 1 and "aligned" in str(e.value)
    # the array is still usable after the rejected calls
    g = gg.workload(1, shrink=3).graphs[0]
    gro, gedges = _device_csr(g)
    d, _ = sp.solve_noalloc(g.n, gro, gedges, 0, sp.IN_OUT)
    assert (sp.as_uint64(d) == oracle.dijkstra(g, 0)).all()

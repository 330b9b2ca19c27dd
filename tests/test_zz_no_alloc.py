"""sssp_solve_noalloc, the entry point for callers that cannot allocate
device memory at solve time (their allocator owns the device, or their request
path cannot take cudaMalloc's device synchronisation).  Its scratch lives in a
fixed file-scope device array, so it is checked here against the regular
sssp_solve on the same graphs, bit for bit, on two calls in a row (the second
call reuses whatever the first left in the array).  This file is collected
last on purpose."""
import numpy as np
import pytest

import graphgen as gg

sp = pytest.importorskip("paper_1903_12085_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _device_csr(g):
    ro = torch.from_numpy(g.row_off.view(np.int64)).cuda()
    pairs = np.empty((g.m, 2), np.uint32)
    pairs[:, 0] = g.col
    pairs[:, 1] = g.w
    edges = torch.from_numpy(pairs.reshape(-1).view(np.int32)).cuda()
    return ro, edges


@pytest.mark.parametrize("crit", [sp.IN_OUT, sp.IN_STATIC, sp.OUT_STATIC, sp.IN_OUT | sp.FRONTIER_DENSE])
def test_noalloc_matches_regular_solve_twice(crit):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    cases = [(gg.workload(1).graphs[0], [0, 77]), (gg.workload(2, shrink=4).graphs[0], [0, 5])]
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
        G.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = sp.NOALLOC_MAX_VERTICES + 1
    ro = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    edges = torch.zeros(2, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    with pytest.raises(sp.SsspError) as e:
        sp.solve_noalloc(n, ro, edges[:0], 0, sp.IN_OUT, out=out)
    assert e.value.status == 1
    with pytest.raises(sp.SsspError) as e:
        sp.solve_noalloc(4, ro[:5], edges[:0], 0, sp.SIMPLE, out=out[:4])
    assert e.value.status == 6

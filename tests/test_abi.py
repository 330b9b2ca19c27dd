"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: only symbols are looked up, nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sssp_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sssp_graph_create", "sssp_graph_destroy", "sssp_solve", "sssp_solve_batch",
                     "sssp_solve_trace", "sssp_last_error"]:
        assert required in names


def test_library_exports_every_declared_function():
    import paper_1903_12085_gb300 as sp
    if not os.path.exists(sp.LIB_PATH):
        from paper_1903_12085_gb300 import _build
        _build.build()
    lib = ctypes.CDLL(sp.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string_without_gpu():
    import paper_1903_12085_gb300 as sp
    assert "sm_103a" in sp.version()


def test_product_path_does_not_touch_oracle():
    """The package never imports, links or loads the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_1903_12085_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            for bad in ("import oracle", "from oracle", "liboracle", "oracle.c"):
                assert bad not in text, (path, bad)


def test_binding_rejects_short_distance_buffers():
    """The binding checks a caller's distance buffer before passing its address
    (the C ABI cannot see the size): too short or strided buffers raise."""
    import numpy as np

    import paper_1903_12085_gb300 as sp

    ok = np.zeros(10, np.uint64)
    assert sp._dist_buffer(10, ok) is ok
    assert sp._dist_buffer(5, ok) is ok
    with pytest.raises(ValueError):
        sp._dist_buffer(11, ok)
    with pytest.raises(ValueError):
        sp._dist_buffer(5, np.zeros(20, np.uint64)[::2])
    with pytest.raises(ValueError):
        sp._dist_buffer(10, np.zeros(10, np.uint32))
    assert sp.approx(4) == sp.APPROX | (4 << 10)
    with pytest.raises(ValueError):
        sp.approx(0)


def test_binding_checks_batch_lengths_before_any_call():
    import types

    import numpy as np

    import paper_1903_12085_gb300 as sp

    g = types.SimpleNamespace(n=3)
    with pytest.raises(ValueError):
        sp.solve_batch([g], [0, 1], outs=[np.zeros(3, np.uint64)])
    with pytest.raises(ValueError):
        sp.solve_batch([g, g], [0, 1], outs=[np.zeros(3, np.uint64), np.zeros(2, np.uint64)])


def test_policy_features_follow_the_documented_formula():
    """sssp_policy_features (a host function; the engine evaluates the same
    code per phase) against the eight features listed in include/sssp.h."""
    import numpy as np

    import paper_1903_12085_gb300 as sp

    cases = [(1, 16384, 131072, 1, 0, 0, 0), (5000, 1 << 22, 1 << 26, 37, 81234, 4021, 6123),
             (1 << 20, 1 << 24, 1 << 28, 1085, 3 << 20, 9 << 10, 1 << 21), (0, 7, 0, 2, 0, 0, 0)]
    for F, n, m, k, e, s, f in cases:
        want = np.array([np.log2(1 + F) / 24, F / n, np.log2(1 + e) / 24, np.log2(1 + s) / 24,
                         np.log2(1 + k) / 16, np.log2(n) / 32, (m / n) / 32, s / (1 + f)])
        got = sp.policy_features(F, n, m, k, e, s, f).astype(np.float64)
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6), (got, want)
    with pytest.raises(sp.SsspError):
        sp.policy_features(1, 0, 0, 1, 0, 0, 0)  # n = 0 is rejected


def test_noalloc_rejects_misaligned_buffers_before_any_cuda_call():
    """sssp_solve_noalloc reads its CSR and distance buffers as 8-byte words:
    a buffer off an 8-byte boundary is refused with SSSP_ERR_INVALID_ARG by a
    host-side check that runs before any CUDA call (so this needs no GPU)."""
    import ctypes

    import paper_1903_12085_gb300 as sp

    L = sp.lib()
    p = ctypes.c_void_p
    for ro, ed, out in [(0x10004, 0x20000, 0x30000), (0x10000, 0x20004, 0x30000), (0x10000, 0x20000, 0x30002)]:
        st = L.sssp_solve_noalloc(16, 8, p(ro), p(ed), 0, sp.IN_OUT, p(out), None, None)
        assert st == 1
        assert b"8-byte aligned" in L.sssp_last_error()


def test_noalloc_binding_checks_its_tensors():
    """The binding refuses CSR inputs the C ABI cannot check: host arrays,
    wrong element sizes, strided views, too few offsets, an odd word count."""
    import numpy as np
    import torch

    import paper_1903_12085_gb300 as sp

    with pytest.raises(ValueError, match="CUDA tensor"):
        sp._noalloc_inputs(4, np.zeros(5, np.int64), np.zeros(2, np.int32))
    with pytest.raises(ValueError, match="CUDA tensor"):
        sp._noalloc_inputs(4, torch.zeros(5, dtype=torch.int64), torch.zeros(2, dtype=torch.int32))


def test_device_memory_cap_refuses_before_cudamalloc():
    """With a cap below the first allocation, sssp_graph_create fails with
    SSSP_ERR_OUT_OF_MEMORY before calling cudaMalloc (so this runs without a
    GPU) and leaves nothing allocated; lifting the cap restores the default."""
    import numpy as np

    import paper_1903_12085_gb300 as sp

    import ctypes

    base = sp.device_memory_in_use()
    sp.set_device_memory_limit(base + 1)
    try:
        ro, col, w = np.array([0, 1, 2, 2], np.uint64), np.array([1, 2], np.uint32), np.array([5, 6], np.uint32)
        h = ctypes.c_void_p()
        st = sp.lib().sssp_graph_create(3, 2, sp._ptr(ro), sp._ptr(col), sp._ptr(w), 0, sp.GRAPH_REVERSE, None,
                                        ctypes.byref(h))
        assert st == 2 and b"limit" in sp.lib().sssp_last_error()
        assert h.value is None
        assert sp.device_memory_in_use() == base
    finally:
        sp.set_device_memory_limit(0)


def test_graph_create_checks_host_offset_ends_before_any_cuda_call():
    """Host CSR: row_offsets[0] != 0, row_offsets[n] != m, and the decreasing
    offsets of an edgeless graph are refused with SSSP_ERR_INVALID_ARG before
    any allocation or CUDA call (so this needs no GPU); the per-edge checks
    run on the device after the copy."""
    import ctypes

    import numpy as np

    import paper_1903_12085_gb300 as sp

    L = sp.lib()
    col, w = np.array([1, 2], np.uint32), np.array([5, 6], np.uint32)
    cases = [(3, 2, np.array([1, 1, 2, 2], np.uint64), "row_offsets[0]"),
             (3, 2, np.array([0, 1, 2, 3], np.uint64), "row_offsets[n]"),
             (2, 0, np.array([0, 1, 0], np.uint64), "decrease")]
    base = sp.device_memory_in_use()
    for n, m, ro, msg in cases:
        h = ctypes.c_void_p()
        st = L.sssp_graph_create(n, m, sp._ptr(ro), sp._ptr(col), sp._ptr(w), 0, 0, None, ctypes.byref(h))
        assert st == 1, msg
        assert msg.encode() in L.sssp_last_error()
        assert h.value is None
    assert sp.device_memory_in_use() == base

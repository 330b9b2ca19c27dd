"""Python binding of the GB300 phase-parallel Dijkstra library (libsssp_gb300.so).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels behind the C ABI of ``include/sssp.h``.  PyTorch provides device
memory and streams.  There is no CPU fallback: if the shared library is not
built, every call raises.

Names follow the C ABI::

    g = Graph(n, row_off, col, w, reverse=True)      # sssp_graph_create
    dist, phases = solve(g, source, IN_STATIC | OUT_STATIC)   # sssp_solve
    dist, stats, settle, trace = solve_trace(g, source, crit)  # sssp_solve_trace
    outs, phases = solve_batch([g, ...], [s, ...], crit)      # sssp_solve_batch
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsssp_gb300.so")

# criterion mask bits and options (include/sssp.h)
IN_STATIC = 1 << 0
OUT_STATIC = 1 << 1
IN_SIMPLE = 1 << 2
OUT_SIMPLE = 1 << 3
IN_FULL = 1 << 4
OUT_WEAK = 1 << 5
DIJK = 1 << 6
APPROX = 1 << 9
APPROX_K_SHIFT = 10
POLICY_LEARNED = 1 << 16
FRONTIER_DENSE = 1 << 17
FRONTIER_AUTO = 1 << 18
GRAPH_REVERSE = 1 << 0
IN_OUT = IN_STATIC | OUT_STATIC
SIMPLE = IN_SIMPLE | OUT_SIMPLE


def approx(k: int) -> int:
    """SSSP_APPROX_K(k): approximate IN (full) / OUT-WEAK minima recomputed in
    every k-th phase (1 <= k <= 63)."""
    if not 1 <= k <= 63:
        raise ValueError("k must be in 1..63")
    return APPROX | (k << APPROX_K_SHIFT)

STATUS = {0: "SSSP_OK", 1: "SSSP_ERR_INVALID_ARG", 2: "SSSP_ERR_OUT_OF_MEMORY", 3: "SSSP_ERR_CUDA",
          4: "SSSP_ERR_TIMEOUT", 5: "SSSP_ERR_INTERNAL", 6: "SSSP_ERR_UNSUPPORTED"}

PHASE_RECORD = np.dtype([("frontier", "<u4"), ("settled", "<u4"), ("min_d", "<u8"), ("min_out", "<u8"),
                         ("deg_settled", "<u8"), ("criterion", "<u4"), ("arm", "<u4"),
                         ("t_start_ns", "<u8"), ("t_end_ns", "<u8"), ("queued", "<u4"),
                         ("select_ns", "<u4")])
assert PHASE_RECORD.itemsize == 64


class SsspError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [("phases", ctypes.c_uint64), ("sum_frontier", ctypes.c_uint64),
                ("settled", ctypes.c_uint64), ("edges_relaxed", ctypes.c_uint64)]


_lib = None


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        u32, u64, p, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        sig = {
            "sssp_graph_create": [u32, u64, p, p, p, i32, u32, p, ctypes.POINTER(p)],
            "sssp_graph_info": [p, p, p, p],
            "sssp_graph_device_arrays": [p, p, p, p, p, p, p],
            "sssp_solve": [p, u32, u32, p, p, p],
            "sssp_solve_trace": [p, u32, u32, p, p, p, p, u64, p],
            "sssp_solve_batch": [p, p, u32, u32, p, p, p],
            "sssp_batch_create": [p, p, u32, u32, p, p, p, ctypes.POINTER(p)],
            "sssp_batch_launch": [p, p],
            "sssp_batch_trace": [p, u32, p, u64, p, p],
            "sssp_set_wait_limit_ns": [u64],
            "sssp_set_l2_fetch_granularity": [u32],
            "sssp_set_device_memory_limit": [u64],
            "sssp_device_memory_in_use": [p],
            "sssp_selftest_wait": [u64],
            "sssp_solve_noalloc": [u32, u64, p, p, u32, u32, p, p, p],
            "sssp_batch_autotune": [p, p, p, p],
            "sssp_set_tuning": [p],
            "sssp_get_tuning": [p],
            "sssp_policy_load": [p, ctypes.c_size_t],
            "sssp_policy_clear": [],
            "sssp_policy_features": [u64, u64, u64, u64, u64, u64, u64, p],
            "sssp_mlp_forward": [p, p, u32, p, p],
            "sssp_mlp_backward": [p, p, p, p, u32, p, p, p],
            "sssp_mlp_adam": [p, p, p, p, u32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              u32, p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sssp_graph_destroy.argtypes = [p]
        L.sssp_graph_destroy.restype = None
        L.sssp_batch_destroy.argtypes = [p]
        L.sssp_batch_destroy.restype = None
        L.sssp_last_error.restype = ctypes.c_char_p
        L.sssp_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise SsspError(status, lib().sssp_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(x):
    """Data pointer of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def version() -> str:
    return lib().sssp_version().decode()


def set_wait_limit_ns(ns: int):
    _check(lib().sssp_set_wait_limit_ns(int(ns)))


def set_l2_fetch_granularity(nbytes: int):
    """sssp_set_l2_fetch_granularity: 32, 64 or 128 bytes per L2 fetch on a
    DRAM miss, for this process's CUDA context on the current device."""
    _check(lib().sssp_set_l2_fetch_granularity(int(nbytes)))


def set_device_memory_limit(nbytes: int):
    """sssp_set_device_memory_limit: cap on the device memory the library
    allocates (0 = no cap)."""
    _check(lib().sssp_set_device_memory_limit(int(nbytes)))


def device_memory_in_use() -> int:
    """sssp_device_memory_in_use: bytes of device memory the library holds."""
    b = ctypes.c_uint64()
    _check(lib().sssp_device_memory_in_use(ctypes.byref(b)))
    return b.value


def selftest_wait(limit_ns: int) -> int:
    """sssp_selftest_wait: status of a bounded wait on a word nothing writes
    (SSSP_ERR_TIMEOUT = 4 is the expected result)."""
    return int(lib().sssp_selftest_wait(int(limit_ns)))


class Tuning(ctypes.Structure):
    _fields_ = [("solo_max_frontier", ctypes.c_uint32), ("batch_blocks_per_solve", ctypes.c_uint32),
                ("grid_blocks", ctypes.c_uint32), ("solo_max_edges", ctypes.c_uint32),
                ("nearfar_min_frontier", ctypes.c_uint32), ("nearfar_target", ctypes.c_uint32),
                ("nearfar_min_share", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def set_tuning(**fields):
    """sssp_set_tuning; fields not given keep their current value (names as in
    sssp_tuning: solo_max_frontier, batch_blocks_per_solve, grid_blocks,
    solo_max_edges, nearfar_min_frontier, nearfar_target, nearfar_min_share).  set_tuning() with
    no argument restores the defaults."""
    if not fields:
        _check(lib().sssp_set_tuning(None))
        return
    t = get_tuning()
    names = {f for f, _ in Tuning._fields_ if f != "reserved"}
    for k, v in fields.items():
        if k not in names:
            raise TypeError(f"unknown tuning field {k!r}")
        if v is not None:
            setattr(t, k, int(v))
    _check(lib().sssp_set_tuning(ctypes.byref(t)))


def get_tuning() -> Tuning:
    t = Tuning()
    _check(lib().sssp_get_tuning(ctypes.byref(t)))
    return t


class Graph:
    """A preprocessed graph on the current CUDA device (sssp_graph_create).

    ``row_off``/``col``/``w`` are either numpy arrays (host) or CUDA tensors
    (device; uint64/int64 offsets, uint32/int32 targets and costs)."""

    def __init__(self, n: int, row_off, col, w, reverse: bool = False, stream=None):
        on_dev = not isinstance(row_off, np.ndarray)
        if not on_dev:
            row_off = np.ascontiguousarray(row_off, dtype=np.uint64)
            col = np.ascontiguousarray(col, dtype=np.uint32)
            w = np.ascontiguousarray(w, dtype=np.uint32)
            m = int(col.shape[0])
        else:
            m = int(col.numel())
        self.n, self.m = int(n), m
        self._keep = (row_off, col, w)
        h = ctypes.c_void_p()
        _check(lib().sssp_graph_create(self.n, m, _ptr(row_off), _ptr(col), _ptr(w), int(on_dev),
                                       GRAPH_REVERSE if reverse else 0, _stream_ptr(stream), ctypes.byref(h)))
        self._keep = None
        self.handle = h
        self.reverse = reverse

    @classmethod
    def from_csr(cls, g, reverse: bool = False, stream=None) -> "Graph":
        """From any object with n, row_off, col, w (e.g. graphgen.Graph)."""
        return cls(g.n, g.row_off, g.col, g.w, reverse=reverse, stream=stream)

    def device_arrays(self):
        """Device addresses (ints) of the preprocessed arrays held by the
        handle: row_off, edges, out_min, in_min, rrow_off, redges (the last
        two 0 without the reverse CSR); valid until close()."""
        ptrs = [ctypes.c_void_p() for _ in range(6)]
        _check(lib().sssp_graph_device_arrays(self.handle, *[ctypes.byref(x) for x in ptrs]))
        return {name: p.value for name, p in zip(["row_off", "edges", "out_min", "in_min", "rrow_off", "redges"], ptrs)}

    def close(self):
        if getattr(self, "handle", None):
            lib().sssp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dist_buffer(n, out):
    """``out`` if it holds at least n 8-byte words, a new CUDA int64 tensor of
    n if it is None."""
    if out is None:
        torch = _torch()
        return torch.empty(n, dtype=torch.int64, device="cuda")
    if isinstance(out, np.ndarray):
        words = out.nbytes // 8 if out.flags.c_contiguous else -1
    else:
        words = out.numel() * out.element_size() // 8 if out.is_contiguous() else -1
    if words < n:
        raise ValueError(f"distance buffer must be a contiguous buffer of at least {n} 8-byte words")
    return out


def solve(g: Graph, source: int, criterion: int = IN_OUT, out=None, stream=None):
    """sssp_solve.  Returns (dist, phases); dist is ``out`` if given (a CUDA
    int64/uint64 tensor or a numpy uint64 array), else a new CUDA int64 tensor
    holding the uint64 bit patterns (view with ``as_uint64``)."""
    out = _dist_buffer(g.n, out)
    phases = ctypes.c_uint64()
    _check(lib().sssp_solve(g.handle, int(source), int(criterion), _ptr(out), ctypes.byref(phases),
                            _stream_ptr(stream)))
    return out, phases.value


def solve_trace(g: Graph, source: int, criterion: int = IN_OUT, out=None, trace_cap: int = 0,
                settle: bool = True, stream=None):
    """sssp_solve_trace.  Returns (dist, stats dict, settle_phase numpy uint32
    or None, trace numpy records or None)."""
    out = _dist_buffer(g.n, out)
    st = _Stats()
    sp = np.zeros(g.n, np.uint32) if settle else None
    tr = np.zeros(trace_cap, PHASE_RECORD) if trace_cap else None
    _check(lib().sssp_solve_trace(g.handle, int(source), int(criterion), _ptr(out), ctypes.byref(st),
                                  _ptr(sp) if sp is not None else None,
                                  _ptr(tr) if tr is not None else None, int(trace_cap), _stream_ptr(stream)))
    stats = {"phases": st.phases, "sum_frontier": st.sum_frontier, "settled": st.settled,
             "edges_relaxed": st.edges_relaxed}
    if tr is not None:
        tr = tr[:min(trace_cap, st.phases)]
    return out, stats, sp, tr


NOALLOC_MAX_VERTICES = 1 << 19


def _noalloc_inputs(n, row_off, edges):
    """Checks what the C ABI cannot see about the caller's CSR tensors: device,
    element size, contiguity and length (the library reads n+1 offsets and m
    {target, cost} pairs through raw pointers).  Raises ValueError."""
    for name, t, size in (("row_off", row_off, 8), ("edges", edges, 4)):
        if isinstance(t, np.ndarray) or not getattr(t, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.element_size() != size or t.is_floating_point() or t.is_complex():
            raise ValueError(f"{name} must hold {8 * size}-bit integers")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if row_off.numel() < n + 1:
        raise ValueError(f"row_off needs at least n+1 = {n + 1} entries, it has {row_off.numel()}")
    if edges.numel() % 2:
        raise ValueError("edges must hold {target, cost} pairs (an even number of 32-bit words)")


def solve_noalloc(n: int, row_off, edges, source: int, criterion: int = IN_OUT, out=None, stream=None):
    """sssp_solve_noalloc: a solve that allocates no device memory.  ``row_off``
    (int64/uint64, n+1) and ``edges`` (int32/uint32 pairs {target, cost}, 2*m)
    are CUDA tensors; ``out`` a CUDA int64 tensor of n (allocated here by torch
    if None -- pass it in to keep the whole call allocation-free).  Returns
    (dist, phases)."""
    _noalloc_inputs(n, row_off, edges)
    out = _dist_buffer(n, out)
    phases = ctypes.c_uint64()
    m = int(edges.numel()) // 2
    _check(lib().sssp_solve_noalloc(int(n), m, _ptr(row_off), _ptr(edges), int(source), int(criterion), _ptr(out),
                                    ctypes.byref(phases), _stream_ptr(stream)))
    return out, phases.value


POLICY_WEIGHTS = 1476
POLICY_FEATURES = 8
POLICY_ARMS = 4


def policy_load(weights):
    """sssp_policy_load: numpy float32[1476] or CUDA float32 tensor."""
    if isinstance(weights, np.ndarray):
        weights = np.ascontiguousarray(weights, dtype=np.float32)
        n = weights.size
    else:
        n = weights.numel()
    _check(lib().sssp_policy_load(_ptr(weights), n))


def policy_clear():
    _check(lib().sssp_policy_clear())


def policy_features(frontier, n, m, phase, edges_prev, settled_prev, frontier_prev) -> np.ndarray:
    out = np.zeros(POLICY_FEATURES, np.float32)
    _check(lib().sssp_policy_features(int(frontier), int(n), int(m), int(phase), int(edges_prev),
                                      int(settled_prev), int(frontier_prev), _ptr(out)))
    return out


def mlp_forward(w, x, y=None, stream=None):
    """sssp_mlp_forward on CUDA float32 tensors; returns y [B, 4]."""
    torch = _torch()
    B = x.shape[0]
    if y is None:
        y = torch.empty(B, POLICY_ARMS, dtype=torch.float32, device=x.device)
    _check(lib().sssp_mlp_forward(_ptr(w), _ptr(x), B, _ptr(y), _stream_ptr(stream)))
    return y


def mlp_backward(w, x, target, arm, grad=None, loss=None, stream=None):
    """sssp_mlp_backward on CUDA tensors; returns (grad [1476], loss [1])."""
    torch = _torch()
    if grad is None:
        grad = torch.empty(POLICY_WEIGHTS, dtype=torch.float32, device=x.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().sssp_mlp_backward(_ptr(w), _ptr(x), _ptr(target), _ptr(arm), x.shape[0], _ptr(grad), _ptr(loss),
                                   _stream_ptr(stream)))
    return grad, loss


def mlp_adam(w, grad, m1, m2, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().sssp_mlp_adam(_ptr(w), _ptr(grad), _ptr(m1), _ptr(m2), w.numel(), float(lr), float(beta1),
                               float(beta2), float(eps), int(step), _stream_ptr(stream)))


def _ptr_array(objs):
    arr = (ctypes.c_void_p * len(objs))()
    for i, o in enumerate(objs):
        arr[i] = o.handle.value if isinstance(o, Graph) else _ptr(o).value
    return arr


def solve_batch(graphs, sources, criterion: int = IN_OUT, outs=None, stream=None):
    """sssp_solve_batch.  ``outs``: list of CUDA tensors (n_i each), allocated
    if None.  Returns (outs, phases numpy uint64)."""
    torch = _torch()
    if outs is None:
        outs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for g in graphs]
    if len(outs) != len(graphs) or len(sources) != len(graphs):
        raise ValueError("graphs, sources and outs must have the same length")
    outs = [_dist_buffer(g.n, o) for g, o in zip(graphs, outs)]
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    phases = np.zeros(len(graphs), np.uint64)
    _check(lib().sssp_solve_batch(_ptr_array(graphs), _ptr(src), len(graphs), int(criterion), _ptr_array(outs),
                                  _ptr(phases), _stream_ptr(stream)))
    return outs, phases


class Batch:
    """A prepared batch (sssp_batch_create): descriptors, workspaces and the
    launch captured once in a CUDA graph; ``launch()`` replays it."""

    def __init__(self, graphs, sources, criterion: int = IN_OUT, outs=None, stream=None):
        torch = _torch()
        self.graphs = list(graphs)
        self.outs = outs if outs is not None else [torch.empty(g.n, dtype=torch.int64, device="cuda")
                                                   for g in self.graphs]
        if len(self.outs) != len(self.graphs) or len(sources) != len(self.graphs):
            raise ValueError("graphs, sources and outs must have the same length")
        self.outs = [_dist_buffer(g.n, o) for g, o in zip(self.graphs, self.outs)]
        self.phases = torch.zeros(len(self.graphs), dtype=torch.int64, device="cuda")
        src = np.ascontiguousarray(sources, dtype=np.uint32)
        h = ctypes.c_void_p()
        _check(lib().sssp_batch_create(_ptr_array(self.graphs), _ptr(src), len(self.graphs), int(criterion),
                                       _ptr_array(self.outs), _ptr(self.phases), _stream_ptr(stream),
                                       ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        _check(lib().sssp_batch_launch(self.handle, _stream_ptr(stream)))

    def attach_trace(self, i: int, trace_cap: int = 1 << 20, stream=None):
        """sssp_batch_trace: later launches record solve i's per-phase records
        (up to trace_cap) and per-vertex settle phases into device buffers
        owned here; read them with ``trace_of(i)``."""
        torch = _torch()
        tr = torch.zeros(trace_cap * PHASE_RECORD.itemsize, dtype=torch.uint8, device="cuda")
        settle = torch.zeros(self.graphs[i].n, dtype=torch.int32, device="cuda")
        _check(lib().sssp_batch_trace(self.handle, int(i), _ptr(tr), int(trace_cap), _ptr(settle),
                                      _stream_ptr(stream)))
        if not hasattr(self, "_traces"):
            self._traces = {}
        self._traces[i] = (tr, settle, trace_cap)

    def detach_trace(self, i: int, stream=None):
        """sssp_batch_trace with no buffers: later launches stop recording
        solve i (its last records stay readable with ``trace_of``)."""
        _check(lib().sssp_batch_trace(self.handle, int(i), None, 0, None, _stream_ptr(stream)))

    def trace_of(self, i: int):
        """(settle_phase numpy uint32, trace records) of solve i after a launch."""
        tr, settle, cap = self._traces[i]
        phases = int(self.phases[i].item())
        recs = tr.cpu().numpy().view(PHASE_RECORD)[:min(cap, phases)]
        return settle.cpu().numpy().view(np.uint32), recs

    def autotune(self, stream=None):
        """sssp_batch_autotune: walk the blocks-per-solve ladder from the
        batch's own choice, keep the fastest candidate timed; returns (blocks
        per solve, ms per launch)."""
        bpg = ctypes.c_uint32()
        ms = ctypes.c_float()
        _check(lib().sssp_batch_autotune(self.handle, _stream_ptr(stream), ctypes.byref(bpg), ctypes.byref(ms)))
        return bpg.value, ms.value

    def close(self):
        if getattr(self, "handle", None):
            lib().sssp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def as_uint64(x) -> np.ndarray:
    """uint64 numpy view of a distance buffer (CUDA tensor or numpy array)."""
    if isinstance(x, np.ndarray):
        return x.view(np.uint64)
    return x.detach().cpu().numpy().view(np.uint64)

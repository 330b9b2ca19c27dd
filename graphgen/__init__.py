"""Seeded synthetic inputs shared by the CPU oracle and the CUDA solver.

This package holds no shortest-path arithmetic.  It draws graphs (uniform
G(n,m), 4-neighbour grids, R-MAT) from SplitMix64 streams in C
(``graphgen.c``) and hands them out as CSR arrays:

* ``row_off``  uint64[n+1]  out-edges of vertex u are ``[row_off[u], row_off[u+1])``
* ``col``      uint32[m]    edge targets
* ``w``        uint32[m]    edge costs, each < 0xFFFFFFFF

The five workloads are the phase-parallel Dijkstra study's input families
(uniform random graphs and Kronecker graphs of Section 4, road networks
replaced by grids), scaled as listed in ``WORKLOADS``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

SEED_BASE = 0x1903120850
INF_W = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (portable C, -O3)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-o", _LIB, _SRC])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u32, u64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        lib.gg_splitmix64_nth.restype = u64
        lib.gg_splitmix64_nth.argtypes = [u64, u64]
        lib.gg_gnm.restype = ctypes.c_int
        lib.gg_gnm.argtypes = [u32, u64, u32, u32, u64, p, p, p]
        lib.gg_grid_edges.restype = u64
        lib.gg_grid_edges.argtypes = [u32, u32]
        lib.gg_grid.restype = ctypes.c_int
        lib.gg_grid.argtypes = [u32, u32, u32, u32, u64, p, p, p]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_rmat.argtypes = [u32, u64, u32, u32, u32, u32, u32, u64, p, p, p]
        lib.gg_batch_params.restype = ctypes.c_int
        lib.gg_batch_params.argtypes = [u32, u32, u32, u32, u32, u32, u64, p, p, p, p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """A directed graph in CSR form (see module docstring)."""

    n: int
    row_off: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def outdeg(self) -> np.ndarray:
        return np.diff(self.row_off).astype(np.int64)


@dataclass
class Workload:
    """Graphs plus the (graph index, source) pairs that are solved on them."""

    name: str
    graphs: list
    solves: list = field(default_factory=list)  # list of (graph_index, source)


def splitmix64_nth(seed: int, k: int) -> int:
    """k-th (0-based) output of the SplitMix64 stream started at ``seed``."""
    return int(_load().gg_splitmix64_nth(seed, k))


def gnm(n: int, m: int, wlo: int, whi: int, seed: int, name: str = "") -> Graph:
    """Directed G(n,m): endpoints uniform, self-loops redrawn, duplicates kept,
    weights uniform in [wlo, whi)."""
    row_off = np.empty(n + 1, np.uint64)
    col = np.empty(max(m, 1), np.uint32)[:m]
    w = np.empty(max(m, 1), np.uint32)[:m]
    rc = _load().gg_gnm(n, m, wlo, whi, seed, _ptr(row_off), _ptr(col), _ptr(w))
    if rc != 0:
        raise ValueError("gg_gnm failed")
    return Graph(n, row_off, col, w, name or f"gnm_n{n}_m{m}")


def grid(rows: int, cols: int, wlo: int, whi: int, seed: int, name: str = "") -> Graph:
    """Undirected rows x cols 4-neighbour grid as symmetric directed edges."""
    n = rows * cols
    m = int(_load().gg_grid_edges(rows, cols))
    row_off = np.empty(n + 1, np.uint64)
    col = np.empty(max(m, 1), np.uint32)[:m]
    w = np.empty(max(m, 1), np.uint32)[:m]
    rc = _load().gg_grid(rows, cols, wlo, whi, seed, _ptr(row_off), _ptr(col), _ptr(w))
    if rc != 0:
        raise ValueError("gg_grid failed")
    return Graph(n, row_off, col, w, name or f"grid_{rows}x{cols}")


def _thr(p: float) -> int:
    return min(int(round(p * 2.0**32)), 2**32 - 1)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, wlo: int, whi: int,
         seed: int, name: str = "", m: int | None = None) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale edges (or
    exactly m edges when m is given)."""
    n = 1 << scale
    m = edge_factor * n if m is None else int(m)
    row_off = np.empty(n + 1, np.uint64)
    col = np.empty(m, np.uint32)
    w = np.empty(m, np.uint32)
    rc = _load().gg_rmat(scale, m, _thr(a), _thr(a + b), _thr(a + b + c), wlo, whi, seed,
                         _ptr(row_off), _ptr(col), _ptr(w))
    if rc != 0:
        raise ValueError("gg_rmat failed")
    return Graph(n, row_off, col, w, name or f"rmat_s{scale}_ef{edge_factor}")


def batch_params(count: int, lo_exp: int, hi_exp: int, deg_lo: int, deg_hi: int,
                 sources_per_graph: int, seed: int):
    n = np.empty(count, np.uint32)
    m = np.empty(count, np.uint64)
    seeds = np.empty(count, np.uint64)
    src = np.empty(count * sources_per_graph, np.uint32)
    rc = _load().gg_batch_params(count, lo_exp, hi_exp, deg_lo, deg_hi, sources_per_graph, seed,
                                 _ptr(n), _ptr(m), _ptr(seeds), _ptr(src))
    if rc != 0:
        raise ValueError("gg_batch_params failed")
    return n, m, seeds, src.reshape(count, sources_per_graph)


def from_edges(n: int, edges, name: str = "") -> Graph:
    """CSR from an explicit list of (u, v, cost) triples; row order kept."""
    edges = list(edges)
    row_off = np.zeros(n + 1, np.uint64)
    for u, _, _ in edges:
        row_off[u + 1] += 1
    row_off = np.cumsum(row_off, dtype=np.uint64)
    fill = row_off[:-1].copy()
    col = np.zeros(len(edges), np.uint32)
    w = np.zeros(len(edges), np.uint32)
    for u, v, c in edges:
        p = int(fill[u])
        col[p] = v
        w[p] = c
        fill[u] += 1
    return Graph(n, row_off, col, w, name or "explicit")


def max_outdeg_vertex(g: Graph) -> int:
    """Vertex of largest out-degree, lowest id on ties."""
    return int(np.argmax(g.outdeg()))


# ---------------------------------------------------------------------------
# The five workloads.  Seed of workload k is SEED_BASE + k.

WORKLOADS = {
    1: "gnm_n16384_m131072: directed G(n,m), n=16384, m=131072, w in [0,2^24), source 0",
    2: "grid_1024x1024: undirected 4-grid, w in [1,2^16), source (0,0)",
    3: "rmat_s22_ef16: R-MAT (.57,.19,.19,.05), w in [0,2^24), source = max out-degree",
    4: "batch_256: 256 G(n,m), n log-uniform in [2^10,2^18), average degree U[4,32], w in [0,2^20), 4 sources each",
    5: "gnm_n2^24_m2^28: directed G(n,m), w in [0,2^24), 8 uniform sources",
}


def workload(k: int, shrink: int = 0) -> Workload:
    """Workload k (1..5).  ``shrink`` > 0 gives a smaller graph of the same
    family for fast tests: every size parameter is divided by 2^shrink (grid
    sides by 2^(shrink/2) each, R-MAT scale reduced by shrink, the batch keeps
    at most 256 >> shrink graphs with the n range shifted down)."""
    seed = SEED_BASE + k
    if k == 1:
        n, m = 16384 >> shrink, 131072 >> shrink
        g = gnm(max(n, 2), max(m, 1), 0, 1 << 24, seed, "gnm_n16384_m131072" if not shrink else "")
        return Workload(g.name, [g], [(0, 0)])
    if k == 2:
        side = 1024 >> (shrink // 2)
        if shrink % 2:
            side = int(side / 2**0.5)
        g = grid(side, side, 1, 1 << 16, seed)
        return Workload(g.name, [g], [(0, 0)])
    if k == 3:
        g = rmat(22 - shrink, 16, 0.57, 0.19, 0.19, 0, 1 << 24, seed)
        return Workload(g.name, [g], [(0, max_outdeg_vertex(g))])
    if k == 4:
        count = max(256 >> shrink, 2)
        lo, hi = 10 - min(shrink, 6), 18 - min(shrink, 6)
        n, m, seeds, src = batch_params(count, lo, hi, 4, 32, 4, seed)
        graphs = [gnm(int(n[i]), int(m[i]), 0, 1 << 20, int(seeds[i]), f"batch{i}")
                  for i in range(count)]
        solves = [(i, int(s)) for i in range(count) for s in src[i]]
        return Workload(f"batch_{count}", graphs, solves)
    if k == 5:
        n, m = (1 << 24) >> shrink, (1 << 28) >> shrink
        g = gnm(n, m, 0, 1 << 24, seed)
        r = [int(splitmix64_nth(seed ^ 0x5EED, i) >> 32) * n >> 32 for i in range(8)]
        return Workload(g.name, [g], [(0, s) for s in r])
    raise ValueError(f"unknown workload {k}")

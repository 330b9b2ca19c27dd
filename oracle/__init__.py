"""CPU oracle for the phase-parallel Dijkstra (Kainer & Traeff, arXiv:1903.12085).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA product path never
imports, links or runs anything here, and this package shares no code with it.

* ``dijkstra``      binary-heap Dijkstra (Section 2): the plain definition of
                    dist(s, v), UINT64_MAX for unreachable vertices.
* ``dijkstra_prefix``  the same run stopped after a number of settled vertices
                    (a bounded sample of a solve's work, for the CPU timings).
* ``bellman_ford``  brute-force relaxation of all edges, for small graphs.
* ``simulate``      the generic phased algorithm (Section 3) with the IN/OUT
                    criteria of Section 3 (eqs. crit:in, crit:out, crit:outweak,
                    crit:instatic, crit:outstatic, crit:insimple,
                    crit:outsimple), DIJK and ORACLE; per phase it settles all
                    fringe vertices that satisfy the criterion mask on the
                    phase-start state.
* ``mlp``           float64 forward/backward of the phase-policy network.

The C source (``oracle.c``) documents each reading of the paper it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

INF = np.uint64(0xFFFFFFFFFFFFFFFF)

# Criterion bits (a disjunction of all bits set).
IN_STATIC = 1
OUT_STATIC = 2
IN_SIMPLE = 4
OUT_SIMPLE = 8
IN_FULL = 16
OUT_WEAK = 32
DIJK = 64
ORACLE = 128
OUT_FULL = 256
APPROX = 512  # approximate IN (full) / OUT-WEAK minima, recomputed every k-th phase


def approx(k: int) -> int:
    """Criterion bits of APPROX with recomputation every k-th phase (1..63)."""
    assert 1 <= k <= 63
    return APPROX | (k << 10)

_ERRORS = {-1: "out of memory", -2: "bad argument", -3: "a phase selected no vertex (criterion not complete)",
           -4: "a selected vertex was not correct (criterion not sound)"}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (portable C, -O3)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-o", _LIB, _SRC])
    return _LIB


def _configure(lib):
    u32, u64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    for name in ("orc_dijkstra", "orc_bellman_ford"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [u32, p, p, p, u32, p]
    lib.orc_dijkstra_prefix.restype = ctypes.c_int
    lib.orc_dijkstra_prefix.argtypes = [u32, p, p, p, u32, u64, p, p]
    lib.orc_simulate.restype = ctypes.c_int
    lib.orc_simulate.argtypes = [u32, p, p, p, u32, p, u64, u32, p, p, p, p, p, u64]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def _csr(g):
    ro = np.ascontiguousarray(g.row_off, dtype=np.uint64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    if col.size == 0:  # keep valid pointers for edgeless graphs
        col = np.zeros(1, np.uint32)
        w = np.zeros(1, np.uint32)
    return ro, col, w


def dijkstra(g, s: int) -> np.ndarray:
    ro, col, w = _csr(g)
    dist = np.empty(g.n, np.uint64)
    rc = _load().orc_dijkstra(g.n, ro.ctypes.data, col.ctypes.data, w.ctypes.data, s, dist.ctypes.data)
    if rc:
        raise RuntimeError(f"orc_dijkstra: {_ERRORS.get(rc, rc)}")
    return dist


def dijkstra_prefix(g, s: int, max_settled: int):
    """Dijkstra from s stopped after max_settled settled vertices (a bounded
    sample of a solve, for timing).  Returns (settled, sum of their
    out-degrees)."""
    ro, col, w = _csr(g)
    dist = np.empty(g.n, np.uint64)
    counts = np.zeros(2, np.uint64)
    rc = _load().orc_dijkstra_prefix(g.n, ro.ctypes.data, col.ctypes.data, w.ctypes.data, s, int(max_settled),
                                     dist.ctypes.data, counts.ctypes.data)
    if rc:
        raise RuntimeError(f"orc_dijkstra_prefix: {_ERRORS.get(rc, rc)}")
    return int(counts[0]), int(counts[1])


def bellman_ford(g, s: int) -> np.ndarray:
    ro, col, w = _csr(g)
    dist = np.empty(g.n, np.uint64)
    rc = _load().orc_bellman_ford(g.n, ro.ctypes.data, col.ctypes.data, w.ctypes.data, s, dist.ctypes.data)
    if rc:
        raise RuntimeError(f"orc_bellman_ford: {_ERRORS.get(rc, rc)}")
    return dist


@dataclass
class SimResult:
    d: np.ndarray             # final distances
    settle_phase: np.ndarray  # uint32, phase in which each vertex settled (0 = never)
    phases: int
    sum_f: int                # sum over phases of |F| at phase start
    settled: int
    relaxed: int              # sum of out-degrees of settled vertices
    trace: np.ndarray | None  # [phases, 6]: |F|, |S'|, minD, minOut, deg(S'), mask


def simulate(g, s: int, crit: int, schedule=None, dist_ref=None, trace: bool = False) -> SimResult:
    """Run the phased algorithm; ``schedule`` (optional) gives the criterion
    mask of phases 1, 2, ...; later phases use ``crit``."""
    ro, col, w = _csr(g)
    d = np.empty(g.n, np.uint64)
    sp = np.empty(g.n, np.uint32)
    stats = np.zeros(4, np.uint64)
    sched = None if schedule is None else np.ascontiguousarray(schedule, dtype=np.uint32)
    ref = None if dist_ref is None else np.ascontiguousarray(dist_ref, dtype=np.uint64)
    cap = g.n + 1 if trace else 0
    tr = np.zeros((max(cap, 1), 6), np.uint64) if trace else None
    rc = _load().orc_simulate(
        g.n, ro.ctypes.data, col.ctypes.data, w.ctypes.data, s,
        None if sched is None else sched.ctypes.data, 0 if sched is None else sched.size, crit,
        None if ref is None else ref.ctypes.data, d.ctypes.data, sp.ctypes.data, stats.ctypes.data,
        None if tr is None else tr.ctypes.data, cap)
    if rc:
        raise RuntimeError(f"orc_simulate: {_ERRORS.get(rc, rc)}")
    phases = int(stats[0])
    return SimResult(d, sp, phases, int(stats[1]), int(stats[2]), int(stats[3]),
                     tr[:phases].copy() if tr is not None else None)

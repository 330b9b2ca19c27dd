"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one (on the CPU; the real oracle is untouched)."""
import ctypes
import os
import subprocess

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "in_le_to_lt": ("sel = dv <= sat_add(minD, in_min(", "sel = dv < sat_add(minD, in_min("),
    "out_le_to_lt": ("sel = dv <= minOut[k];", "sel = dv < minOut[k];"),
    "in_dynamic_skips_F_not_S": ("if (g->st[x] == ST_S) continue;                  /* edges from S",
                                 "if (g->st[x] == ST_F) continue;                  /* edges from S"),
    "out_dynamic_keeps_S": ("if (g->st[x] == ST_S) continue;                  /* edges into S",
                            "if (0) continue;                  /* edges into S"),
    "out_static_uses_in_min": ("return w64(g->out_st[u]);", "return w64(g->in_st[u]);"),
    "in_static_uses_out_min": ("return w64(g->in_st[v]);", "return w64(g->out_st[v]);"),
    "in_full_uses_out_min": ("c = sat_add(c, w64(g->in_st[x]));", "c = sat_add(c, w64(g->out_st[x]));"),
    "out_weak_drops_second_edge": ("if (which == ORC_OUT_WEAK) c = sat_add(c, w64(g->out_st[x]));",
                                   "if (which == ORC_OUT_WEAK) c = c;"),
    "in_full_drops_unexplored_term": ("if (which == ORC_IN_FULL && g->st[x] == ST_U)    /* two edges outside S */\n            c = sat_add(",
                                      "if (0)\n            c = sat_add("),
    "in_full_term_for_fringe_sources": ("if (which == ORC_IN_FULL && g->st[x] == ST_U)    /* two edges outside S */",
                                        "if (which == ORC_IN_FULL && g->st[x] != ST_S)    /* two edges outside S */"),
    "out_weak_term_for_fringe_targets": ("if (g->st[x] == ST_U) {\n            if (which == ORC_OUT_WEAK)",
                                         "if (g->st[x] != ST_S) {\n            if (which == ORC_OUT_WEAK)"),
    "dijk_tie_takes_queue_order": ("(d_out[v] == minD && v < argmin)", "(d_out[v] == minD && v > argmin)"),
    "heap_wrong_child": ("h->a[r].key < h->a[l].key) c = r;", "h->a[r].key > h->a[l].key) c = r;"),
    "new_vertex_not_queued": ("g.st[t] = ST_F; Fn[nFn++] = t;", "g.st[t] = ST_F;"),
    "sum_f_off_by_one": ("sumF += nF;", "sumF += nF - 1;"),
    "bellman_ford_one_round_short": ("round + 1 < n || round == 0", "round + 2 < n"),
    "minout_misses_first_entry": ("for (uint64_t i = 0; i < nF; ++i) {\n                uint64_t val = sat_add(d_out[F[i]], out_min(",
                                  "for (uint64_t i = 1; i < nF; ++i) {\n                uint64_t val = sat_add(d_out[F[i]], out_min("),
    "approx_skips_in_update": ("if (g.st[col[e]] == ST_F && w[e] < ain[col[e]]) ain[col[e]] = w[e];",
                               "if (0) ain[col[e]] = w[e];"),
    "approx_never_recomputes": ("if ((phases - 1) % kk == 0)", "if (phases == 0)"),
    "approx_out_update_wrong_side": ("if (g.st[g.rsrc[e]] == ST_F && g.rw[e] < aout[g.rsrc[e]]) aout[g.rsrc[e]] = g.rw[e];",
                                     "if (0) aout[g.rsrc[e]] = g.rw[e];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path_c = tmp_path / "mut.c"
    path_c.write_text(src.replace(old, new))
    path_so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(path_so), str(path_c)])
    saved = oracle._load()
    oracle._lib = oracle._configure(ctypes.CDLL(str(path_so)))
    caught = []
    try:
        for pin in P.ALL_PINS:
            try:
                pin(oracle)
            except (AssertionError, RuntimeError) as e:  # RuntimeError: oracle's own soundness check
                caught.append(pin.__name__)
                break
    finally:
        oracle._lib = saved
    assert caught, f"no pin caught mutant {name}"

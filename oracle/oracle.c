/*
 * oracle.c -- plain, sequential CPU oracle for the phase-parallel Dijkstra
 * of Kainer & Traeff, "More Parallelism in Dijkstra's Single-Source Shortest
 * Path Algorithm" (arXiv:1903.12085).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only the tests, the package smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header or table with the CUDA solver.
 *
 * Contents
 *   orc_dijkstra      Dijkstra's algorithm (Section 2) with a binary heap and
 *                     lazy deletion: the plain definition of dist(s, v).
 *   orc_dijkstra_prefix  the same run stopped after a given number of settled
 *                     vertices (a bounded sample of its work, for timing).
 *   orc_bellman_ford  n-1 rounds of relaxing every edge: an independent
 *                     brute-force check of the distances on small graphs.
 *   orc_simulate      the generic phased SSSP algorithm (Section 3) run with a
 *                     per-phase criterion mask.  Every phase evaluates the
 *                     chosen criteria on the state at the start of the phase,
 *                     settles ALL fringe vertices that satisfy one of them
 *                     (the phase model of Section 4's simulations, where
 *                     every vertex meeting the criterion at the start of a
 *                     phase is taken), then relaxes their out-edges.
 *
 * Criterion bits (a disjunction of every bit set), with the equations they
 * restate:
 *   1   IN-STATIC   d[v] - min_{(w,v) in E} c(w,v)            <= min_F d   (eq. crit:instatic)
 *   2   OUT-STATIC  d[v] <= min_{u in F} d[u] + min_{(u,w)} c  (eq. crit:outstatic)
 *   4   IN-SIMPLE   as IN-STATIC over in-edges from w not in S (eq. crit:insimple)
 *   8   OUT-SIMPLE  as OUT-STATIC over out-edges to w not in S (eq. crit:outsimple,
 *                   read with u in F and w in F u U; the printed index set is
 *                   garbled and, taken literally, equals OUT-STATIC)
 *   16  IN (full)   eq. crit:in: in-edge from w in F costs c(w,v); from w in U
 *                   it costs c(w,v) + M'[w] with M'[w] the static in-minimum of
 *                   w (the precomputation argument of Proposition 1)
 *   32  OUT-WEAK    eq. crit:outweak: out-edge to w in F costs c(u,w); to w in U
 *                   it costs c(u,w) + M[w] with M[w] the static out-minimum
 *   64  DIJK        one vertex of minimum d (lowest id on ties)
 *   128 ORACLE      d[v] = dist(s,v), using the caller's reference distances
 *   256 OUT (full)  eq. crit:out: to w in U it costs c(u,w) + min over out-edges
 *                   (w,w') with w' not in S
 *   512 APPROX(k)   the approximate IN (full) and OUT-WEAK minima of the paper's
 *                   closing remark in Section 3, in a deterministic schedule: in
 *                   every k-th phase (phases 1, k+1, 2k+1, ...) each fringe
 *                   vertex gets the exact IN (full) and OUT-WEAK terms; a vertex
 *                   that enters F starts from its static minima; when w enters F
 *                   every fringe v with an edge (w,v) lowers its IN value to
 *                   c(w,v) if smaller, every fringe u with an edge (u,w) lowers
 *                   its OUT value to c(u,w) if smaller; nothing else changes the
 *                   values between recomputations.  A value is then never above
 *                   the exact term (deletions are ignored: too small is
 *                   conservative) and never below the static minimum, so the
 *                   criterion is sound and complete.  k sits in mask bits 10..15
 *                   (0 means 1).
 * All arithmetic is exact unsigned integer.  "d[v] - x <= minD" is evaluated as
 * d[v] <= minD + x so nothing underflows; an empty minimum is infinite and
 * makes the IN test true and contributes nothing to an OUT threshold.
 * The minima of the dynamic criteria are evaluated against S as it stands at
 * the start of the phase.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF64 UINT64_MAX
#define ORC_INF32 0xFFFFFFFFu

enum {
    ORC_IN_STATIC = 1u, ORC_OUT_STATIC = 2u, ORC_IN_SIMPLE = 4u, ORC_OUT_SIMPLE = 8u,
    ORC_IN_FULL = 16u, ORC_OUT_WEAK = 32u, ORC_DIJK = 64u, ORC_ORACLE = 128u, ORC_OUT_FULL = 256u,
    ORC_APPROX = 512u, ORC_APPROX_K_SHIFT = 10u, ORC_APPROX_K_MASK = 63u
};
enum { ST_U = 0, ST_F = 1, ST_S = 2 };

/* ------------------------------------------------------------------ */
/* Binary min-heap of (key, vertex) pairs, lazy deletion.              */
typedef struct { uint64_t key; uint32_t v; } orc_item;
typedef struct { orc_item* a; size_t len, cap; } orc_heap;

static int heap_push(orc_heap* h, uint64_t key, uint32_t v) {
    if (h->len == h->cap) {
        size_t nc = h->cap ? 2 * h->cap : 1024;
        orc_item* na = (orc_item*)realloc(h->a, nc * sizeof(orc_item));
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    size_t i = h->len++;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key; h->a[i].v = v;
    return 0;
}

static orc_item heap_pop(orc_heap* h) {
    orc_item top = h->a[0];
    orc_item last = h->a[--h->len];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, c = l;
        if (l >= h->len) break;
        if (r < h->len && h->a[r].key < h->a[l].key) c = r;
        if (h->a[c].key >= last.key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->len) h->a[i] = last;
    return top;
}

/* Dijkstra (Section 2): repeatedly settle the fringe vertex of minimum
 * tentative distance and relax its out-edges, until the heap is empty or
 * max_settled vertices are settled.  counts (may be NULL) receives the number
 * of settled vertices and the sum of their out-degrees.  Returns 0, -1 on OOM,
 * -2 on a bad argument. */
static int dijkstra_run(uint32_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                        uint32_t s, uint64_t max_settled, uint64_t* dist, uint64_t* counts) {
    if (s >= n) return -2;
    for (uint32_t v = 0; v < n; ++v) dist[v] = ORC_INF64;
    uint8_t* done = (uint8_t*)calloc(n, 1);
    orc_heap h = {0, 0, 0};
    if (!done) return -1;
    dist[s] = 0;
    if (heap_push(&h, 0, s)) { free(done); return -1; }
    uint64_t settled = 0, scanned = 0;
    while (h.len && settled < max_settled) {
        orc_item it = heap_pop(&h);
        uint32_t u = it.v;
        if (done[u] || it.key != dist[u]) continue;
        done[u] = 1;
        ++settled;
        scanned += row_off[u + 1] - row_off[u];
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint32_t t = col[e];
            uint64_t cand = dist[u] + w[e];
            if (cand < dist[t]) {
                dist[t] = cand;
                if (heap_push(&h, cand, t)) { free(h.a); free(done); return -1; }
            }
        }
    }
    free(h.a);
    free(done);
    if (counts) { counts[0] = settled; counts[1] = scanned; }
    return 0;
}

int orc_dijkstra(uint32_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                 uint32_t s, uint64_t* dist) {
    return dijkstra_run(n, row_off, col, w, s, UINT64_MAX, dist, NULL);
}

/* The first max_settled settled vertices of a Dijkstra run (a bounded sample
 * of a solve's work for timing; dist is final only for the settled ones). */
int orc_dijkstra_prefix(uint32_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                        uint32_t s, uint64_t max_settled, uint64_t* dist, uint64_t* counts) {
    return dijkstra_run(n, row_off, col, w, s, max_settled, dist, counts);
}

/* Bellman-Ford: relax every edge until nothing changes (at most n-1 rounds). */
int orc_bellman_ford(uint32_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                     uint32_t s, uint64_t* dist) {
    if (s >= n) return -2;
    for (uint32_t v = 0; v < n; ++v) dist[v] = ORC_INF64;
    dist[s] = 0;
    for (uint32_t round = 0; round + 1 < n || round == 0; ++round) {
        int changed = 0;
        for (uint32_t u = 0; u < n; ++u) {
            if (dist[u] == ORC_INF64) continue;
            for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
                uint64_t cand = dist[u] + w[e];
                if (cand < dist[col[e]]) { dist[col[e]] = cand; changed = 1; }
            }
        }
        if (!changed) break;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Simulator of the generic phased algorithm.                          */

typedef struct {
    uint32_t n;
    const uint64_t* ro; const uint32_t* col; const uint32_t* w;
    uint64_t* rro; uint32_t* rsrc; uint32_t* rw;  /* reverse CSR (in-edges) */
    uint32_t* out_st;   /* M[v]  = min over out-edges, INF32 if none */
    uint32_t* in_st;    /* M'[v] = min over in-edges,  INF32 if none */
    uint8_t* st;        /* ST_U / ST_F / ST_S */
    uint64_t* d;
} orc_sim;

static uint64_t sat_add(uint64_t a, uint64_t b) {
    return (a == ORC_INF64 || b == ORC_INF64 || a > ORC_INF64 - b) ? ORC_INF64 : a + b;
}
static uint64_t w64(uint32_t x) { return x == ORC_INF32 ? ORC_INF64 : (uint64_t)x; }

/* Minimum in-edge cost into v for the IN variant `which` (one bit). */
static uint64_t in_min(const orc_sim* g, uint32_t v, uint32_t which) {
    if (which == ORC_IN_STATIC) return w64(g->in_st[v]);
    uint64_t best = ORC_INF64;
    for (uint64_t e = g->rro[v]; e < g->rro[v + 1]; ++e) {
        uint32_t x = g->rsrc[e];
        if (g->st[x] == ST_S) continue;                  /* edges from S are gone */
        uint64_t c = g->rw[e];
        if (which == ORC_IN_FULL && g->st[x] == ST_U)    /* two edges outside S */
            c = sat_add(c, w64(g->in_st[x]));
        if (c < best) best = c;
    }
    return best;
}

/* Minimum out-edge cost out of u for the OUT variant `which` (one bit). */
static uint64_t out_min(const orc_sim* g, uint32_t u, uint32_t which) {
    if (which == ORC_OUT_STATIC) return w64(g->out_st[u]);
    uint64_t best = ORC_INF64;
    for (uint64_t e = g->ro[u]; e < g->ro[u + 1]; ++e) {
        uint32_t x = g->col[e];
        if (g->st[x] == ST_S) continue;                  /* edges into S are gone */
        uint64_t c = g->w[e];
        if (g->st[x] == ST_U) {
            if (which == ORC_OUT_WEAK) c = sat_add(c, w64(g->out_st[x]));
            else if (which == ORC_OUT_FULL) {
                uint64_t b2 = ORC_INF64;
                for (uint64_t f = g->ro[x]; f < g->ro[x + 1]; ++f)
                    if (g->st[g->col[f]] != ST_S && g->w[f] < b2) b2 = g->w[f];
                c = sat_add(c, b2);
            }
        }
        if (c < best) best = c;
    }
    return best;
}

/*
 * orc_simulate -- run the generic phased algorithm from source s.
 *
 * schedule[k] is the criterion mask of phase k+1; phases beyond schedule_len
 * use default_crit.  dist_ref (may be NULL unless ORACLE is requested) are the
 * true distances; when given, every settled vertex is checked against them
 * (soundness).  Outputs:
 *   d_out[n]          final tentative distances
 *   settle_phase[n]   phase (1-based) in which each vertex was settled, 0 if never
 *   stats[4]          phases, sum over phases of |F| at phase start,
 *                     vertices settled, edges relaxed (sum of their out-degrees)
 *   trace (optional, trace_cap records of 6 uint64 each):
 *                     |F|, |S'|, minD, minOut (of the strongest OUT bit set, else
 *                     INF), sum of out-degrees of S', criterion mask
 * Returns 0; -1 out of memory; -2 bad argument; -3 a phase selected nothing
 * while F was non-empty (criterion not complete); -4 a selected vertex had
 * d != dist_ref (criterion not sound).
 */
int orc_simulate(uint32_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                 uint32_t s, const uint32_t* schedule, uint64_t schedule_len, uint32_t default_crit,
                 const uint64_t* dist_ref, uint64_t* d_out, uint32_t* settle_phase,
                 uint64_t* stats, uint64_t* trace, uint64_t trace_cap) {
    if (s >= n || !d_out || !settle_phase || !stats) return -2;
    uint64_t m = row_off[n];
    orc_sim g;
    memset(&g, 0, sizeof g);
    g.n = n; g.ro = row_off; g.col = col; g.w = w; g.d = d_out;
    g.rro = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    g.rsrc = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    g.rw = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    g.out_st = (uint32_t*)malloc(sizeof(uint32_t) * n);
    g.in_st = (uint32_t*)malloc(sizeof(uint32_t) * n);
    g.st = (uint8_t*)calloc(n, 1);
    uint32_t* F = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint32_t* Fn = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint32_t* Sp = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* fill = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint64_t* ain = (uint64_t*)malloc(sizeof(uint64_t) * n);   /* APPROX: IN values */
    uint64_t* aout = (uint64_t*)malloc(sizeof(uint64_t) * n);  /* APPROX: OUT-WEAK values */
    uint32_t* fresh = (uint32_t*)malloc(sizeof(uint32_t) * n);  /* vertices that entered F this phase */
    int rc = 0;
    if (!g.rro || !g.rsrc || !g.rw || !g.out_st || !g.in_st || !g.st || !F || !Fn || !Sp || !fill ||
        !ain || !aout || !fresh) {
        rc = -1; goto done;
    }
    /* Preprocessing (Section 5): static minima and the in-edge lists. */
    for (uint32_t v = 0; v < n; ++v) { g.out_st[v] = ORC_INF32; g.in_st[v] = ORC_INF32; }
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            if (w[e] < g.out_st[u]) g.out_st[u] = w[e];
            if (w[e] < g.in_st[col[e]]) g.in_st[col[e]] = w[e];
            g.rro[col[e] + 1]++;
        }
    for (uint32_t v = 0; v < n; ++v) g.rro[v + 1] += g.rro[v];
    memcpy(fill, g.rro, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint64_t p = fill[col[e]]++;
            g.rsrc[p] = u;
            g.rw[p] = w[e];
        }

    for (uint32_t v = 0; v < n; ++v) { d_out[v] = ORC_INF64; settle_phase[v] = 0; }
    d_out[s] = 0;
    g.st[s] = ST_F;
    ain[s] = w64(g.in_st[s]);
    aout[s] = w64(g.out_st[s]);
    uint64_t nF = 1, phases = 0, sumF = 0, settled = 0, relaxed = 0;
    F[0] = s;

    while (nF > 0) {
        ++phases;
        uint32_t crit = (phases - 1 < schedule_len && schedule) ? schedule[phases - 1] : default_crit;
        if (crit == 0) { rc = -2; break; }
        if ((crit & ORC_ORACLE) && !dist_ref) { rc = -2; break; }
        sumF += nF;

        /* Thresholds from the phase-start snapshot. */
        uint64_t minD = ORC_INF64;
        uint32_t argmin = ORC_INF32;
        for (uint64_t i = 0; i < nF; ++i) {
            uint32_t v = F[i];
            if (d_out[v] < minD || (d_out[v] == minD && v < argmin)) { minD = d_out[v]; argmin = v; }
        }
        static const uint32_t out_bits[4] = {ORC_OUT_STATIC, ORC_OUT_SIMPLE, ORC_OUT_WEAK, ORC_OUT_FULL};
        static const uint32_t in_bits[3] = {ORC_IN_STATIC, ORC_IN_SIMPLE, ORC_IN_FULL};
        uint64_t minOut[4];
        for (int k = 0; k < 4; ++k) {
            minOut[k] = ORC_INF64;
            if (!(crit & out_bits[k])) continue;
            for (uint64_t i = 0; i < nF; ++i) {
                uint64_t val = sat_add(d_out[F[i]], out_min(&g, F[i], out_bits[k]));
                if (val < minOut[k]) minOut[k] = val;
            }
        }
        /* APPROX: exact terms in every k-th phase, then the threshold. */
        uint64_t minOutA = ORC_INF64;
        if (crit & ORC_APPROX) {
            uint32_t kk = (crit >> ORC_APPROX_K_SHIFT) & ORC_APPROX_K_MASK;
            if (kk == 0) kk = 1;
            if ((phases - 1) % kk == 0)
                for (uint64_t i = 0; i < nF; ++i) {
                    ain[F[i]] = in_min(&g, F[i], ORC_IN_FULL);
                    aout[F[i]] = out_min(&g, F[i], ORC_OUT_WEAK);
                }
            for (uint64_t i = 0; i < nF; ++i) {
                uint64_t val = sat_add(d_out[F[i]], aout[F[i]]);
                if (val < minOutA) minOutA = val;
            }
        }
        /* Select S': every v in F satisfying one of the criteria. */
        uint64_t nS = 0, nFn = 0, degS = 0;
        for (uint64_t i = 0; i < nF; ++i) {
            uint32_t v = F[i];
            uint64_t dv = d_out[v];
            int sel = 0;
            for (int k = 0; k < 3 && !sel; ++k)
                if (crit & in_bits[k]) sel = dv <= sat_add(minD, in_min(&g, v, in_bits[k]));
            for (int k = 0; k < 4 && !sel; ++k)
                if (crit & out_bits[k]) sel = dv <= minOut[k];
            if (!sel && (crit & ORC_APPROX)) sel = dv <= sat_add(minD, ain[v]) || dv <= minOutA;
            if (!sel && (crit & ORC_DIJK)) sel = (v == argmin);
            if (!sel && (crit & ORC_ORACLE)) sel = (dv == dist_ref[v]);
            if (sel) Sp[nS++] = v; else Fn[nFn++] = v;
        }
        if (nS == 0) { rc = -3; break; }
        if (trace && phases <= trace_cap) {
            uint64_t* r = trace + 6 * (phases - 1);
            uint64_t mo = ORC_INF64;
            for (int k = 3; k >= 0; --k) if (crit & out_bits[k]) { mo = minOut[k]; break; }
            if (mo == ORC_INF64 && !(crit & (ORC_OUT_STATIC | ORC_OUT_SIMPLE | ORC_OUT_WEAK | ORC_OUT_FULL)))
                mo = minOutA;  /* APPROX alone: its OUT threshold */
            r[0] = nF; r[1] = nS; r[2] = minD; r[3] = mo; r[4] = 0; r[5] = crit;
        }
        /* Settle: move S' to S (before relaxing), check soundness. */
        for (uint64_t i = 0; i < nS; ++i) {
            uint32_t v = Sp[i];
            if (dist_ref && d_out[v] != dist_ref[v]) { rc = -4; goto done; }
            g.st[v] = ST_S;
            settle_phase[v] = (uint32_t)phases;
            degS += row_off[v + 1] - row_off[v];
        }
        if (trace && phases <= trace_cap) trace[6 * (phases - 1) + 4] = degS;
        settled += nS;
        relaxed += degS;
        /* Relax all out-edges of S'; newly reached vertices join F. */
        uint64_t nFresh = 0;
        for (uint64_t i = 0; i < nS; ++i) {
            uint32_t u = Sp[i];
            for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
                uint32_t t = col[e];
                if (g.st[t] == ST_S) continue;
                uint64_t cand = d_out[u] + w[e];
                if (cand < d_out[t]) {
                    d_out[t] = cand;
                    if (g.st[t] == ST_U) { g.st[t] = ST_F; Fn[nFn++] = t; fresh[nFresh++] = t; }
                }
            }
        }
        /* APPROX bookkeeping for the vertices that entered F (every phase, so
         * the values are right whatever the next phase's criterion is): static
         * start values first, then every edge between a new fringe vertex and a
         * fringe vertex lowers the fringe vertex's value. */
        for (uint64_t i = 0; i < nFresh; ++i) {
            ain[fresh[i]] = w64(g.in_st[fresh[i]]);
            aout[fresh[i]] = w64(g.out_st[fresh[i]]);
        }
        for (uint64_t i = 0; i < nFresh; ++i) {
            uint32_t x = fresh[i];
            for (uint64_t e = row_off[x]; e < row_off[x + 1]; ++e)
                if (g.st[col[e]] == ST_F && w[e] < ain[col[e]]) ain[col[e]] = w[e];
            for (uint64_t e = g.rro[x]; e < g.rro[x + 1]; ++e)
                if (g.st[g.rsrc[e]] == ST_F && g.rw[e] < aout[g.rsrc[e]]) aout[g.rsrc[e]] = g.rw[e];
        }
        uint32_t* tmp = F; F = Fn; Fn = tmp;
        nF = nFn;
    }
    stats[0] = phases; stats[1] = sumF; stats[2] = settled; stats[3] = relaxed;
done:
    free(g.rro); free(g.rsrc); free(g.rw); free(g.out_st); free(g.in_st); free(g.st);
    free(F); free(Fn); free(Sp); free(fill); free(ain); free(aout); free(fresh);
    return rc;
}

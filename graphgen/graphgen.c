/*
 * graphgen.c -- seeded synthetic graph generators (input recipes only).
 *
 * This module produces the CSR inputs that both the CPU oracle and the CUDA
 * solver consume.  It holds none of the shortest-path arithmetic: it only
 * draws random graphs and lays them out as a compressed sparse row (CSR)
 * structure grouped by source vertex (the adjacency-array layout of the
 * paper's Section 5).
 *
 * Random numbers: one SplitMix64 stream per graph (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the state
 * advances by the golden-ratio increment 0x9E3779B97F4A7C15 and each output is
 * the state passed through the published variant-13 finaliser.  Bounded
 * integers use Lemire's multiply-shift on the high 32 bits of a draw
 * (floor(hi32 * range / 2^32)).  Only integer arithmetic is used, so the same
 * seed gives the same graph on every machine.
 *
 * Families (the paper's inputs are uniform random graphs and Kronecker graphs,
 * Section 4; road networks stand in via grids):
 *   gg_gnm    directed G(n,m): m edges, endpoints uniform, self-loops redrawn,
 *             duplicate edges kept.
 *   gg_grid   R x C 4-neighbour grid, one weight per undirected edge used for
 *             both directions (the paper's road preprocessing doubles each
 *             undirected edge into two directed ones).
 *   gg_rmat   R-MAT edge sampling with quadrant probabilities (a,b,c,d), one
 *             32-bit draw per level, no noise, no vertex permutation,
 *             self-loops and duplicates kept.
 * Within a row the edges keep generation order (counting sort is stable).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s; } gg_rng;

static inline uint64_t gg_next(gg_rng* r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* floor(hi32(x) * range / 2^32): uniform-ish integer in [0, range). */
static inline uint32_t gg_bounded(uint64_t x, uint64_t range) {
    return (uint32_t)(((x >> 32) * range) >> 32);
}

/* Exposed so the Python side can check the stream against the published
 * reference outputs of SplitMix64. */
uint64_t gg_splitmix64_nth(uint64_t seed, uint64_t k) {
    gg_rng r = {seed};
    uint64_t v = 0;
    for (uint64_t i = 0; i <= k; ++i) v = gg_next(&r);
    return v;
}

/* Stable counting sort of (src,dst,w) triples into CSR. Returns 0 or -1. */
static int gg_to_csr(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                     const uint32_t* w, uint64_t* row_off, uint32_t* col, uint32_t* wout) {
    memset(row_off, 0, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < m; ++i) row_off[(size_t)src[i] + 1]++;
    for (uint32_t v = 0; v < n; ++v) row_off[v + 1] += row_off[v];
    uint64_t* fill = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    if (!fill) return -1;
    memcpy(fill, row_off, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t p = fill[src[i]]++;
        col[p] = dst[i];
        wout[p] = w[i];
    }
    free(fill);
    return 0;
}

int gg_gnm(uint32_t n, uint64_t m, uint32_t wlo, uint32_t whi, uint64_t seed,
           uint64_t* row_off, uint32_t* col, uint32_t* w) {
    if (n < 2 || whi <= wlo) return -1;
    uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* ww = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!src || !dst || !ww) { free(src); free(dst); free(ww); return -1; }
    gg_rng r = {seed};
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = gg_bounded(gg_next(&r), n);
        uint32_t b;
        do { b = gg_bounded(gg_next(&r), n); } while (b == a);
        src[i] = a;
        dst[i] = b;
        ww[i] = wlo + gg_bounded(gg_next(&r), (uint64_t)whi - wlo);
    }
    int rc = gg_to_csr(n, m, src, dst, ww, row_off, col, w);
    free(src); free(dst); free(ww);
    return rc;
}

uint64_t gg_grid_edges(uint32_t rows, uint32_t cols) {
    return 2ull * ((uint64_t)rows * (cols - 1) + (uint64_t)(rows - 1) * cols);
}

/* Vertex (r,c) has id r*cols + c.  Undirected edges are drawn in the order:
 * all horizontal edges (r,c)-(r,c+1) row by row, then all vertical edges
 * (r,c)-(r+1,c) row by row; each gets one weight.  Every vertex lists its
 * out-edges by increasing neighbour id. */
int gg_grid(uint32_t rows, uint32_t cols, uint32_t wlo, uint32_t whi, uint64_t seed,
            uint64_t* row_off, uint32_t* col, uint32_t* w) {
    if (rows < 1 || cols < 1 || whi <= wlo) return -1;
    uint64_t nh = (uint64_t)rows * (cols - 1), nv = (uint64_t)(rows - 1) * cols;
    uint32_t* wh = (uint32_t*)malloc(sizeof(uint32_t) * (nh ? nh : 1));
    uint32_t* wv = (uint32_t*)malloc(sizeof(uint32_t) * (nv ? nv : 1));
    if (!wh || !wv) { free(wh); free(wv); return -1; }
    gg_rng r = {seed};
    for (uint64_t i = 0; i < nh; ++i) wh[i] = wlo + gg_bounded(gg_next(&r), (uint64_t)whi - wlo);
    for (uint64_t i = 0; i < nv; ++i) wv[i] = wlo + gg_bounded(gg_next(&r), (uint64_t)whi - wlo);
    uint64_t p = 0;
    row_off[0] = 0;
    for (uint32_t rr = 0; rr < rows; ++rr) {
        for (uint32_t cc = 0; cc < cols; ++cc) {
            uint64_t id = (uint64_t)rr * cols + cc;
            if (rr > 0) { col[p] = (uint32_t)(id - cols); w[p] = wv[(uint64_t)(rr - 1) * cols + cc]; ++p; }
            if (cc > 0) { col[p] = (uint32_t)(id - 1); w[p] = wh[(uint64_t)rr * (cols - 1) + cc - 1]; ++p; }
            if (cc + 1 < cols) { col[p] = (uint32_t)(id + 1); w[p] = wh[(uint64_t)rr * (cols - 1) + cc]; ++p; }
            if (rr + 1 < rows) { col[p] = (uint32_t)(id + cols); w[p] = wv[(uint64_t)rr * cols + cc]; ++p; }
            row_off[id + 1] = p;
        }
    }
    free(wh); free(wv);
    return 0;
}

/* R-MAT: each edge descends `scale` levels of the 2x2 quadrant recursion.  At
 * every level one 32-bit uniform u is compared against the cumulative
 * thresholds ta <= tab <= tabc (probabilities scaled by 2^32):
 *   u < ta   -> (src bit 0, dst bit 0)
 *   u < tab  -> (0, 1)
 *   u < tabc -> (1, 0)
 *   else     -> (1, 1)
 * Bits are assigned from the most significant level down.  A 64-bit draw
 * supplies two levels (high half first).  One more draw gives the weight. */
int gg_rmat(uint32_t scale, uint64_t m, uint32_t ta, uint32_t tab, uint32_t tabc,
            uint32_t wlo, uint32_t whi, uint64_t seed,
            uint64_t* row_off, uint32_t* col, uint32_t* w) {
    if (scale < 1 || scale > 31 || whi <= wlo) return -1;
    uint32_t n = 1u << scale;
    uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* ww = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!src || !dst || !ww) { free(src); free(dst); free(ww); return -1; }
    gg_rng r = {seed};
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = 0, b = 0;
        uint64_t x = 0;
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            uint32_t u;
            if ((lvl & 1u) == 0) { x = gg_next(&r); u = (uint32_t)(x >> 32); }
            else u = (uint32_t)x;
            uint32_t bit = 1u << (scale - 1 - lvl);
            if (u < ta) { }
            else if (u < tab) b |= bit;
            else if (u < tabc) a |= bit;
            else { a |= bit; b |= bit; }
        }
        src[i] = a;
        dst[i] = b;
        ww[i] = wlo + gg_bounded(gg_next(&r), (uint64_t)whi - wlo);
    }
    int rc = gg_to_csr(n, m, src, dst, ww, row_off, col, w);
    free(src); free(dst); free(ww);
    return rc;
}

/* Fractional part of log2(x) for x in [2^L, 2^(L+1)), in Q32 (0 .. 2^32-1),
 * by the bit-by-bit squaring method: with y = x / 2^L in [1, 2) held in Q31,
 * each step squares y; a square >= 2 yields a 1 bit and is halved.  Integer
 * arithmetic with truncation only, so every host computes the same bits, and
 * the result never decreases as x grows. */
static uint32_t gg_log2_frac_q32(uint32_t x, uint32_t L) {
    uint64_t y = (uint64_t)x << (31 - L);  /* in [2^31, 2^32) */
    uint32_t f = 0;
    for (int i = 0; i < 32; ++i) {
        y = (y * y) >> 31;
        f <<= 1;
        if (y >= (1ull << 32)) { y >>= 1; f |= 1u; }
    }
    return f;
}

/* floor(2^t) for t = T / 2^32 (Q32, integer part 0..30): the largest x in
 * [2^L, 2^(L+1)) whose log2 fraction does not exceed that of t. */
static uint32_t gg_exp2_floor(uint64_t T) {
    const uint32_t L = (uint32_t)(T >> 32), f = (uint32_t)T;
    uint32_t lo = 1u << L, hi = (L < 31) ? (1u << (L + 1)) - 1 : 0xFFFFFFFFu;
    while (lo < hi) {  /* invariant: the answer lies in [lo, hi] */
        uint32_t mid = lo + (hi - lo + 1) / 2;
        if (gg_log2_frac_q32(mid, L) <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Parameters of the uneven batch: for graph g the caller receives n_g, m_g, its
 * seed and `sources_per_graph` source vertices.  n is log-uniform in
 * [2^lo_exp, 2^hi_exp): one 32-bit draw u gives t = lo_exp + (hi_exp - lo_exp)
 * * u / 2^32 in Q32 and n = floor(2^t) (integer fixed-point, above).  The
 * average out-degree is uniform in [deg_lo, deg_hi] (deg = deg_lo + (deg_hi -
 * deg_lo) * u' / 2^32 for a second draw u') and m = round(n * deg). */
int gg_batch_params(uint32_t count, uint32_t lo_exp, uint32_t hi_exp, uint32_t deg_lo,
                    uint32_t deg_hi, uint32_t sources_per_graph, uint64_t seed,
                    uint32_t* n_out, uint64_t* m_out, uint64_t* seed_out, uint32_t* src_out) {
    if (hi_exp <= lo_exp || hi_exp > 30 || deg_hi < deg_lo || deg_hi > 1024) return -1;
    gg_rng r = {seed};
    for (uint32_t g = 0; g < count; ++g) {
        const uint64_t u = gg_next(&r) >> 32;
        const uint64_t T = ((uint64_t)lo_exp << 32) + (uint64_t)(hi_exp - lo_exp) * u;
        const uint32_t n = gg_exp2_floor(T);
        const uint64_t v = gg_next(&r) >> 32;
        /* n * deg * 2^32 = n * (deg_lo * 2^32 + (deg_hi - deg_lo) * v) < 2^30 * 2^43 */
        const uint64_t deg_q32 = ((uint64_t)deg_lo << 32) + (uint64_t)(deg_hi - deg_lo) * v;
        const unsigned __int128 prod = (unsigned __int128)n * deg_q32;
        n_out[g] = n;
        m_out[g] = (uint64_t)((prod + (1ull << 31)) >> 32);
        seed_out[g] = seed + ((uint64_t)(g + 1) << 20);
        for (uint32_t k = 0; k < sources_per_graph; ++k)
            src_out[(size_t)g * sources_per_graph + k] = gg_bounded(gg_next(&r), n);
    }
    return 0;
}

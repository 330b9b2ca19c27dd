/*
 * sssp.h -- C ABI of the GB300 phase-parallel Dijkstra library.
 *
 * The library computes single-source shortest paths on a directed graph with
 * non-negative integer edge costs (Section 2 of Kainer & Traeff, "More
 * Parallelism in Dijkstra's Single-Source Shortest Path Algorithm",
 * arXiv:1903.12085) with the generic phased algorithm of Section 3: in every
 * phase, every fringe vertex that a correctness criterion proves final is
 * settled at once, and all of their out-edges are relaxed together.
 *
 * Conventions shared by every entry point
 *   - Vertices are 0..n-1.  Edge costs are uint32 and must be < 0xFFFFFFFF
 *     (that value is the "no edge" sentinel of the minima).  Distances are
 *     uint64; an unreachable vertex gets UINT64_MAX.  Limits: 1 <= n < 2^31,
 *     m < 2^32.  Self-loops and parallel edges are accepted; they take part
 *     in every minimum and never change a distance.
 *   - All arithmetic is exact unsigned integer: results do not depend on the
 *     order of relaxations, so distances and phase counts are unique.
 *   - Every call returns an sssp_status.  Nothing is thrown across the ABI.
 *     On failure, sssp_last_error() gives a message (thread-local).
 *   - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Unless stated otherwise a call returns after the work
 *     it queued on the stream has finished.
 *   - The library allocates device memory only inside sssp_graph_create,
 *     the first solve on a graph (its workspace) and sssp_batch_create; it
 *     frees it in the matching destroy call.
 *   - Solves on one graph handle share its workspace: do not run two solves
 *     on the same handle at the same time (use sssp_solve_batch instead).
 *   - Every call works on the CUDA device that is current on the calling
 *     thread.  The first solve on a device sets the solve kernels' launch
 *     attributes for that device, under a lock, so threads may make their
 *     first solves concurrently and a process may use several devices.
 *     Handles belong to the device they were created on.
 */
#ifndef SSSP_GB300_H
#define SSSP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SSSP_OK = 0,
  SSSP_ERR_INVALID_ARG = 1,   /* bad CSR, source >= n, reserved cost, bad mask */
  SSSP_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
  SSSP_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  SSSP_ERR_TIMEOUT = 4,       /* an in-kernel wait exceeded its time limit */
  SSSP_ERR_INTERNAL = 5,      /* a device-side consistency check failed */
  SSSP_ERR_UNSUPPORTED = 6    /* option not available (e.g. IN-SIMPLE without reverse CSR) */
} sssp_status;

/* Criterion mask: a phase settles every fringe vertex v satisfying ANY of
 * the criteria whose bits are set (a disjunction of sound criteria is sound,
 * and complete if one disjunct is, Section 3).  With
 * minD = min_{u in F} d[u] taken on the phase-start state:
 *   SSSP_IN_STATIC   d[v] <= minD + min_{(w,v) in E} c(w,v)             (eq. crit:instatic)
 *   SSSP_OUT_STATIC  d[v] <= min_{u in F} (d[u] + min_{(u,w) in E} c(u,w)) (eq. crit:outstatic)
 *   SSSP_IN_SIMPLE   as IN_STATIC, minimum over in-edges from unsettled w  (eq. crit:insimple)
 *   SSSP_OUT_SIMPLE  as OUT_STATIC, minimum over out-edges to unsettled w  (eq. crit:outsimple)
 *   SSSP_IN_FULL     d[v] <= minD + min over in-edges (w,v), w unsettled, of
 *                    c(w,v) for w in F and c(w,v) + min_{(x,w) in E} c(x,w)
 *                    for w unexplored (eq. crit:in, with Proposition 1's
 *                    precomputed minimum for unexplored w)
 *   SSSP_OUT_WEAK    d[v] <= min_{u in F} (d[u] + min over out-edges (u,w), w
 *                    unsettled, of c(u,w) for w in F and c(u,w) +
 *                    min_{(w,x) in E} c(w,x) for w unexplored) (eq. crit:outweak)
 *   SSSP_DIJK        the single fringe vertex of minimum d, lowest id on ties (Section 3)
 *   SSSP_APPROX      approximate IN (full) and OUT-WEAK minima (the closing
 *                    remark of Section 3), recomputed exactly in every k-th
 *                    phase (phases 1, k+1, ...; k from SSSP_APPROX_K(k), 1..63,
 *                    0 = 1); between recomputations a vertex entering F starts
 *                    from its static minima and lowers the values of its fringe
 *                    neighbours to the connecting edge's cost, and nothing else
 *                    changes them.  Every value lies between the static
 *                    minimum and the exact term, so the test
 *                    d[v] <= minD + inA(v) or d[v] <= min_{u in F}(d[u] + outA(u))
 *                    is sound and complete.
 * An empty minimum is infinite: the IN test then holds, and the vertex adds
 * nothing to the OUT threshold.  IN_SIMPLE, IN_FULL and APPROX need a graph
 * built with SSSP_GRAPH_REVERSE.  "IN+OUT" = SSSP_IN_STATIC | SSSP_OUT_STATIC is the
 * criterion of the paper's implementation (Section 5). */
enum {
  SSSP_IN_STATIC = 1u << 0,
  SSSP_OUT_STATIC = 1u << 1,
  SSSP_IN_SIMPLE = 1u << 2,
  SSSP_OUT_SIMPLE = 1u << 3,
  SSSP_IN_FULL = 1u << 4,
  SSSP_OUT_WEAK = 1u << 5,
  SSSP_DIJK = 1u << 6,
  SSSP_APPROX = 1u << 9,
  SSSP_APPROX_K_SHIFT = 10, /* bits 10..15: k of SSSP_APPROX */
  SSSP_CRITERIA_MASK = 0xFFFFu,
  /* Execution options (do not change results, only speed). */
  SSSP_POLICY_LEARNED = 1u << 16,  /* per-phase arm chosen by the loaded policy network (below) */
  SSSP_FRONTIER_DENSE = 1u << 17,  /* scan the vertex-status array instead of the queue */
  SSSP_FRONTIER_AUTO = 1u << 18    /* dense when |F| > n/8, else sparse */
};

/* Criterion mask of APPROX with recomputation period k (1..63). */
#define SSSP_APPROX_K(k) (SSSP_APPROX | (((uint32_t)(k) & 63u) << SSSP_APPROX_K_SHIFT))

/* sssp_graph_create build flags. */
enum { SSSP_GRAPH_REVERSE = 1u << 0 /* also build the in-edge CSR */ };

typedef struct sssp_graph sssp_graph;

/*
 * sssp_graph_create -- copy a CSR graph to the device and preprocess it.
 *   row_offsets  uint64[n+1], non-decreasing, row_offsets[0] = 0,
 *                row_offsets[n] = m; out-edges of u are [row_offsets[u],
 *                row_offsets[u+1]) (the adjacency array of Section 5)
 *   col_idx      uint32[m] edge targets, each < n
 *   weights      uint32[m] edge costs, each < 0xFFFFFFFF
 *   inputs_on_device  0: the three arrays are host memory; 1: device memory
 *                (read during the call only)
 * Preprocessing (Section 5 "Preprocessing" and Proposition 3): every out-row
 * is sorted by (cost, target); the static out-minimum of u is the cost of
 * its first edge; the static in-minimum of v is an atomic minimum over all
 * edges into v; with SSSP_GRAPH_REVERSE the in-edge CSR is built and its
 * rows sorted by (cost, source).  The caller keeps ownership of its arrays;
 * the handle owns its device copies.  Invalid input -> SSSP_ERR_INVALID_ARG
 * with nothing left allocated: the ends of host row_offsets are checked
 * before any allocation, everything else by one device pass over the copied
 * arrays (host and device inputs alike), after which the call frees what it
 * took.  *out is set only on success.
 */
sssp_status sssp_graph_create(uint32_t n, uint64_t m, const uint64_t* row_offsets,
                              const uint32_t* col_idx, const uint32_t* weights,
                              int inputs_on_device, uint32_t build_flags, void* stream,
                              sssp_graph** out);

/* Frees the handle and every device buffer it owns.  NULL is ignored. */
void sssp_graph_destroy(sssp_graph* g);

/* n, m and build flags of a handle (any pointer may be NULL). */
sssp_status sssp_graph_info(const sssp_graph* g, uint32_t* n, uint64_t* m, uint32_t* flags);

/* Device copies held by a handle, for callers that inspect the preprocessed
 * graph (any pointer may be NULL).  edges: uint32 pairs {target, cost} per
 * edge, rows sorted by (cost, target); out_min/in_min: uint32[n] static
 * minima (0xFFFFFFFF = no edge); rrow_off/redges: the in-edge CSR ({source,
 * cost} pairs) or NULL.  The pointers stay valid until sssp_graph_destroy. */
sssp_status sssp_graph_device_arrays(const sssp_graph* g, const uint64_t** row_off,
                                     const uint32_t** edges, const uint32_t** out_min,
                                     const uint32_t** in_min, const uint64_t** rrow_off,
                                     const uint32_t** redges);

/* Per-solve counters. */
typedef struct {
  uint64_t phases;         /* phases until F was empty (phase 1 settles the source) */
  uint64_t sum_frontier;   /* sum over phases of |F| at the start of the phase */
  uint64_t settled;        /* vertices settled (= vertices reachable from the source) */
  uint64_t edges_relaxed;  /* sum of out-degrees of settled vertices (each edge once) */
} sssp_stats;

/* One record per phase (sssp_solve_trace).  64 bytes, little-endian. */
typedef struct {
  uint32_t frontier;       /* |F| at phase start */
  uint32_t settled;        /* |S'| */
  uint64_t min_d;          /* minD */
  uint64_t min_out;        /* OUT threshold used (UINT64_MAX if none) */
  uint64_t deg_settled;    /* sum of out-degrees of S' */
  uint32_t criterion;      /* criterion mask applied in this phase */
  uint32_t arm;            /* bit 0: dense frontier; bit 1: phase ran on one block;
                              bit 2: near/far split active; bit 3: far part refilled
                              by a scan of all vertices (or split made) at phase
                              start; bit 4: bound raised from the far-vertex bucket
                              lists instead; bit 7: policy choice, bits 8..15: its
                              arm index */
  uint64_t t_start_ns;     /* device %globaltimer at phase start */
  uint64_t t_end_ns;       /* device %globaltimer at phase end */
  uint32_t queued;         /* fringe vertices in the scanned queue (|F| minus the
                              far part of a near/far split) */
  uint32_t select_ns;      /* from phase start to the end of the selection step
                              (the rest of the phase is the relaxation) */
} sssp_phase_record;

/*
 * sssp_solve -- one shortest-path solve from `source` (Sections 2-3).
 *   criterion   criterion mask plus execution options (see above); at least
 *               one criterion bit.
 *   dist_out    uint64[n], host or device memory (detected), caller-owned.
 *               Receives dist(source, v), UINT64_MAX if unreachable.
 *   phases_out  host uint64 (may be NULL): number of phases.
 * Synchronous.  The first call on a handle allocates its workspace.
 */
sssp_status sssp_solve(sssp_graph* g, uint32_t source, uint32_t criterion, uint64_t* dist_out,
                       uint64_t* phases_out, void* stream);

/*
 * sssp_solve_trace -- sssp_solve plus diagnostics (each output may be NULL):
 *   stats         host sssp_stats
 *   settle_phase  uint32[n], host or device: phase in which each vertex was
 *                 settled (0 = never) -- the per-phase settled sets S'
 *   trace         host array of trace_cap records; phases beyond trace_cap
 *                 are not recorded
 */
sssp_status sssp_solve_trace(sssp_graph* g, uint32_t source, uint32_t criterion,
                             uint64_t* dist_out, sssp_stats* stats, uint32_t* settle_phase,
                             sssp_phase_record* trace, uint64_t trace_cap, void* stream);

/*
 * sssp_solve_batch -- `count` independent solves in one persistent launch:
 * solve i runs on graphs[i] from sources[i] (graphs may repeat).  Blocks of
 * the launch pull solves from a device work queue, largest graph first.
 *   dist_out[i]  uint64[n_i] device memory
 *   phases_out   uint64[count], host or device (detected); may be NULL
 * Synchronous.  Workspaces are allocated per call; for repeated batches use
 * sssp_batch_create / sssp_batch_launch.
 */
sssp_status sssp_solve_batch(sssp_graph* const* graphs, const uint32_t* sources, uint32_t count,
                             uint32_t criterion, uint64_t* const* dist_out, uint64_t* phases_out,
                             void* stream);

/* A prepared batch: descriptors and workspaces allocated once, the launch
 * captured in a CUDA graph.  sssp_batch_launch replays it on `stream`
 * (stream-ordered, returns immediately); outputs are the device buffers given
 * at creation.  phases_out must be device memory here.  With
 * SSSP_POLICY_LEARNED the batch copies the policy network loaded at creation
 * and uses that copy in every launch (loading or clearing a network later does
 * not affect it); its graphs need SSSP_GRAPH_REVERSE for the IN-SIMPLE arms. */
typedef struct sssp_batch sssp_batch;
sssp_status sssp_batch_create(sssp_graph* const* graphs, const uint32_t* sources, uint32_t count,
                              uint32_t criterion, uint64_t* const* dist_out, uint64_t* phases_out,
                              void* stream, sssp_batch** out);
sssp_status sssp_batch_launch(sssp_batch* b, void* stream);
void sssp_batch_destroy(sssp_batch* b);

/* Diagnostics for solve i (caller order) of a prepared batch: every later
 * launch writes its per-phase records (trace_cap of them) to `trace` and the
 * phase in which each vertex settled (0 = never) to `settle_phase`, both
 * device memory owned by the caller (NULL stops that output).  The records are
 * those of sssp_solve_trace; with SSSP_POLICY_LEARNED they give the arm each
 * phase ran with, so the schedule of a batched solve can be replayed.  Call it
 * when no launch of the batch is in flight; synchronous on `stream`.  A
 * library feature with no counterpart in the paper. */
sssp_status sssp_batch_trace(sssp_batch* b, uint32_t i, sssp_phase_record* trace, uint64_t trace_cap,
                             uint32_t* settle_phase, void* stream);

/* Autotuner of a prepared batch: picks the number of blocks per solve from
 * the ladder 1, 2, 4, ..., all co-resident blocks (plus the batch's own
 * choice).  It times the batch's own choice, then walks up and then down the
 * ladder from it; every candidate runs once to warm up and three times timed
 * with CUDA events on `stream` (scored by the median), and a walk stops at the
 * first candidate more than 10 % slower than the best so far, or whose warm-up
 * alone took 1.5 times the best median (it gets no timed runs).  Another
 * candidate must beat the batch's own choice by 3 %.  The CUDA graph is
 * re-captured with the winner.  Results never depend on the choice (the
 * outputs hold the last run's, identical to any other run's).  bpg_out and
 * ms_out (either may be NULL) get the chosen value and its launch time.
 * Synchronous.  A library feature with no counterpart in the paper. */
sssp_status sssp_batch_autotune(sssp_batch* b, void* stream, uint32_t* bpg_out, float* ms_out);

/* ---- per-phase policy network ------------------------------------------
 * With SSSP_POLICY_LEARNED (criterion bits must be IN_STATIC | OUT_STATIC, the
 * fallback arm) every phase of a single or batched solve picks one of four arms:
 *   0: IN-STATIC | OUT-STATIC, sparse queue   1: the same, dense scan
 *   2: IN-SIMPLE | OUT-STATIC, sparse queue   3: the same, dense scan
 * with a small MLP over 8 phase-start features (IN-SIMPLE arms need a graph
 * built with SSSP_GRAPH_REVERSE).  Every arm is sound and complete (Section 3),
 * so distances never depend on the policy; phase counts do, and
 * sssp_solve_trace reports each phase's criterion and arm
 * (arm field: bit 0 dense, bit 1 single-block, bit 7 policy, bits 8..15 index).
 * Network: W1[8][32] b1[32] W2[32][32] b2[32] W3[32][4] b3[4] (float32,
 * input index first, ReLU after both hidden layers); outputs are predicted
 * log2(phase time / settled vertices) per arm; the smallest one wins if it
 * is below arm 0's by a margin of 0.35, else arm 0 runs; the dense arms take
 * part only while |F| >= n/32.  While the fringe is
 * split into near and far parts (sssp_tuning's nearfar fields) every phase
 * runs arm 0, whose sparse queue is then the near part.
 * Features (sssp_policy_features computes them on the host):
 *   log2(1+|F|)/24, |F|/n, log2(1+E')/24, log2(1+S')/24, log2(1+k)/16,
 *   log2(n)/32, (m/n)/32, S'/(1+F')
 * with E', S', F' the relaxed edges, settled vertices and fringe size of the
 * previous phase and k the phase index. */
#define SSSP_POLICY_FEATURES 8
#define SSSP_POLICY_ARMS 4
#define SSSP_POLICY_WEIGHTS 1476

/* Load the network (host or device float32[SSSP_POLICY_WEIGHTS]) for the
 * current device; it is used by solves made after the call.  The library
 * keeps its own device copy until sssp_policy_clear. */
sssp_status sssp_policy_load(const float* weights, size_t count);
sssp_status sssp_policy_clear(void);

/* The 8 features of a phase (host function, same formula as the device). */
sssp_status sssp_policy_features(uint64_t frontier, uint64_t n, uint64_t m, uint64_t phase,
                                 uint64_t edges_prev, uint64_t settled_prev, uint64_t frontier_prev,
                                 float* out8);

/* FP32 training kernels (all pointers device memory, stream-ordered):
 *   sssp_mlp_forward   y[b][0..3] = network(x[b][0..7]) for b < batch
 *   sssp_mlp_backward  grad[SSSP_POLICY_WEIGHTS] = d loss / d w and *loss =
 *                      (1/B) sum_b (y_b[arm[b]] - target[b])^2 (loss may be
 *                      NULL); fixed summation order (deterministic)
 *   sssp_mlp_adam      one Adam step (bias-corrected with `step` >= 1) */
sssp_status sssp_mlp_forward(const float* w, const float* x, uint32_t batch, float* y, void* stream);
sssp_status sssp_mlp_backward(const float* w, const float* x, const float* target, const uint32_t* arm,
                              uint32_t batch, float* grad, float* loss, void* stream);
sssp_status sssp_mlp_adam(float* w, const float* grad, float* m1, float* m2, uint32_t count, float lr,
                          float beta1, float beta2, float eps, uint32_t step, void* stream);

/* Largest n accepted by sssp_solve_noalloc. */
#define SSSP_NOALLOC_MAX_VERTICES (1u << 19)

/*
 * sssp_solve_noalloc -- a solve that allocates nothing (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory at
 * solve time, e.g. an application whose allocator has reserved the whole
 * device up front, or a latency-critical service that cannot take the
 * implicit device synchronisation of cudaMalloc/cudaFree in its request path).
 *   row_offsets  uint64[n+1] device memory (as in sssp_graph_create)
 *   edges        uint32 pairs {target, cost}, 2*m words, device memory; rows
 *                need not be sorted
 *   (row_offsets, edges and dist_out must start on an 8-byte boundary:
 *   anything else is rejected with SSSP_ERR_INVALID_ARG before any CUDA call)
 *   criterion    SSSP_IN_STATIC, SSSP_OUT_STATIC and/or SSSP_DIJK (plus the
 *                frontier options); other criteria -> SSSP_ERR_UNSUPPORTED
 *   dist_out     uint64[n] device memory, receives the distances
 *   phases_out   host uint64 (may be NULL)
 * n must be in [1, SSSP_NOALLOC_MAX_VERTICES]; larger graphs are rejected with
 * SSSP_ERR_INVALID_ARG.  All scratch (status, queues, relax list, distance
 * records, static minima, row starts and degrees, control block: 57 bytes per
 * vertex of the maximum, about 28.5 MiB in all) is one file-scope __device__
 * array that every GPU loading the library
 * holds until the process exits.  The call makes no cudaMalloc/cudaFree or
 * other allocating call.  Its first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and the co-resident block count; make
 * that first call before any stream capture.  Every call reuses the same
 * array: it clears the control block itself, and calls that overlap on the
 * GPU (two streams, two host threads) race on the array.  Synchronous.
 */
sssp_status sssp_solve_noalloc(uint32_t n, uint64_t m, const uint64_t* row_offsets,
                               const uint32_t* edges, uint32_t source, uint32_t criterion,
                               uint64_t* dist_out, uint64_t* phases_out, void* stream);

/* Execution tuning (results never depend on it).  solo_max_frontier: a
 * phase whose fringe has at most this many vertices (and at most 2048) runs on
 * a single block with its queues in shared memory (0 = never); if its relax
 * list then has more than solo_max_edges edges, the relax step is handed to
 * all blocks of the solve;
 * batch_blocks_per_solve: blocks that cooperate on one solve of a batch (0 =
 * chosen from the batch); grid_blocks: blocks of a single solve (0 = chosen
 * from n, capped at the co-resident maximum);
 * nearfar_min_frontier: with static criteria only (IN-STATIC and/or
 * OUT-STATIC) and n <= 2^30, a fringe of at least this many vertices per
 * block working on the solve (all blocks of a single solve, the group of a
 * batched one) is split into a near part, kept in the queue that every phase
 * scans, and a far part of vertices that no phase can settle before a bound B
 * on d(v) - inmin(v) is raised (0 = never split);
 * nearfar_target: vertices the near part is sized to when B is set or raised
 * (0 = four times the settled count of the last phase, at least 8192; by
 * sssp_solve_noalloc, which keeps no bucket lists, chosen from n and that
 * count); far vertices are listed in buckets of d(v) - inmin(v), so raising B
 * usually reads just the passed buckets' lists, and all n vertex records only
 * when B passes the listed range;
 * nearfar_min_share: the split also needs a fringe of at least this many
 * 256ths of n (0 = no such condition).
 * Applies to launches made after the call; sssp_set_tuning(NULL) restores the
 * defaults (2048, 0, 0, 2048, 8192, 0, 8). */
typedef struct {
  uint32_t solo_max_frontier;
  uint32_t batch_blocks_per_solve;
  uint32_t grid_blocks;
  uint32_t solo_max_edges;
  uint32_t nearfar_min_frontier;
  uint32_t nearfar_target;
  uint32_t nearfar_min_share;
  uint32_t reserved;
} sssp_tuning;
sssp_status sssp_set_tuning(const sssp_tuning* t);
sssp_status sssp_get_tuning(sssp_tuning* t);

/* Device memory the library holds, and an optional cap on it (a library
 * feature with no counterpart in the paper).  Every device allocation of the
 * library (graph handles, solve workspaces, batches, the policy network and
 * the temporaries of preprocessing and training) is counted, over all devices
 * of the process.  With a cap (bytes > 0) a request that would take the total
 * above it fails with SSSP_ERR_OUT_OF_MEMORY before cudaMalloc is called, and
 * the failing call frees everything it had taken, exactly as for a failed
 * cudaMalloc; 0 removes the cap (the default).  sssp_solve_noalloc allocates
 * nothing and is not affected.  Applies to calls made after it. */
sssp_status sssp_set_device_memory_limit(uint64_t bytes);
sssp_status sssp_device_memory_in_use(uint64_t* bytes);

/* Upper bound, in nanoseconds, on any single in-kernel wait (grid barrier,
 * work queue).  A wait that runs out sets SSSP_ERR_TIMEOUT and the kernel
 * returns.  Default 2e9.  Applies to launches made after the call. */
sssp_status sssp_set_wait_limit_ns(uint64_t ns);

/* Largest L2 fetch on a DRAM miss, in bytes (32, 64 or 128), for the CUDA
 * context of the current device: cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity).
 * The solves gather 16-byte vertex records at random, so a fetch larger than
 * a 32-byte sector mostly moves bytes nobody reads; the setting lasts until
 * the process exits or it is set again and applies to all work of the
 * context, which is why the library never changes it by itself.  A library
 * feature with no counterpart in the paper. */
sssp_status sssp_set_l2_fetch_granularity(uint32_t bytes);

/* Self-test of the bounded in-kernel wait that every grid barrier uses: one
 * thread waits on a device word that nothing writes, so the wait must run out
 * after limit_ns.  Returns SSSP_ERR_TIMEOUT (the expected outcome) and leaves
 * the CUDA context usable.  Allocates and frees two words of device memory. */
sssp_status sssp_selftest_wait(uint64_t limit_ns);

/* Message of the last failed call on this thread ("" if none). */
const char* sssp_last_error(void);

/* Library version string. */
const char* sssp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SSSP_GB300_H */

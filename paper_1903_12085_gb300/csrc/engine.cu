// engine.cu -- the phase engine of the generic phased SSSP algorithm (Section 3).
//
// One persistent launch runs a whole solve.  Every phase is three steps
// separated by group barriers (a bounded grid barrier for a single solve, the
// block barrier for the batched solver):
//
//   A  thresholds   minD   = min_{u in F} d[u]
//                   minOut = min_{u in F} d[u] + outmin(u)          (OUT criteria)
//                   warp shuffle -> block -> one 64-bit atomicMin per block.
//                   For the dynamic (SIMPLE) criteria the per-vertex cursors into
//                   the cost-sorted rows are first advanced past settled endpoints
//                   (Proposition 3: the minimum over the remaining edges is the
//                   first live element of the presorted list).
//   B  select       v in F is settled iff
//                     IN : d[v] <= minD + inmin(v)   (inmin empty -> holds)
//                     OUT: d[v] <= minOut
//                   (eqs. crit:instatic / crit:insimple / crit:outstatic /
//                   crit:outsimple), all against the phase-start state.  Settled
//                   vertices are marked S before any relaxation; those with
//                   out-edges go to the relax list with an exclusive prefix of
//                   their degrees (one packed 64-bit atomicAdd per warp reserves
//                   both the slots and the edge range, so the prefix is monotone);
//                   the rest of F is compacted into the next queue.
//   C  relax        edge-balanced over the relax list: each block takes a tile of
//                   consecutive edges, finds the owning settled vertices by binary
//                   search, and for every edge (u,t) with t not in S does
//                   cand = d[u] + c(u,t); if cand < d[t]: atomicMin(d[t], cand); a
//                   vertex whose old value was infinite moves U -> F (appended).
//
// Phase control: the phase that settles the source is phase 1; the loop ends
// when the next queue is empty.  The frontier is either the compacted queue
// (sparse) or a scan of the status array (dense); both keep the queue exact.
#include <algorithm>
#include <cstring>
#include <vector>

#include "engine.h"
#include "internal.h"

namespace sssp {

struct GridGroup {
  GridBarrier* bar;
  int* err;
  unsigned long long limit;
  __device__ unsigned int rank() const { return blockIdx.x; }
  __device__ unsigned int size() const { return gridDim.x; }
  __device__ bool sync() const { return grid_sync(bar, gridDim.x, limit, err); }
};

struct BlockGroup {
  __device__ unsigned int rank() const { return 0; }
  __device__ unsigned int size() const { return 1; }
  __device__ bool sync() const {
    __syncthreads();
    return true;
  }
};

// Number of elements <= x in the strictly increasing array a[0..len), by one
// warp (31 pivots per round).  All 32 lanes must call it; every lane gets the result.
__device__ __forceinline__ uint32_t warp_upper_bound(const uint32_t* a, uint32_t len, uint32_t x) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = len;
  while (hi - lo > 32) {
    const uint32_t span = hi - lo;
    const uint32_t p = lo + (uint32_t)(((uint64_t)span * (uint32_t)(lane + 1)) >> 5);
    const bool le = lane < 31 && ldcg_u32(a + p) <= x;
    const unsigned int mask = __ballot_sync(0xFFFFFFFFu, le);
    const int c = __popc(mask);
    const uint32_t plo = __shfl_sync(0xFFFFFFFFu, p, c > 0 ? c - 1 : 0);
    const uint32_t phi = __shfl_sync(0xFFFFFFFFu, p, c < 31 ? c : 0);
    if (c > 0) lo = plo + 1;
    if (c < 31) hi = phi;
  }
  const bool le = lo + lane < hi && ldcg_u32(a + lo + lane) <= x;
  return lo + __popc(__ballot_sync(0xFFFFFFFFu, le));
}

// Advance the out-cursor of v past targets in S; return the dynamic out-minimum.
__device__ __forceinline__ uint32_t out_min_dynamic(const GraphView& g, const SolveWS& w, uint32_t v) {
  const uint32_t c0 = ldcg_u32(&w.cur_out[v]);
  const uint32_t end = (uint32_t)__ldg(&g.row_off[v + 1]);
  uint32_t c = c0;
  uint32_t cost = kInf32;
  while (c < end) {
    const uint2 e = __ldg(&g.edges[c]);
    if (ldcg_u8(&w.status[e.x]) != kS) { cost = e.y; break; }
    ++c;
  }
  if (c != c0) w.cur_out[v] = c;
  return cost;
}

// Advance the in-cursor of v past sources in S (result read back in step B).
__device__ __forceinline__ void in_cursor_advance(const GraphView& g, const SolveWS& w, uint32_t v) {
  const uint32_t c0 = ldcg_u32(&w.cur_in[v]);
  const uint32_t end = (uint32_t)__ldg(&g.rrow_off[v + 1]);
  uint32_t c = c0;
  while (c < end && ldcg_u8(&w.status[__ldg(&g.redges[c]).x]) == kS) ++c;
  if (c != c0) w.cur_in[v] = c;
}

__device__ __forceinline__ uint32_t in_min_dynamic(const GraphView& g, const SolveWS& w, uint32_t v) {
  const uint32_t c = ldcg_u32(&w.cur_in[v]);
  return c < (uint32_t)__ldg(&g.rrow_off[v + 1]) ? __ldg(&g.redges[c]).y : kInf32;
}

template <class G>
__device__ void solve_body(const SolveParams& p, const G& grp, unsigned char* smem) {
  const GraphView& g = p.g;
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x;
  const unsigned int lane = tid & 31, warp = tid >> 5;
  const uint64_t grank = grp.rank(), gsize = grp.size();
  const uint64_t gthreads = gsize * nthr;
  const uint64_t gtid = grank * nthr + tid;
  const bool leader = grank == 0 && tid == 0;

  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* s_base = reinterpret_cast<uint32_t*>(smem + 64 * sizeof(unsigned long long));
  unsigned long long* s_row = reinterpret_cast<unsigned long long*>(s_base + kTile);
  unsigned long long* s_d = s_row + kTile;
  uint32_t* s_range = reinterpret_cast<uint32_t*>(s_d + kTile);

  const uint32_t crit = p.crit;
  const bool in_dyn = (crit & SSSP_IN_SIMPLE) != 0;
  const bool in_st = !in_dyn && (crit & SSSP_IN_STATIC) != 0;
  const bool use_in = in_dyn || in_st;
  const bool out_dyn = (crit & SSSP_OUT_SIMPLE) != 0;
  const bool use_out = out_dyn || (crit & SSSP_OUT_STATIC) != 0;
  const bool dijk = (crit & SSSP_DIJK) != 0;

  // ---- initialisation: d = inf, all vertices unexplored, cursors at row starts
  for (uint64_t v = gtid; v < n; v += gthreads) {
    w.d[v] = kInf64;
    w.status[v] = kU;
    if (w.cur_out) w.cur_out[v] = (uint32_t)g.row_off[v];
    if (w.cur_in) w.cur_in[v] = (uint32_t)g.rrow_off[v];
    if (w.settle_phase) w.settle_phase[v] = 0;
  }
  if (leader) {
    ctl->min_d[0] = ctl->min_d[1] = kInf64;
    ctl->min_out[0] = ctl->min_out[1] = kInf64;
    ctl->argmin[0] = ctl->argmin[1] = kInf32;
    ctl->qcount[0] = 1;
    ctl->qcount[1] = 0;
    ctl->phases = ctl->sum_f = ctl->settled = ctl->relaxed = 0;
  }
  if (!grp.sync()) return;
  if (leader) {
    w.d[p.source] = 0;
    w.status[p.source] = kF;
    w.q[0][0] = p.source;
  }
  if (!grp.sync()) return;

  uint64_t phase = 1;
  for (;; ++phase) {
    const int cur = (int)((phase - 1) & 1), nxt = cur ^ 1;
    const uint32_t nF = ldcg_u32(&ctl->qcount[cur]);
    if (nF == 0) break;
    const bool dense = (crit & SSSP_FRONTIER_DENSE) || ((crit & SSSP_FRONTIER_AUTO) && nF > (n >> 3));
    const uint32_t* Q = w.q[cur];
    uint32_t* Qn = w.q[nxt];
    unsigned long long t0 = 0;
    if (leader) {
      t0 = globaltimer_ns();
      ctl->qcount[nxt] = 0;
      ctl->relax_packed = 0;
      ctl->settled_now = 0;
      ctl->min_d[nxt] = kInf64;
      ctl->min_out[nxt] = kInf64;
      ctl->argmin[nxt] = kInf32;
      ctl->sum_f += nF;
    }

    // ---- A: thresholds over the phase-start state
    {
      unsigned long long lmin_d = kInf64, lmin_out = kInf64;
      auto visit = [&](uint32_t v) {
        const unsigned long long dv = ldcg_u64(&w.d[v]);
        lmin_d = dv < lmin_d ? dv : lmin_d;
        if (use_out) {
          const uint32_t om = out_dyn ? out_min_dynamic(g, w, v) : __ldg(&g.out_min[v]);
          if (om != kInf32) {
            const unsigned long long k = dv + om;
            lmin_out = k < lmin_out ? k : lmin_out;
          }
        }
        if (in_dyn) in_cursor_advance(g, w, v);
      };
      if (dense) {
        for (uint64_t v = gtid; v < n; v += gthreads)
          if (ldcg_u8(&w.status[v]) == kF) visit((uint32_t)v);
      } else {
        for (uint64_t i = gtid; i < nF; i += gthreads) visit(ldcg_u32(&Q[i]));
      }
      block_min2_to_global(lmin_d, lmin_out, &ctl->min_d[cur], use_out ? &ctl->min_out[cur] : nullptr, red);
    }
    if (!grp.sync()) return;
    const unsigned long long minD = ldcg_u64(&ctl->min_d[cur]);
    const unsigned long long minOut = use_out ? ldcg_u64(&ctl->min_out[cur]) : 0;

    uint32_t amin = kInf32;
    if (dijk) {  // DIJK: the lowest id among vertices of minimum d
      uint32_t lid = kInf32;
      if (dense) {
        for (uint64_t v = gtid; v < n; v += gthreads)
          if (ldcg_u8(&w.status[v]) == kF && ldcg_u64(&w.d[v]) == minD) lid = min(lid, (uint32_t)v);
      } else {
        for (uint64_t i = gtid; i < nF; i += gthreads) {
          const uint32_t v = ldcg_u32(&Q[i]);
          if (ldcg_u64(&w.d[v]) == minD) lid = min(lid, v);
        }
      }
      lid = __reduce_min_sync(0xFFFFFFFFu, lid);
      if (lane == 0 && lid != kInf32) atomicMin(&ctl->argmin[cur], lid);
      if (!grp.sync()) return;
      amin = ldcg_u32(&ctl->argmin[cur]);
    }

    // ---- B: select S', mark settled, build relax list, compact the rest of F
    {
      const uint64_t total = dense ? n : nF;
      uint32_t settled_here = 0;
      for (uint64_t base = gtid & ~31ull; base < total; base += gthreads) {
        const uint64_t i = base + lane;
        bool valid = i < total;
        uint32_t v = 0;
        if (valid) {
          v = dense ? (uint32_t)i : ldcg_u32(&Q[i]);
          if (dense) valid = ldcg_u8(&w.status[v]) == kF;
        }
        bool sel = false;
        uint32_t deg = 0;
        if (valid) {
          const unsigned long long dv = ldcg_u64(&w.d[v]);
          if (use_in) {
            const uint32_t im = in_dyn ? in_min_dynamic(g, w, v) : __ldg(&g.in_min[v]);
            sel = (im == kInf32) || dv <= minD + im;
          }
          if (!sel && use_out) sel = dv <= minOut;
          if (!sel && dijk) sel = (v == amin);
          if (sel) {
            w.status[v] = kS;
            if (w.settle_phase) w.settle_phase[v] = (uint32_t)phase;
            deg = (uint32_t)(__ldg(&g.row_off[v + 1]) - __ldg(&g.row_off[v]));
          }
        }
        // relax list (settled vertices with out-edges): slots and edge range in one atomic
        const bool rl = sel && deg > 0;
        const unsigned int rmask = __ballot_sync(0xFFFFFFFFu, rl);
        if (rmask) {
          const uint32_t c = rl ? deg : 0;
          const uint32_t incl = warp_inclusive_scan(c);
          const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
          unsigned long long old = 0;
          if (lane == 0) old = atomicAdd(&ctl->relax_packed, ((unsigned long long)__popc(rmask) << 32) | tot);
          old = __shfl_sync(0xFFFFFFFFu, old, 0);
          if (rl) {
            const uint32_t slot = (uint32_t)(old >> 32) + __popc(rmask & ((1u << lane) - 1u));
            if (slot < n) {
              w.sp_v[slot] = v;
              w.sp_base[slot] = (uint32_t)old + incl - c;
            } else {
              atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
            }
          }
        }
        warp_append(Qn, &ctl->qcount[nxt], valid && !sel, v, n, &ctl->err);
        settled_here += __popc(__ballot_sync(0xFFFFFFFFu, sel));
      }
      if (lane == 0 && settled_here) atomicAdd(&ctl->settled_now, settled_here);
    }
    if (!grp.sync()) return;

    // ---- C: relax every out-edge of S' (edge-balanced tiles)
    const unsigned long long packed = ldcg_u64(&ctl->relax_packed);
    const uint32_t nS = (uint32_t)(packed >> 32);
    const uint32_t E = (uint32_t)packed;
    for (uint64_t tile = grank; tile * kTile < E; tile += gsize) {
      const uint32_t e0 = (uint32_t)(tile * kTile);
      const uint32_t e1 = (uint64_t)e0 + kTile < E ? e0 + kTile : E;
      if (warp == 0) {
        uint32_t lo = 0, hi = nS - 1;
        if (!(e0 == 0 && e1 == E)) {
          lo = warp_upper_bound(w.sp_base, nS, e0) - 1;
          hi = warp_upper_bound(w.sp_base, nS, e1 - 1) - 1;
        }
        if (lane == 0) { s_range[0] = lo; s_range[1] = hi; }
      }
      __syncthreads();
      const uint32_t lo = s_range[0], cnt = s_range[1] - s_range[0] + 1;
      for (uint32_t k = tid; k < cnt; k += nthr) {
        const uint32_t v = ldcg_u32(&w.sp_v[lo + k]);
        s_base[k] = ldcg_u32(&w.sp_base[lo + k]);
        s_row[k] = __ldg(&g.row_off[v]);
        s_d[k] = ldcg_u64(&w.d[v]);
      }
      __syncthreads();
      for (uint32_t eb = e0 + warp * 32; eb < e1; eb += nthr) {
        const uint32_t e = eb + lane;
        bool fresh = false;
        uint32_t t = 0;
        if (e < e1) {
          uint32_t a = 0, b = cnt;  // owner = last k with s_base[k] <= e
          while (b - a > 1) {
            const uint32_t mid = (a + b) >> 1;
            if (s_base[mid] <= e) a = mid; else b = mid;
          }
          const uint2 ed = __ldg(&g.edges[s_row[a] + (e - s_base[a])]);
          t = ed.x;
          if (ldcg_u8(&w.status[t]) != kS) {
            const unsigned long long cand = s_d[a] + ed.y;
            if (cand < ldcg_u64(&w.d[t])) {
              const unsigned long long old = atomicMin(&w.d[t], cand);
              if (old == kInf64) {
                w.status[t] = kF;
                fresh = true;
              }
            }
          }
        }
        warp_append(Qn, &ctl->qcount[nxt], fresh, t, n, &ctl->err);
      }
      __syncthreads();
    }
    if (leader) {
      ctl->relaxed += E;
      ctl->settled += ctl->settled_now;
    }
    if (!grp.sync()) return;
    if (leader && w.trace && phase <= w.trace_cap) {
      sssp_phase_record r;
      r.frontier = nF;
      r.settled = ldcg_u32(&ctl->settled_now);
      r.min_d = minD;
      r.min_out = use_out ? minOut : kInf64;
      r.deg_settled = E;
      r.criterion = crit & SSSP_CRITERIA_MASK;
      r.arm = dense ? 1u : 0u;
      r.t_start_ns = t0;
      r.t_end_ns = globaltimer_ns();
      r.reserved = 0;
      w.trace[phase - 1] = r;
    }
  }
  if (leader) {
    ctl->phases = phase - 1;
    __threadfence();
    ctl->done = 1;
  }
}

__global__ void __launch_bounds__(kThreads) k_solve_grid(SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  GridGroup grp{&p.ws.ctl->bar, &p.ws.ctl->err, p.wait_ns};
  solve_body(p, grp, smem);
}

// Batched solver: each block runs whole solves, pulling the next one from a
// device counter (descriptors sorted largest first by the host).
struct BatchItem {
  GraphView g;
  SolveWS ws;
  uint32_t source;
  uint32_t out_index;  // position of this solve in the caller's arrays
};

__global__ void __launch_bounds__(kThreads) k_solve_batch(const BatchItem* items, uint32_t count,
                                                           unsigned int* next, uint32_t crit,
                                                           unsigned long long* phases_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= count) break;
    SolveParams p;
    p.g = items[it].g;
    p.ws = items[it].ws;
    p.source = items[it].source;
    p.crit = crit;
    p.wait_ns = 0;
    solve_body(p, BlockGroup{}, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (p.ws.ctl->err != 0) atomicCAS(&items[0].ws.ctl->err, 0, p.ws.ctl->err);
      if (phases_out) phases_out[items[it].out_index] = p.ws.ctl->phases;
    }
  }
}

// ---------------------------------------------------------------------------
// host side

namespace {

int g_blocks_per_sm = 0;

sssp_status ensure_kernel_attrs() {
  static bool done = false;
  if (done) return SSSP_OK;
  SSSP_CUDA_TRY(cudaFuncSetAttribute(k_solve_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  SSSP_CUDA_TRY(cudaFuncSetAttribute(k_solve_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  SSSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_blocks_per_sm, k_solve_grid, kThreads, kSmemBytes));
  if (g_blocks_per_sm < 1) return fail(SSSP_ERR_CUDA, "solve kernel cannot be resident");
  done = true;
  return SSSP_OK;
}

sssp_status check_crit(const sssp_graph* g, uint32_t crit) {
  const uint32_t known = SSSP_IN_STATIC | SSSP_OUT_STATIC | SSSP_IN_SIMPLE | SSSP_OUT_SIMPLE | SSSP_DIJK |
                         SSSP_POLICY_LEARNED | SSSP_FRONTIER_DENSE | SSSP_FRONTIER_AUTO;
  if ((crit & SSSP_CRITERIA_MASK) == 0) return fail(SSSP_ERR_INVALID_ARG, "criterion mask has no criterion bit");
  if (crit & ~known) return fail(SSSP_ERR_INVALID_ARG, "unknown criterion bits 0x%x", crit & ~known);
  if ((crit & SSSP_IN_SIMPLE) && !g->rrow_off)
    return fail(SSSP_ERR_UNSUPPORTED, "IN-SIMPLE needs a graph built with SSSP_GRAPH_REVERSE");
  return SSSP_OK;
}

template <class T>
sssp_status dev_alloc(T** p, size_t count) {
  SSSP_CUDA_TRY(cudaMalloc(p, std::max<size_t>(count, 1) * sizeof(T)));
  return SSSP_OK;
}

}  // namespace

void workspace_free(Workspace* ws) {
  if (!ws) return;
  cudaFree(ws->d);
  cudaFree(ws->status);
  cudaFree(ws->q0);
  cudaFree(ws->q1);
  cudaFree(ws->sp_v);
  cudaFree(ws->sp_base);
  cudaFree(ws->cur_out);
  cudaFree(ws->cur_in);
  cudaFree(ws->ctl);
  cudaFreeHost(ws->ctl_host);
  delete ws;
}

sssp_status workspace_alloc(uint32_t n, bool want_cursors, Workspace** out) {
  Workspace* ws = new (std::nothrow) Workspace();
  if (!ws) return fail(SSSP_ERR_OUT_OF_MEMORY, "host allocation failed");
  ws->n = n;
  sssp_status s = SSSP_OK;
  if ((s = dev_alloc(&ws->d, n)) || (s = dev_alloc(&ws->status, n)) || (s = dev_alloc(&ws->q0, n)) ||
      (s = dev_alloc(&ws->q1, n)) || (s = dev_alloc(&ws->sp_v, n)) || (s = dev_alloc(&ws->sp_base, n)) ||
      (s = dev_alloc(&ws->ctl, 1))) {
    workspace_free(ws);
    return s;
  }
  if (want_cursors && ((s = dev_alloc(&ws->cur_out, n)) || (s = dev_alloc(&ws->cur_in, n)))) {
    workspace_free(ws);
    return s;
  }
  if (cudaMallocHost(&ws->ctl_host, sizeof(Ctl)) != cudaSuccess) {
    workspace_free(ws);
    return fail(SSSP_ERR_OUT_OF_MEMORY, "pinned host allocation failed");
  }
  *out = ws;
  return SSSP_OK;
}

sssp_status workspace_get(sssp_graph* g, Workspace** out) {
  if (!g->ws) {
    sssp_status s = workspace_alloc(g->n, true, &g->ws);
    if (s != SSSP_OK) return s;
  }
  *out = g->ws;
  return SSSP_OK;
}

namespace {

SolveWS ws_view(Workspace* ws, unsigned long long* d, uint32_t crit, bool has_reverse) {
  SolveWS w;
  memset(&w, 0, sizeof w);
  w.d = d ? d : ws->d;
  w.status = ws->status;
  w.q[0] = ws->q0;
  w.q[1] = ws->q1;
  w.sp_v = ws->sp_v;
  w.sp_base = ws->sp_base;
  w.cur_out = (crit & (SSSP_OUT_SIMPLE | SSSP_POLICY_LEARNED)) ? ws->cur_out : nullptr;
  w.cur_in = ((crit & (SSSP_IN_SIMPLE | SSSP_POLICY_LEARNED)) && has_reverse) ? ws->cur_in : nullptr;
  w.ctl = ws->ctl;
  return w;
}

}  // namespace

sssp_status solve_one(sssp_graph* g, uint32_t source, uint32_t crit, uint64_t* dist_out, sssp_stats* stats,
                      uint32_t* settle_phase, sssp_phase_record* trace, uint64_t trace_cap, uint64_t* phases_out,
                      cudaStream_t st) {
  clear_error();
  if (!g) return fail(SSSP_ERR_INVALID_ARG, "graph is NULL");
  if (source >= g->n) return fail(SSSP_ERR_INVALID_ARG, "source %u >= n = %u", source, g->n);
  if (!dist_out) return fail(SSSP_ERR_INVALID_ARG, "dist_out is NULL");
  sssp_status s = check_crit(g, crit);
  if (s != SSSP_OK) return s;
  if ((s = ensure_kernel_attrs()) != SSSP_OK) return s;
  Workspace* ws = nullptr;
  if ((s = workspace_get(g, &ws)) != SSSP_OK) return s;

  const bool dist_dev = is_device_pointer(dist_out);
  const bool sp_dev = settle_phase && is_device_pointer(settle_phase);
  uint32_t* sp_buf = nullptr;
  sssp_phase_record* tr_buf = nullptr;
  if (settle_phase && !sp_dev) SSSP_CUDA_TRY(cudaMallocAsync(&sp_buf, g->n * sizeof(uint32_t), st));
  if (trace && trace_cap) SSSP_CUDA_TRY(cudaMallocAsync(&tr_buf, trace_cap * sizeof(sssp_phase_record), st));

  SolveParams p;
  memset(&p, 0, sizeof p);
  p.g = view_of(g);
  p.ws = ws_view(ws, dist_dev ? reinterpret_cast<unsigned long long*>(dist_out) : nullptr, crit, g->rrow_off);
  p.ws.settle_phase = settle_phase ? (sp_dev ? settle_phase : sp_buf) : nullptr;
  p.ws.trace = tr_buf;
  p.ws.trace_cap = tr_buf ? trace_cap : 0;
  p.source = source;
  p.crit = crit;
  p.wait_ns = wait_limit_ns();

  // Enough blocks to cover the vertices, at most all co-resident blocks.
  const int max_blocks = g_blocks_per_sm * sm_count();
  const uint64_t want = ((uint64_t)g->n + kTile - 1) / kTile;
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)max_blocks));
  SSSP_CUDA_TRY(cudaMemsetAsync(ws->ctl, 0, sizeof(Ctl), st));
  void* args[] = {&p};
  SSSP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_solve_grid, dim3(blocks), dim3(kThreads), args,
                                            kSmemBytes, st));
  SSSP_CUDA_TRY(cudaMemcpyAsync(ws->ctl_host, ws->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  if (!dist_dev)
    SSSP_CUDA_TRY(cudaMemcpyAsync(dist_out, ws->d, g->n * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  if (sp_buf) SSSP_CUDA_TRY(cudaMemcpyAsync(settle_phase, sp_buf, g->n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
  const Ctl& c = *ws->ctl_host;
  if (c.err != 0) {
    if (sp_buf) cudaFree(sp_buf);
    if (tr_buf) cudaFree(tr_buf);
    return fail((sssp_status)c.err, c.err == SSSP_ERR_TIMEOUT ? "an in-kernel wait exceeded its limit"
                                                               : "device-side error %d", c.err);
  }
  if (tr_buf) {
    const uint64_t rec = std::min<uint64_t>(trace_cap, c.phases);
    if (rec) SSSP_CUDA_TRY(cudaMemcpy(trace, tr_buf, rec * sizeof(sssp_phase_record), cudaMemcpyDeviceToHost));
    SSSP_CUDA_TRY(cudaFree(tr_buf));
  }
  if (sp_buf) SSSP_CUDA_TRY(cudaFree(sp_buf));
  if (phases_out) *phases_out = c.phases;
  if (stats) {
    stats->phases = c.phases;
    stats->sum_frontier = c.sum_f;
    stats->settled = c.settled;
    stats->edges_relaxed = c.relaxed;
  }
  return SSSP_OK;
}

// ---- batch

struct BatchPlan {
  uint32_t count = 0;
  uint32_t crit = 0;
  BatchItem* items = nullptr;          // device, largest graph first
  unsigned int* next = nullptr;        // device work counter
  std::vector<Workspace*> ws;          // one per solve
  unsigned long long* phases = nullptr;  // device [count], caller order
  bool own_phases = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace sssp

struct sssp_batch : sssp::BatchPlan {};

namespace sssp {
namespace {

void batch_free(sssp_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (Workspace* w : b->ws) workspace_free(w);
  cudaFree(b->items);
  cudaFree(b->next);
  if (b->own_phases) cudaFree(b->phases);
  delete b;
}

// Queue the batch on `st`: reset the work counter and every control block,
// then one launch of resident blocks that pull solves until none is left.
sssp_status batch_enqueue(sssp_batch* b, cudaStream_t st) {
  SSSP_CUDA_TRY(cudaMemsetAsync(b->next, 0, sizeof(unsigned int), st));
  for (Workspace* w : b->ws) SSSP_CUDA_TRY(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl), st));
  const int blocks = (int)std::min<uint64_t>(b->count, (uint64_t)g_blocks_per_sm * sm_count());
  k_solve_batch<<<blocks, kThreads, kSmemBytes, st>>>(b->items, b->count, b->next, b->crit, b->phases);
  SSSP_CUDA_TRY(cudaGetLastError());
  return SSSP_OK;
}

sssp_status batch_build(sssp_graph* const* graphs, const uint32_t* sources, uint32_t count, uint32_t crit,
                        uint64_t* const* dist_out, uint64_t* phases_dev, cudaStream_t st, sssp_batch** out) {
  if (!graphs || !sources || !dist_out || count == 0) return fail(SSSP_ERR_INVALID_ARG, "empty or NULL batch");
  if (crit & SSSP_POLICY_LEARNED) return fail(SSSP_ERR_UNSUPPORTED, "the learned policy is not available in batches");
  for (uint32_t i = 0; i < count; ++i) {
    if (!graphs[i]) return fail(SSSP_ERR_INVALID_ARG, "graph %u is NULL", i);
    if (sources[i] >= graphs[i]->n) return fail(SSSP_ERR_INVALID_ARG, "source of solve %u out of range", i);
    if (!dist_out[i] || !is_device_pointer(dist_out[i]))
      return fail(SSSP_ERR_INVALID_ARG, "dist_out[%u] must be device memory", i);
    sssp_status s = check_crit(graphs[i], crit);
    if (s != SSSP_OK) return s;
  }
  sssp_status s = ensure_kernel_attrs();
  if (s != SSSP_OK) return s;
  sssp_batch* b = new (std::nothrow) sssp_batch();
  if (!b) return fail(SSSP_ERR_OUT_OF_MEMORY, "host allocation failed");
  b->count = count;
  b->crit = crit;
  // Largest solves first, so the tail of the queue holds the short ones.
  std::vector<uint32_t> order(count);
  for (uint32_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
    return graphs[a]->m + graphs[a]->n > graphs[c]->m + graphs[c]->n;
  });
  std::vector<BatchItem> h(count);
  b->ws.assign(count, nullptr);
  const bool cursors = (crit & (SSSP_IN_SIMPLE | SSSP_OUT_SIMPLE)) != 0;
  for (uint32_t k = 0; k < count; ++k) {
    const uint32_t i = order[k];
    if ((s = workspace_alloc(graphs[i]->n, cursors, &b->ws[k])) != SSSP_OK) {
      batch_free(b);
      return s;
    }
    h[k].g = view_of(graphs[i]);
    h[k].ws = ws_view(b->ws[k], reinterpret_cast<unsigned long long*>(dist_out[i]), crit, graphs[i]->rrow_off);
    h[k].source = sources[i];
    h[k].out_index = i;
  }
  if (cudaMalloc(&b->items, count * sizeof(BatchItem)) != cudaSuccess ||
      cudaMalloc(&b->next, sizeof(unsigned int)) != cudaSuccess) {
    batch_free(b);
    return fail(SSSP_ERR_OUT_OF_MEMORY, "device allocation failed");
  }
  if (phases_dev) {
    b->phases = reinterpret_cast<unsigned long long*>(phases_dev);
  } else {
    b->own_phases = true;
    if (cudaMalloc(&b->phases, count * sizeof(unsigned long long)) != cudaSuccess) {
      batch_free(b);
      return fail(SSSP_ERR_OUT_OF_MEMORY, "device allocation failed");
    }
  }
  if (cudaMemcpyAsync(b->items, h.data(), count * sizeof(BatchItem), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    batch_free(b);
    return fail(SSSP_ERR_CUDA, "copy of batch descriptors failed");
  }
  *out = b;
  return SSSP_OK;
}

// First control block that recorded an error (0 if none); reads all of them.
sssp_status batch_status(sssp_batch* b) {
  for (Workspace* w : b->ws) {
    SSSP_CUDA_TRY(cudaMemcpy(w->ctl_host, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (w->ctl_host->err != 0) return fail((sssp_status)w->ctl_host->err, "device-side error %d in a batched solve",
                                           w->ctl_host->err);
  }
  return SSSP_OK;
}

}  // namespace
}  // namespace sssp

using namespace sssp;

extern "C" sssp_status sssp_solve(sssp_graph* g, uint32_t source, uint32_t criterion, uint64_t* dist_out,
                                  uint64_t* phases_out, void* stream) {
  return solve_one(g, source, criterion, dist_out, nullptr, nullptr, nullptr, 0, phases_out,
                   static_cast<cudaStream_t>(stream));
}

extern "C" sssp_status sssp_solve_trace(sssp_graph* g, uint32_t source, uint32_t criterion, uint64_t* dist_out,
                                        sssp_stats* stats, uint32_t* settle_phase, sssp_phase_record* trace,
                                        uint64_t trace_cap, void* stream) {
  return solve_one(g, source, criterion, dist_out, stats, settle_phase, trace, trace_cap, nullptr,
                   static_cast<cudaStream_t>(stream));
}

extern "C" sssp_status sssp_solve_batch(sssp_graph* const* graphs, const uint32_t* sources, uint32_t count,
                                        uint32_t criterion, uint64_t* const* dist_out, uint64_t* phases_out,
                                        void* stream) {
  clear_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool ph_dev = phases_out && is_device_pointer(phases_out);
  sssp_batch* b = nullptr;
  sssp_status s = batch_build(graphs, sources, count, criterion, dist_out, ph_dev ? phases_out : nullptr, st, &b);
  if (s != SSSP_OK) return s;
  s = batch_enqueue(b, st);
  if (s == SSSP_OK && cudaStreamSynchronize(st) != cudaSuccess) s = fail(SSSP_ERR_CUDA, "batched solve failed");
  if (s == SSSP_OK) s = batch_status(b);
  if (s == SSSP_OK && phases_out && !ph_dev &&
      cudaMemcpy(phases_out, b->phases, count * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    s = fail(SSSP_ERR_CUDA, "copy of phase counts failed");
  batch_free(b);
  return s;
}

extern "C" sssp_status sssp_batch_create(sssp_graph* const* graphs, const uint32_t* sources, uint32_t count,
                                         uint32_t criterion, uint64_t* const* dist_out, uint64_t* phases_out,
                                         void* stream, sssp_batch** out) {
  clear_error();
  if (!out) return fail(SSSP_ERR_INVALID_ARG, "out is NULL");
  if (phases_out && !is_device_pointer(phases_out))
    return fail(SSSP_ERR_INVALID_ARG, "phases_out of a prepared batch must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  sssp_batch* b = nullptr;
  sssp_status s = batch_build(graphs, sources, count, criterion, dist_out, phases_out, st, &b);
  if (s != SSSP_OK) return s;
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    batch_free(b);
    return fail(SSSP_ERR_CUDA, "stream creation failed");
  }
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    s = batch_enqueue(b, cap);
    e = cudaStreamEndCapture(cap, &b->graph);
  }
  if (e == cudaSuccess && s == SSSP_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess || s != SSSP_OK) {
    batch_free(b);
    return s != SSSP_OK ? s : fail(SSSP_ERR_CUDA, "CUDA graph capture failed: %s", cudaGetErrorString(e));
  }
  *out = b;
  return SSSP_OK;
}

extern "C" sssp_status sssp_batch_launch(sssp_batch* b, void* stream) {
  clear_error();
  if (!b) return fail(SSSP_ERR_INVALID_ARG, "batch is NULL");
  SSSP_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return SSSP_OK;
}

extern "C" void sssp_batch_destroy(sssp_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_free(b);
}

// engine.cu -- the phase engine of the generic phased SSSP algorithm (Section 3).
//
// One persistent launch runs a whole solve (or, for batches, each group of
// blocks runs whole solves one after another).  A phase settles every fringe
// vertex that the criterion proves final, against the state at the start of
// the phase, then relaxes all of their out-edges:
//
//   select   v in F is settled iff                          (step B)
//              IN : d[v] <= minD + inmin(v)     (inmin empty -> holds)
//              OUT: d[v] <= minOut
//            (eqs. crit:instatic / crit:insimple / crit:outstatic /
//            crit:outsimple).  Settled vertices are marked S before any
//            relaxation; those with out-edges go to the relax list with an
//            exclusive prefix of their degrees (one packed 64-bit atomicAdd per
//            warp reserves the slots and the edge range together, so the prefix
//            is monotone); the rest of F is compacted into the next queue.
//   relax    edge-balanced over the relax list: a block takes a tile of
//            consecutive edges, finds the owners by binary search, and for every
//            edge (u,t) with t not in S: cand = d[u] + c(u,t); if cand < d[t]:
//            atomicMin(d[t], cand); an old value of infinity moves t U -> F.
//
// Thresholds minD = min_F d and minOut = min_F (d + outmin) come either
//   - fused (two barriers per phase): the values of phase k+1 are accumulated
//     during phase k from the kept fringe entries (step B) and from every
//     relaxation that lowered a distance (step C).  The final d of every
//     vertex of the next fringe is among the accumulated values and every
//     accumulated value is >= its vertex's final d, so the minima are exact.
//     Used when the OUT minimum is static (it never changes for a vertex).
//     With IN-SIMPLE the in-cursor of every target of a relaxed edge is
//     advanced in step C, so the dynamic in-minima are exact for the next phase.
//   - or by a separate pass (step A, three barriers) that also advances the
//     out-/in-cursors lazily over the cost-sorted rows (Proposition 3): needed
//     by OUT-SIMPLE (out-minima grow when a target settles) and DIJK.
//
// Solo mode: while |F| is small, block 0 of the group runs whole phases alone
// with block barriers (tens of ns instead of ~1 us per grid barrier); the other
// blocks wait on a bounded gate and rejoin when |F| grows or the solve ends.
//
// Phase control: the phase that settles the source is phase 1; the loop ends
// when the next queue is empty.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "engine.h"
#include "internal.h"
#include "policy.cuh"

namespace sssp {

// A group of co-resident blocks running one solve.  size == 1: block barriers.
struct Grp {
  GridBarrier* bar;
  int* err;
  unsigned long long limit;
  unsigned int rank;
  unsigned int size;
  __device__ bool sync() const {
    if (size == 1) {
      __syncthreads();
      return true;
    }
    return grid_sync(bar, rank, size, limit, err);
  }
};

// Per-phase choice: which IN variant and which fringe representation.
struct Arm {
  bool in_simple;
  bool dense;
  int index;  // policy arm (0..3), -1 without a policy
};

// Number of relax-list entries whose base is <= x (bases strictly increasing),
// by one warp with 31 pivots per round.  All 32 lanes call it.
__device__ __forceinline__ uint32_t warp_upper_bound_sp(const SpEnt* a, uint32_t len, uint32_t x) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = len;
  while (hi - lo > 32) {
    const uint32_t span = hi - lo;
    const uint32_t p = lo + (uint32_t)(((uint64_t)span * (uint32_t)(lane + 1)) >> 5);
    const bool le = lane < 31 && ldcg_u32(&a[p].base) <= x;
    const unsigned int mask = __ballot_sync(0xFFFFFFFFu, le);
    const int c = __popc(mask);
    const uint32_t plo = __shfl_sync(0xFFFFFFFFu, p, c > 0 ? c - 1 : 0);
    const uint32_t phi = __shfl_sync(0xFFFFFFFFu, p, c < 31 ? c : 0);
    if (c > 0) lo = plo + 1;
    if (c < 31) hi = phi;
  }
  const bool le = lo + lane < hi && ldcg_u32(&a[lo + lane].base) <= x;
  return lo + __popc(__ballot_sync(0xFFFFFFFFu, le));
}

// Advance the out-cursor of v past targets in S; return the dynamic out-minimum.
__device__ __forceinline__ uint32_t out_min_dynamic(const GraphView& g, const SolveWS& w, uint32_t v) {
  const uint32_t c0 = ldcg_u32(&w.cur_out[v]);
  const uint32_t end = (uint32_t)__ldg(&g.row_off[v + 1]);
  uint32_t c = c0, cost = kInf32;
  while (c < end) {
    const uint2 e = __ldg(&g.edges[c]);
    if (ldcg_u8(&w.status[e.x]) != kS) { cost = e.y; break; }
    ++c;
  }
  if (c != c0) w.cur_out[v] = c;
  return cost;
}

// Advance the in-cursor of v past sources in S; return the dynamic in-minimum.
// Concurrent callers for the same v compute the same position (S does not
// change while they run), published with atomicMax.
__device__ __forceinline__ uint32_t in_min_dynamic(const GraphView& g, const SolveWS& w, uint32_t v, bool shared_v) {
  const uint32_t c0 = ldcg_u32(&w.cur_in[v]);
  const uint32_t end = (uint32_t)__ldg(&g.rrow_off[v + 1]);
  uint32_t c = c0, cost = kInf32;
  while (c < end) {
    const uint2 e = __ldg(&g.redges[c]);
    if (ldcg_u8(&w.status[e.x]) != kS) { cost = e.y; break; }
    ++c;
  }
  if (c != c0) {
    if (shared_v) atomicMax(&w.cur_in[v], c);
    else w.cur_in[v] = c;
  }
  return cost;
}

// OUT-WEAK term of fringe vertex u on the phase-start state: the minimum over
// out-edges (u,w) with w not settled of c(u,w) for w in F and c(u,w) +
// outmin(w) for w unexplored (eq. crit:outweak).  The term is not monotone (it
// drops when w enters F and grows when w settles), so it is recomputed in every
// phase, but cheaply: the row is sorted by cost, every term of an edge is at
// least its cost, so the scan stops at the first edge whose cost reaches the
// best term found; and it starts at the out-cursor, which skips the row's
// prefix of settled targets (S only grows, so the cursor only moves forward,
// as in Proposition 3).  The caller is the only thread computing u's term in
// the phase.
__device__ __forceinline__ unsigned long long out_min_weak(const GraphView& g, const SolveWS& w, uint32_t u) {
  const uint64_t e = __ldg(&g.row_off[u + 1]);
  const uint64_t c0 = w.cur_out ? (uint64_t)ldcg_u32(&w.cur_out[u]) : __ldg(&g.row_off[u]);
  uint64_t skip = c0;  // end of the settled prefix
  unsigned long long best = kInf64;
  for (uint64_t c = c0; c < e; ++c) {
    const uint2 ed = __ldg(&g.edges[c]);
    if ((unsigned long long)ed.y >= best) break;  // no later edge can give a smaller term
    const uint8_t st = ldcg_u8(&w.status[ed.x]);
    if (st == kS) {
      if (skip == c) skip = c + 1;
      continue;
    }
    unsigned long long x = ed.y;
    if (st == kU) {
      const uint32_t o = __ldg(&g.out_min[ed.x]);
      if (o == kInf32) continue;  // no out-edge of w: no path through it
      x += o;
    }
    best = x < best ? x : best;
  }
  if (w.cur_out && skip != c0) w.cur_out[u] = (uint32_t)skip;
  return best;
}

// IN (full) term of fringe vertex v on the phase-start state: the minimum over
// in-edges (w,v) with w not settled of c(w,v) for w in F and c(w,v) + inmin(w)
// for w unexplored (eq. crit:in; an unexplored w has no settled in-neighbour,
// so its static in-minimum is the one the criterion needs, Proposition 1).
// Same scan as out_min_weak over the cost-sorted in-row, from the in-cursor.
__device__ __forceinline__ unsigned long long in_min_full(const GraphView& g, const SolveWS& w, uint32_t v) {
  const uint64_t e = __ldg(&g.rrow_off[v + 1]);
  const uint64_t c0 = w.cur_in ? (uint64_t)ldcg_u32(&w.cur_in[v]) : __ldg(&g.rrow_off[v]);
  uint64_t skip = c0;
  unsigned long long best = kInf64;
  for (uint64_t c = c0; c < e; ++c) {
    const uint2 ed = __ldg(&g.redges[c]);
    if ((unsigned long long)ed.y >= best) break;
    const uint8_t st = ldcg_u8(&w.status[ed.x]);
    if (st == kS) {
      if (skip == c) skip = c + 1;
      continue;
    }
    unsigned long long x = ed.y;
    if (st == kU) {
      const uint32_t i = __ldg(&g.in_min[ed.x]);
      if (i == kInf32) continue;  // w is never reached: the term is infinite
      x += i;
    }
    best = x < best ? x : best;
  }
  if (w.cur_in && skip != c0) w.cur_in[v] = (uint32_t)skip;
  return best;
}

struct Shared {
  unsigned long long* red;    // 64
  unsigned long long* bases;  // 2: output offsets reserved by the block
  uint32_t* s_base;           // kWarps * kTile (one relax tile per warp)
  uint32_t* s_row;            // kWarps * kTile
  unsigned long long* s_d;    // kWarps * kTile
  uint32_t* s_range;          // 2
  uint32_t* scan;             // 34
  uint32_t* whist;            // kWarps * kNfRing: per-warp bucket-list counts of a relax tile
};

__device__ __forceinline__ Shared carve(unsigned char* smem) {
  Shared s;
  s.red = reinterpret_cast<unsigned long long*>(smem);
  s.bases = s.red + 64;
  s.s_d = s.bases + 2;
  s.s_base = reinterpret_cast<uint32_t*>(s.s_d + kWarps * kTile);
  s.s_row = s.s_base + kWarps * kTile;
  s.s_range = s.s_row + kWarps * kTile;
  s.scan = s.s_range + 2;
  s.whist = s.scan + 34;
  return s;
}

// Solve-wide constants derived from the criterion mask.
struct Mode {
  bool fused;        // thresholds accumulated in B and C
  bool use_in;       // some IN criterion
  bool use_out;
  bool out_dyn;      // OUT-SIMPLE (three-step kind)
  bool out_weak;     // OUT-WEAK (three-step kind)
  bool in_full;      // IN (full) (three-step kind)
  bool approx;       // APPROX(k) (three-step kind)
  uint32_t apx_k;    // its recomputation interval
  bool dijk;
  bool nearfar;      // the fringe may be split into a near queue and a far part
  // Status bytes (U/F/S) are read only by dense scans, the dynamic and
  // full/weak minima, APPROX and DIJK; with static criteria on the sparse queue
  // nothing reads them, so settling and discovering a vertex write none.  A
  // policy (its arms may scan densely or use IN-SIMPLE) needs them only until
  // the fringe is split: from then on every phase runs its static sparse arm.
  bool status;          // maintain the status bytes
  bool status_presplit;  // ... only while the fringe is not split
};

__device__ __forceinline__ bool status_live(const Mode& md, bool split) {
  return md.status && !(md.status_presplit && split);
}

// The near/far split needs static keys d(v) - inmin(v) (no IN-SIMPLE phase
// while it is active: a policy is then limited to its IN-STATIC arms), fused
// thresholds, and n <= 2^30 for the far bit.
__device__ __forceinline__ Mode mode_of(const SolveParams& p) {
  const uint32_t crit = p.crit;
  Mode m;
  m.out_weak = (crit & SSSP_OUT_WEAK) != 0;
  m.in_full = (crit & SSSP_IN_FULL) != 0 && p.ws.im_full != nullptr;
  m.out_dyn = (crit & SSSP_OUT_SIMPLE) != 0;
  m.use_out = m.out_dyn || m.out_weak || (crit & SSSP_OUT_STATIC) != 0;
  m.dijk = (crit & SSSP_DIJK) != 0;
  m.approx = (crit & SSSP_APPROX) != 0 && p.ws.apx_in != nullptr;
  m.apx_k = (crit >> SSSP_APPROX_K_SHIFT) & 63u;
  if (m.apx_k == 0) m.apx_k = 1;
  m.fused = !m.out_dyn && !m.out_weak && !m.in_full && !m.dijk && !m.approx;
  const bool policy = (crit & SSSP_POLICY_LEARNED) != 0;
  m.use_in = (crit & (SSSP_IN_STATIC | SSSP_IN_SIMPLE | SSSP_IN_FULL)) != 0 || policy;
  m.nearfar = m.fused && !(crit & SSSP_IN_SIMPLE) && p.nf_min != 0 && p.g.n <= kNearFarMaxVertices;
  const bool reads_status = (crit & (SSSP_FRONTIER_DENSE | SSSP_FRONTIER_AUTO | SSSP_IN_SIMPLE | SSSP_OUT_SIMPLE |
                                     SSSP_IN_FULL | SSSP_OUT_WEAK | SSSP_APPROX | SSSP_DIJK)) != 0;
  m.status = reads_status || policy;
  m.status_presplit = policy && !reads_status;
  return m;
}

// Counters of a solve, kept in registers of the group leader (block 0,
// thread 0) and written to the control block when the solve ends.
struct Stats {
  unsigned long long phases, sum_f, settled, relaxed;
};

__device__ __forceinline__ Arm arm_for(const SolveParams& p, uint32_t nF) {
  Arm a;
  a.in_simple = (p.crit & SSSP_IN_SIMPLE) != 0;
  a.dense = (p.crit & SSSP_FRONTIER_DENSE) != 0 || ((p.crit & SSSP_FRONTIER_AUTO) && nF > (p.g.n >> 2));
  a.index = -1;
  return a;
}

// Arm of phase k: from the criterion mask, or (SSSP_POLICY_LEARNED) from the
// policy network on the phase-start features, evaluated by warp 0 of the block
// and shared through shared memory.  Every thread of the block calls it; every
// block computes the same arm from the same inputs.
static_assert(kPolWeights * sizeof(float) == kSmemBytes - kPolicySmemOffset, "policy smem size");

// The policy weights staged in dynamic shared memory by solve_body.
__device__ __forceinline__ const float* policy_smem() {
  extern __shared__ __align__(16) unsigned char smem_all[];
  return reinterpret_cast<const float*>(smem_all + kPolicySmemOffset);
}

// split = true (the fringe is split into near and far parts) fixes arm 0,
// IN-STATIC on the sparse queue: the split exists for large fringes, where the
// queue scan is what it saves, and IN-SIMPLE cannot use its static keys.
// nQ: queue length (the dense/sparse choice without a policy); nF: |F|.
__device__ Arm choose_arm(const SolveParams& p, uint64_t k, uint32_t nQ, uint32_t nF, uint64_t e_prev,
                          uint64_t s_prev, uint64_t f_prev, bool split) {
  if (!(p.crit & SSSP_POLICY_LEARNED) || p.policy == nullptr) return arm_for(p, nQ);
  if (split) {
    Arm a;
    a.in_simple = false;
    a.dense = false;
    a.index = 0;
    return a;
  }
  __shared__ int s_arm;
  if ((threadIdx.x >> 5) == 0) {
    float f[kPolFeat], y[kPolArms];
    policy_features(f, nF, p.g.n, p.g.m, k, e_prev, s_prev, f_prev);
    policy_forward_warp(policy_smem(), f, y);
    if (threadIdx.x == 0) s_arm = policy_pick(y, p.ws.cur_in != nullptr, (uint64_t)nF * 32 >= p.g.n);
  }
  __syncthreads();
  Arm a;
  a.index = s_arm;
  a.in_simple = a.index >= 2;
  a.dense = (a.index & 1) != 0;
  __syncthreads();
  return a;
}

// Trace arm bits of the near/far split: split active in the phase; the far
// part was refilled (or the split made) at the start of the phase.
constexpr uint32_t kArmNfActive = 4u, kArmNfRefill = 8u, kArmNfPull = 16u;

__device__ __forceinline__ uint32_t arm_code(const Arm& a, bool solo) {
  return (a.dense ? 1u : 0u) | (solo ? 2u : 0u) | (a.index >= 0 ? ((uint32_t)a.index << 8) | 0x80u : 0u);
}

__device__ __forceinline__ void reset_slot(PhaseSlot* s) {
  s->min_d = s->min_out = s->a_min_d = s->a_min_out = kInf64;
  s->relax_packed = 0;
  s->qcount = 0;
  s->argmin = kInf32;
  s->settled_now = 0;
  s->arm = 0;
  s->fsize = 0;
  s->a_min_apx = kInf64;
  s->fresh_count = 0;
}

// Near/far state every relaxation needs: the bound B and the far-vertex
// buckets (see kNfRing).  Identical in every block of the group.
constexpr uint32_t kNoBucket = 0xFFFFFFFFu;
struct NfView {
  unsigned long long bound;   // B (kNoBound: no far vertex)
  unsigned long long origin;  // O
  uint32_t shift;             // s
  uint32_t cursor;            // c
  uint32_t cap;               // entries per list
  uint32_t* lists;            // [kNfRing * cap], or nullptr: no lists (full refills only)
  unsigned int* cnt;          // [kNfRing] list fills
  unsigned int* beyond;       // lowest bucket with an unlisted far vertex
};

// Bucket of a far vertex's stored word (key > B >= O).
__device__ __forceinline__ uint32_t nf_bucket(const NfView& nv, unsigned long long word, uint32_t im) {
  const unsigned long long d = word & ~kFarBit;
  const unsigned long long key = (im == kInf32 || d <= im) ? 0ull : d - im;
  const unsigned long long x = key > nv.origin ? (key - nv.origin) >> nv.shift : 0ull;
  return x < 0xFFFFFF00ull ? (uint32_t)x : 0xFFFFFF00u;
}

// Warp-aggregated listing of far vertices: lane with b != kNoBucket lists v in
// bucket b (lanes with the same ring slot share one atomicAdd).  A bucket past
// the ring or a full list leaves v unlisted and lowers `beyond` to b, so the
// bound never passes b without a full refill.  All 32 lanes call it.
__device__ __forceinline__ void nf_list_append(const NfView& nv, uint32_t b, uint32_t v) {
  const bool want = b != kNoBucket;
  if (!__any_sync(0xFFFFFFFFu, want)) return;
  const unsigned int lane = threadIdx.x & 31;
  const bool listed = want && b <= nv.cursor + kNfRing;
  uint32_t unl = (want && !listed) ? b : kInf32;
  const uint32_t slot = listed ? (b & (kNfRing - 1)) : kInf32;
  const unsigned int peers = __match_any_sync(0xFFFFFFFFu, slot);
  if (listed) {
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(&nv.cnt[slot], (unsigned int)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t pos = base + __popc(peers & ((1u << lane) - 1u));
    if (pos < nv.cap) nv.lists[(uint64_t)slot * nv.cap + pos] = v;
    else unl = b;
  }
  unl = __reduce_min_sync(0xFFFFFFFFu, unl);
  if (lane == 0 && unl != kInf32) atomicMin(nv.beyond, unl);
}

// nf_list_append for N items per lane at once: the slot atomics of all items
// are issued before any of their results is used (one round trip, not N).
template <int N>
__device__ __forceinline__ void nf_list_append_n(const NfView& nv, const uint32_t (&b)[N], const uint32_t (&v)[N]) {
  bool any = false;
#pragma unroll
  for (int i = 0; i < N; ++i) any |= b[i] != kNoBucket;
  if (!__any_sync(0xFFFFFFFFu, any)) return;
  const unsigned int lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
  uint32_t slot[N], base[N], rank[N];
  int lead[N];
  uint32_t unl = kInf32;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const bool want = b[i] != kNoBucket;
    const bool listed = want && b[i] <= nv.cursor + kNfRing;
    if (want && !listed) unl = min(unl, b[i]);
    slot[i] = listed ? (b[i] & (kNfRing - 1)) : kInf32;
    const unsigned int peers = __match_any_sync(0xFFFFFFFFu, slot[i]);
    lead[i] = __ffs(peers) - 1;
    rank[i] = __popc(peers & lt);
    base[i] = 0;
    if (listed && (int)lane == lead[i]) base[i] = atomicAdd(&nv.cnt[slot[i]], (unsigned int)__popc(peers));
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint32_t pos = __shfl_sync(0xFFFFFFFFu, base[i], lead[i]) + rank[i];
    if (slot[i] != kInf32) {
      if (pos < nv.cap) nv.lists[(uint64_t)slot[i] * nv.cap + pos] = v[i];
      else unl = min(unl, b[i]);
    }
  }
  unl = __reduce_min_sync(0xFFFFFFFFu, unl);
  if (lane == 0 && unl != kInf32) atomicMin(nv.beyond, unl);
}

// Relaxation of one edge (u -> t) with d[u] = du (step C, any mode): one
// load of t's record gives d[t] and whether t is settled (kSettledBit); a
// settled target is skipped.  Otherwise d[t] is lowered to du + c: a target
// still unexplored is claimed with atomicMin (its old value tells whether it is
// new to F); any other target gets a fire-and-forget red.min.  A candidate
// below the value read before the update contributes to the next phase's fused
// thresholds: the final d[t] is always contributed by the relaxation that
// wrote it, and every contribution is >= the final d[t].
// Near/far split (B < kNoBound): the candidate is stored with kFarBit when its
// key du + c - inmin(t) exceeds B.  A new vertex that is far is counted (dfar)
// and listed in its bucket (`app`); a far vertex lowered into another bucket is
// listed again (older entries go stale and are skipped when their bucket is
// pulled); a far vertex whose stored word loses the bit is moved to the near
// queue by the one relaxation whose atomicMin saw the bit go.  `fresh` asks the
// caller to append t to the next queue.  kNF = false is the same code for a
// solve with no far vertex (B = kNoBound).
template <bool kNF>
__device__ __forceinline__ void relax_edge_rec(const SolveParams& p, const Mode& md, uint32_t t, uint32_t cost,
                                               unsigned long long du, const VRec& rt, const NfView& nv,
                                               unsigned long long& pd, unsigned long long& po, bool& fresh,
                                               int& dfar, uint32_t& app) {
  const SolveWS& w = p.ws;
  if (rt.d & kSettledBit) return;
  const unsigned long long cand = du + cost;
  unsigned long long enc = cand;
  if (kNF && cand > nv.bound + rt.im) enc |= kFarBit;
  if (enc < rt.d) {
    unsigned long long old = rt.d;
    if (rt.d == kUnexplored) {
      old = atomicMin(&w.vrec[t].d, enc);
      if (old == kUnexplored) {
        if (status_live(md, kNF)) w.status[t] = kF;
        if (kNF && (enc & kFarBit)) {
          ++dfar;
          if (nv.lists) app = nf_bucket(nv, enc, rt.im);
        } else {
          fresh = true;
        }
      } else if (kNF && (old & kFarBit) && !(enc & kFarBit)) {
        fresh = true;  // old < kUnexplored: t was far and is near now
        --dfar;
      } else if (kNF && (enc & kFarBit) && enc < old && nv.lists) {
        const uint32_t b = nf_bucket(nv, enc, rt.im);  // lowered another relaxation's far value
        if (b != nf_bucket(nv, old, rt.im)) app = b;
      }
    } else if (kNF && (rt.d & kFarBit) && !(enc & kFarBit)) {
      old = atomicMin(&w.vrec[t].d, enc);
      if (old & kFarBit) {  // old <= rt.d < kUnexplored
        fresh = true;
        --dfar;
      }
    } else {
      red_min_u64(&w.vrec[t].d, enc);
      if (kNF && (enc & kFarBit) && nv.lists) {  // far and lowered (rt.d is far: its key is larger)
        const uint32_t b = nf_bucket(nv, enc, rt.im);
        if (b != nf_bucket(nv, rt.d, rt.im)) app = b;
      }
    }
    if (md.fused && enc < old) {
      pd = cand < pd ? cand : pd;
      if (rt.om != kInf32) {
        const unsigned long long x = cand + rt.om;
        po = x < po ? x : po;
      }
    }
  }
}

// The same with t's record loaded here (rt above is the record as read
// before any update of this relaxation).
template <bool kNF>
__device__ __forceinline__ void relax_edge(const SolveParams& p, const Mode& md, uint32_t t, uint32_t cost,
                                           unsigned long long du, const NfView& nv, unsigned long long& pd,
                                           unsigned long long& po, bool& fresh, int& dfar, uint32_t& app) {
  relax_edge_rec<kNF>(p, md, t, cost, du, ldcg_vrec(&p.ws.vrec[t]), nv, pd, po, fresh, dfar, app);
}

// Relax-list entry `slot` covers edges [base, base + deg) of the phase's edge
// sequence: it owns the first edge of every tile that starts in that range.
__device__ __forceinline__ void mark_tile_owner(uint32_t* owner, uint32_t slot, uint32_t base, uint32_t deg) {
  const uint64_t end = (uint64_t)base + deg;
  for (uint64_t t = ((uint64_t)base + kTile - 1) / kTile; t * kTile < end; ++t) owner[t] = slot;
}

// Start-of-phase values every block reads once, right after the previous
// phase's last barrier (or a refill's or pull's): the queue length, the far
// part of F, and the fused thresholds with the minima of the far vertices a
// refill or pull of this phase moved to the queue (a_min_*, kInf64 otherwise).
// (After a pull only the group leader's far count is current; no other block
// uses it.)
struct PhaseHead {
  uint32_t nQ;
  uint32_t far;
  unsigned long long min_d, min_out;
  bool split;  // near/far split active (from the block's own state)
};

__device__ __forceinline__ PhaseHead load_head(const Ctl* ctl, uint64_t k, bool split) {
  const PhaseSlot* S0 = &ctl->slot[k % 4];
  PhaseHead h;
  h.split = split;
  h.nQ = ldcg_u32(&S0->qcount);
  h.far = ldcg_u32(&ctl->far_count);
  h.min_d = min(ldcg_u64(&S0->min_d), ldcg_u64(&S0->a_min_d));
  h.min_out = min(ldcg_u64(&S0->min_out), ldcg_u64(&S0->a_min_out));
  return h;
}

// ---------------------------------------------------------------------------
// Step B of phase k (after step A for the three-step kind), by every block of
// the group, ending with a group barrier.  Returns false if a barrier gave up.
__device__ __noinline__ bool phase_select(const SolveParams& p, const Grp& grp, const Mode& md, const Arm arm, uint64_t k,
                                          const PhaseHead& h, const Shared& sh, Stats& st) {
  const GraphView& g = p.g;
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x;
  const unsigned int lane = tid & 31;
  const uint64_t gthreads = (uint64_t)grp.size * nthr;
  const uint64_t gtid = (uint64_t)grp.rank * nthr + tid;
  const bool leader = grp.rank == 0 && tid == 0;
  const int cur = (int)((k - 1) & 1);
  const uint32_t* Q = w.q[cur];
  uint32_t* Qn = w.q[cur ^ 1];
  PhaseSlot* S0 = &ctl->slot[k % 4];
  PhaseSlot* S1 = &ctl->slot[(k + 1) % 4];
  const uint32_t nF = h.nQ;
  const bool wstat = status_live(md, h.split);
  const bool dense = arm.dense;
  const bool in_dyn = md.use_in && arm.in_simple && w.cur_in != nullptr;
  if (leader) {
    reset_slot(&ctl->slot[(k + 2) % 4]);
    const uint32_t fs = nF + (md.nearfar ? h.far : 0u);
    S0->fsize = fs;
    st.sum_f += fs;
    if (w.trace) S0->t_start = globaltimer_ns();
  }

  // ---- thresholds
  unsigned long long minD, minOut, min_apx = kInf64;
  if (md.fused) {
    minD = h.min_d;
    minOut = h.min_out;
    if (in_dyn) {
      // A': dynamic in-minima against S at the start of the phase (no vertex of
      // this phase is marked before the barrier).  Cursors only move forward,
      // so advancing them lazily here is exact.
      if (dense) {
        for (uint64_t v = gtid; v < n; v += gthreads)
          if (ldcg_u8(&w.status[v]) == kF) w.im_dyn[v] = in_min_dynamic(g, w, (uint32_t)v, false);
      } else {
        for (uint64_t i = gtid; i < nF; i += gthreads) {
          const uint32_t v = ldcg_u32(&Q[i]);
          w.im_dyn[v] = in_min_dynamic(g, w, v, false);
        }
      }
      if (!grp.sync()) return false;
    }
  } else {
    const bool apx_recompute = md.approx && (k - 1) % md.apx_k == 0;
    if (md.approx && !apx_recompute) {
      // APPROX bookkeeping for the vertices that entered F in the last relax
      // step: static start values, then every edge between such a vertex and
      // a fringe vertex lowers the fringe vertex's value to the edge's cost
      const uint32_t nfr = ldcg_u32(&S0->fresh_count);
      for (uint64_t i = gtid; i < nfr; i += gthreads) {
        const uint32_t x = ldcg_u32(&w.fresh[i]);
        const uint32_t im = __ldg(&g.in_min[x]), om = __ldg(&g.out_min[x]);
        w.apx_in[x] = im == kInf32 ? kInf64 : im;
        w.apx_out[x] = om == kInf32 ? kInf64 : om;
      }
      if (!grp.sync()) return false;
      for (uint64_t i = gtid; i < nfr; i += gthreads) {
        const uint32_t x = ldcg_u32(&w.fresh[i]);
        for (uint64_t e = __ldg(&g.row_off[x]), e1 = __ldg(&g.row_off[x + 1]); e < e1; ++e) {
          const uint2 ed = __ldg(&g.edges[e]);
          if (ldcg_u8(&w.status[ed.x]) == kF) atomicMin(&w.apx_in[ed.x], (unsigned long long)ed.y);
        }
        for (uint64_t e = __ldg(&g.rrow_off[x]), e1 = __ldg(&g.rrow_off[x + 1]); e < e1; ++e) {
          const uint2 ed = __ldg(&g.redges[e]);
          if (ldcg_u8(&w.status[ed.x]) == kF) atomicMin(&w.apx_out[ed.x], (unsigned long long)ed.y);
        }
      }
      if (!grp.sync()) return false;
    }
    // A: thresholds over the phase-start state, advancing cursors lazily
    unsigned long long lmin_d = kInf64, lmin_out = kInf64, lmin_apx = kInf64;
    auto visit = [&](uint32_t v) {
      const unsigned long long dv = ldcg_u64(&w.vrec[v].d);
      lmin_d = dv < lmin_d ? dv : lmin_d;
      if (md.use_out) {  // the strongest OUT bit set gives the largest threshold
        unsigned long long om;
        if (md.out_weak) {
          om = out_min_weak(g, w, v);
        } else {
          const uint32_t o = md.out_dyn ? out_min_dynamic(g, w, v) : __ldg(&g.out_min[v]);
          om = o == kInf32 ? kInf64 : o;
        }
        if (om != kInf64) {
          const unsigned long long x = dv + om;
          lmin_out = x < lmin_out ? x : lmin_out;
        }
      }
      if (md.in_full) w.im_full[v] = in_min_full(g, w, v);
      else if (in_dyn) w.im_dyn[v] = in_min_dynamic(g, w, v, false);
      if (md.approx) {  // exact terms in every k-th phase, then APPROX's OUT threshold
        unsigned long long ao;
        if (apx_recompute) {
          w.apx_in[v] = in_min_full(g, w, v);
          ao = out_min_weak(g, w, v);
          w.apx_out[v] = ao;
        } else {
          ao = ldcg_u64(&w.apx_out[v]);
        }
        if (ao != kInf64) {
          const unsigned long long x = dv + ao;
          lmin_apx = x < lmin_apx ? x : lmin_apx;
        }
      }
    };
    if (dense) {
      for (uint64_t v = gtid; v < n; v += gthreads)
        if (ldcg_u8(&w.status[v]) == kF) visit((uint32_t)v);
    } else {
      for (uint64_t i = gtid; i < nF; i += gthreads) visit(ldcg_u32(&Q[i]));
    }
    block_min2_to_global(lmin_d, lmin_out, &S0->a_min_d, md.use_out ? &S0->a_min_out : nullptr, sh.red);
    if (md.approx) block_min2_to_global(lmin_apx, kInf64, &S0->a_min_apx, nullptr, sh.red);
    if (!grp.sync()) return false;
    minD = ldcg_u64(&S0->a_min_d);
    minOut = ldcg_u64(&S0->a_min_out);
    if (md.approx) min_apx = ldcg_u64(&S0->a_min_apx);
  }
  uint32_t amin = kInf32;
  if (md.dijk) {  // DIJK: the lowest id among fringe vertices of minimum d
    uint32_t lid = kInf32;
    if (dense) {
      for (uint64_t v = gtid; v < n; v += gthreads)
        if (ldcg_u8(&w.status[v]) == kF && ldcg_u64(&w.vrec[v].d) == minD) lid = min(lid, (uint32_t)v);
    } else {
      for (uint64_t i = gtid; i < nF; i += gthreads) {
        const uint32_t v = ldcg_u32(&Q[i]);
        if (ldcg_u64(&w.vrec[v].d) == minD) lid = min(lid, v);
      }
    }
    lid = __reduce_min_sync(0xFFFFFFFFu, lid);
    if (lane == 0 && lid != kInf32) atomicMin(&S0->argmin, lid);
    if (!grp.sync()) return false;
    amin = ldcg_u32(&S0->argmin);
  }

  // ---- B: select S', mark settled, build the relax list, compact the rest of F.
  // Warp-centric: each warp of the group takes chunks of 32 * kSelItems
  // consecutive entries (lane-interleaved, so the queue loads are coalesced),
  // with all of a lane's record gathers in flight together.  The kept entries
  // and the relax-list entries of a chunk get their slots from one atomicAdd
  // each by lane 0 (the relax list's slots and edge range from one packed
  // 64-bit add, so the edge prefix is monotone in the slot); there is no block
  // barrier inside the loop, so the warps of a block stream independently.
  unsigned long long pd = kInf64, po = kInf64;  // fused partials for phase k+1
  const uint64_t total = dense ? n : nF;
  const unsigned int nwarps = nthr >> 5, warp = tid >> 5;
  const uint64_t gwarps = (uint64_t)grp.size * nwarps;
  const uint64_t wchunk = 32ull * kSelItems;
  const unsigned int lt = (1u << lane) - 1u;
  uint32_t settled_here = 0;
  for (uint64_t c0 = ((uint64_t)grp.rank * nwarps + warp) * wchunk; c0 < total; c0 += gwarps * wchunk) {
    uint32_t vv[kSelItems];
    bool ok[kSelItems];
#pragma unroll
    for (int j = 0; j < kSelItems; ++j) {
      const uint64_t i = c0 + (uint64_t)j * 32 + lane;
      ok[j] = i < total;
      vv[j] = ok[j] ? (dense ? (uint32_t)i : ldcg_u32(&Q[i])) : 0u;
    }
    if (dense) {
#pragma unroll
      for (int j = 0; j < kSelItems; ++j)
        if (ok[j]) ok[j] = ldcg_u8(&w.status[vv[j]]) == kF;
    }
    VRec rr[kSelItems];
#pragma unroll
    for (int j = 0; j < kSelItems; ++j)
      if (ok[j]) rr[j] = ldcg_vrec(&w.vrec[vv[j]]);
    if (dense && md.nearfar) {  // a dense scan also meets the far part of F
#pragma unroll
      for (int j = 0; j < kSelItems; ++j)
        if (ok[j] && (rr[j].d & kFarBit)) ok[j] = false;
    }
    uint32_t selm = 0, keepm = 0;
    uint2 rd[kSelItems];
#pragma unroll
    for (int j = 0; j < kSelItems; ++j) {
      rd[j] = make_uint2(0, 0);
      if (!ok[j]) continue;
      const uint32_t v = vv[j];
      const unsigned long long dv = rr[j].d;
      bool sel = false;
      if (md.use_in) {
        if (md.in_full) {
          const unsigned long long im = ldcg_u64(&w.im_full[v]);
          sel = (im == kInf64) || dv <= minD + im;
        } else {
          const uint32_t im = in_dyn ? ldcg_u32(&w.im_dyn[v]) : rr[j].im;
          sel = (im == kInf32) || dv <= minD + im;
        }
      }
      if (!sel && md.use_out) sel = dv <= minOut;
      if (!sel && md.approx) {
        const unsigned long long ai = ldcg_u64(&w.apx_in[v]);
        sel = ai == kInf64 || dv <= minD + ai || dv <= min_apx;
      }
      if (!sel && md.dijk) sel = (v == amin);
      if (sel) {
        if (wstat) w.status[v] = kS;
        w.vrec[v].d = dv | kSettledBit;
        if (w.settle_phase) w.settle_phase[v] = (uint32_t)k;
        rd[j] = __ldg(&g.rowdeg[v]);
        selm |= 1u << j;
      } else {
        keepm |= 1u << j;
        if (md.fused) {
          pd = dv < pd ? dv : pd;
          if (rr[j].om != kInf32) {
            const unsigned long long x = dv + rr[j].om;
            po = x < po ? x : po;
          }
        }
      }
    }
    settled_here += __popc(selm);
    // slots: entries of step j come before those of step j + 1, lanes in order
    uint32_t kb[kSelItems], rb[kSelItems], eincl[kSelItems];
    uint32_t nk = 0, nr = 0, ne = 0;
#pragma unroll
    for (int j = 0; j < kSelItems; ++j) {
      const bool rl = ((selm >> j) & 1u) && rd[j].y > 0;
      kb[j] = __ballot_sync(0xFFFFFFFFu, (keepm >> j) & 1u);
      rb[j] = __ballot_sync(0xFFFFFFFFu, rl);
      eincl[j] = rb[j] ? warp_inclusive_scan(rl ? rd[j].y : 0u) : 0u;
      nk += __popc(kb[j]);
      nr += __popc(rb[j]);
      ne += __shfl_sync(0xFFFFFFFFu, eincl[j], 31);
    }
    unsigned int kbase = 0;
    unsigned long long rbase = 0;
    if (lane == 0) {
      if (nk) kbase = atomicAdd(&S1->qcount, nk);
      if (nr) rbase = atomicAdd(&S0->relax_packed, ((unsigned long long)nr << 32) | ne);
    }
    kbase = __shfl_sync(0xFFFFFFFFu, kbase, 0);
    rbase = __shfl_sync(0xFFFFFFFFu, rbase, 0);
    uint32_t rslot = (uint32_t)(rbase >> 32), ebase = (uint32_t)rbase;
    // relax-list entries spanning several tiles mark the later tiles' owners
    // together with the warp (a hub's row can span thousands of tiles)
    uint32_t wide = 0;
#pragma unroll
    for (int j = 0; j < kSelItems; ++j) {
      if ((keepm >> j) & 1u) {
        const uint32_t slot = kbase + __popc(kb[j] & lt);
        if (slot < n) Qn[slot] = vv[j];
        else atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
      }
      kbase += __popc(kb[j]);
      if ((rb[j] >> lane) & 1u) {
        const uint32_t slot = rslot + __popc(rb[j] & lt);
        const uint32_t eb = ebase + eincl[j] - rd[j].y;
        if (slot < n) {
          *reinterpret_cast<ulonglong2*>(&w.sp[slot]) =
              make_ulonglong2(rr[j].d, (unsigned long long)rd[j].x | ((unsigned long long)eb << 32));
          if (w.tile_owner) {
            const uint64_t t0 = ((uint64_t)eb + kTile - 1) / kTile;  // first tile starting inside [eb, eb + deg)
            if (t0 * kTile < (uint64_t)eb + rd[j].y) {
              w.tile_owner[t0] = slot;
              if ((t0 + 1) * kTile < (uint64_t)eb + rd[j].y) wide |= 1u << j;
            }
          }
        } else {
          atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
        }
      }
      rslot += __popc(rb[j]);
      ebase += __shfl_sync(0xFFFFFFFFu, eincl[j], 31);
    }
    if (w.tile_owner && __any_sync(0xFFFFFFFFu, wide != 0)) {
      // recompute each wide entry's slot and edge range and share it
      uint32_t rs = (uint32_t)(rbase >> 32), es = (uint32_t)rbase;
#pragma unroll
      for (int j = 0; j < kSelItems; ++j) {
        unsigned int wm = __ballot_sync(0xFFFFFFFFu, (wide >> j) & 1u);
        while (wm) {
          const int src = __ffs(wm) - 1;
          wm &= wm - 1;
          const uint32_t slot = rs + __popc(rb[j] & ((1u << src) - 1u));
          const uint32_t eb = es + __shfl_sync(0xFFFFFFFFu, eincl[j] - rd[j].y, src);
          const uint32_t deg = __shfl_sync(0xFFFFFFFFu, rd[j].y, src);
          const uint64_t end = (uint64_t)eb + deg;
          for (uint64_t t = ((uint64_t)eb + kTile - 1) / kTile + 1 + lane; t * kTile < end; t += 32) w.tile_owner[t] = slot;
        }
        rs += __popc(rb[j]);
        es += __shfl_sync(0xFFFFFFFFu, eincl[j], 31);
      }
    }
  }
  settled_here = __reduce_add_sync(0xFFFFFFFFu, settled_here);
  if (lane == 0 && settled_here) atomicAdd(&S0->settled_now, settled_here);
  if (md.fused) block_min2_to_global(pd, po, &S1->min_d, md.use_out ? &S1->min_out : nullptr, sh.red);
  return grp.sync();
}

// Step C of phase k (relax every out-edge of S', edge-balanced tiles), then
// the end-of-phase barrier, counters and trace.  Every block of the group
// calls it.  Returns false if a barrier gave up.
//
// Warp-centric: each warp takes tiles of kTile consecutive edges of the relax
// list's edge sequence.  The relax-list entries overlapping a tile (found with
// the tile-owner marks of step B, or by a warp search without them) are staged
// in the warp's own shared-memory slice; every lane then finds the owner of
// each of its kRelaxItems edges by binary search there, issues all of its edge
// loads, then all of its target-record loads, and relaxes.  Vertices new to
// the next queue get their slots from one atomicAdd per tile.
template <bool kNF>
__device__ __noinline__ bool phase_relax(const SolveParams& p, const Grp& grp, const Mode& md, const Arm arm, uint64_t k,
                                         const NfView& nv, bool resumed, const Shared& sh, Stats& st) {
  const GraphView& g = p.g;
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x;
  const unsigned int lane = tid & 31, warp = tid >> 5;
  const bool leader = grp.rank == 0 && tid == 0;
  const int cur = (int)((k - 1) & 1);
  uint32_t* Qn = w.q[cur ^ 1];
  PhaseSlot* S0 = &ctl->slot[k % 4];
  PhaseSlot* S1 = &ctl->slot[(k + 1) % 4];
  unsigned long long pd = kInf64, po = kInf64;
  int dfar = 0;
  const unsigned int nwarps = nthr >> 5;
  const uint64_t gwarps = (uint64_t)grp.size * nwarps;
  // The warp's tiles are software-pipelined: while tile i's slot
  // reservations (next queue, bucket lists) are in flight, tile i+1's relax
  // entries are staged and its edge loads issued; tile i+1's owner marks are
  // loaded before tile i is relaxed.
  const uint64_t tile0 = (uint64_t)grp.rank * nwarps + warp;
  const uint64_t owner_len = g.m / kTile + 2;  // length of the tile-owner array
  uint32_t mlo = 0, mhi = 0;  // owner marks of the next tile to stage
  if (w.tile_owner && tile0 + 1 < owner_len) {
    mlo = ldcg_u32(&w.tile_owner[tile0]);
    mhi = ldcg_u32(&w.tile_owner[tile0 + 1]);
  }
  const unsigned long long packed = ldcg_u64(&S0->relax_packed);
  const uint32_t nS = (uint32_t)(packed >> 32);
  const uint32_t E = (uint32_t)packed;
  if (leader && w.trace && !resumed) S0->t_select = globaltimer_ns();  // (a hand-off set it)
  const unsigned int lt = (1u << lane) - 1u;
  uint32_t* s_base = sh.s_base + warp * kTile;
  uint32_t* s_row = sh.s_row + warp * kTile;
  unsigned long long* s_d = sh.s_d + warp * kTile;
  uint32_t* wh = sh.whist + warp * kNfRing;
  if (kNF) {
    for (uint32_t j = lane; j < kNfRing; j += 32) wh[j] = 0;
    __syncwarp();
  }
  // Front half of tile t: stage the relax-list entries overlapping it in the
  // warp's slice, find each edge's owner entry (ownp: 8 bits per item, the
  // entry's index in the slice) and issue the edge loads.
  uint2 ed[kRelaxItems];
  uint32_t ownp = 0, valid = 0;
  auto front = [&](uint64_t t) {
    const uint32_t e0 = (uint32_t)(t * kTile);
    const uint32_t e1 = (uint64_t)e0 + kTile < E ? e0 + kTile : E;
    uint32_t lo = 0, hi = nS - 1;
    if (w.tile_owner) {
      // entries lo .. hi intersect the tile (hi may start just past it, and is
      // then dropped by the kTile cap below: the per-edge search never picks it)
      lo = mlo;
      if (e1 < E) hi = mhi;
    } else if (!(e0 == 0 && e1 == E)) {
      lo = warp_upper_bound_sp(w.sp, nS, e0) - 1;
      hi = warp_upper_bound_sp(w.sp, nS, e1 - 1) - 1;
    }
    const uint32_t cnt = min(hi - lo + 1, (uint32_t)kTile);
    for (uint32_t j = lane; j < cnt; j += 32) {
      const SpEnt e = ldcg_sp(&w.sp[lo + j]);
      s_base[j] = e.base;
      s_row[j] = e.row;
      s_d[j] = e.d;
    }
    __syncwarp();
    ownp = 0;
    valid = 0;
#pragma unroll
    for (int it = 0; it < kRelaxItems; ++it) {
      const uint32_t e = e0 + it * 32 + lane;
      ed[it] = make_uint2(0, 0);
      if (e < e1) {
        uint32_t a = 0, b = cnt;  // owner = last j with s_base[j] <= e
        while (b - a > 1) {
          const uint32_t mid = (a + b) >> 1;
          if (s_base[mid] <= e) a = mid; else b = mid;
        }
        ed[it] = __ldg(&g.edges[s_row[a] + (e - s_base[a])]);
        ownp |= a << (8 * it);
        valid |= 1u << it;
      }
    }
  };
  static_assert(kTile <= 256 && kRelaxItems <= 4, "owner indices packed 8 bits per item");
  if (tile0 * kTile < E) front(tile0);
  for (uint64_t tile = tile0; tile * kTile < E;) {
    const uint64_t next = tile + gwarps;
    const bool has_next = next * kTile < E;
    if (has_next && w.tile_owner && next + 1 < owner_len) {
      mlo = ldcg_u32(&w.tile_owner[next]);
      mhi = ldcg_u32(&w.tile_owner[next + 1]);
    }
    // ---- back half of this tile: target records, relaxations
    VRec rt[kRelaxItems];
#pragma unroll
    for (int it = 0; it < kRelaxItems; ++it)
      if ((valid >> it) & 1u) rt[it] = ldcg_vrec(&w.vrec[ed[it].x]);
    uint32_t fmask = 0;
    uint32_t app[kRelaxItems], tv[kRelaxItems];
#pragma unroll
    for (int it = 0; it < kRelaxItems; ++it) {
      app[it] = kNoBucket;
      tv[it] = ed[it].x;
      if ((valid >> it) & 1u) {
        bool fresh = false;
        relax_edge_rec<kNF>(p, md, ed[it].x, ed[it].y, s_d[(ownp >> (8 * it)) & 0xFFu], rt[it], nv, pd, po, fresh,
                            dfar, app[it]);
        if (fresh) fmask |= 1u << it;
      }
    }
    // reservations, issued now and consumed after the next tile's front half:
    // next-queue slots (one atomic per tile) ...
    uint32_t nfr = 0;
#pragma unroll
    for (int it = 0; it < kRelaxItems; ++it) nfr += __popc(__ballot_sync(0xFFFFFFFFu, (fmask >> it) & 1u));
    unsigned int fslot = 0, xslot = 0;
    if (nfr && lane == 0) {
      fslot = atomicAdd(&S1->qcount, nfr);
      if (md.approx) xslot = atomicAdd(&S1->fresh_count, nfr);
    }
    // ... and bucket-list ranges: ranks within the warp per ring slot
    // (shared-memory atomics), then one global atomicAdd per slot used, its
    // result kept by the lane of that slot (slot j: lane j & 31, word j >> 5)
    uint32_t rankp = 0, lmask = 0, unl = kInf32;
    unsigned int lb0 = 0, lb1 = 0;
    bool any_far = false;
    if (kNF) {
      bool mine = false;
#pragma unroll
      for (int it = 0; it < kRelaxItems; ++it) mine |= app[it] != kNoBucket;
      any_far = __any_sync(0xFFFFFFFFu, mine);
    }
    if (any_far) {
#pragma unroll
      for (int it = 0; it < kRelaxItems; ++it) {
        const bool want = app[it] != kNoBucket;
        const bool listed = want && app[it] <= nv.cursor + kNfRing;
        if (want && !listed) unl = min(unl, app[it]);
        if (listed) {
          rankp |= atomicAdd(&wh[app[it] & (kNfRing - 1)], 1u) << (8 * it);
          lmask |= 1u << it;
        }
      }
      __syncwarp();
      const uint32_t c0 = wh[lane], c1 = wh[lane + 32];
      if (c0) lb0 = atomicAdd(&nv.cnt[lane], c0);
      if (c1) lb1 = atomicAdd(&nv.cnt[lane + 32], c1);
      wh[lane] = 0;
      wh[lane + 32] = 0;
    }
    static_assert(kNfRing == 64, "two ring slots per lane");
    __syncwarp();  // the slice is read; the next tile may overwrite it
    // ---- front half of the next tile
    if (has_next) front(next);
    // ---- this tile's appends
    if (nfr) {
      fslot = __shfl_sync(0xFFFFFFFFu, fslot, 0);
      xslot = __shfl_sync(0xFFFFFFFFu, xslot, 0);
#pragma unroll
      for (int it = 0; it < kRelaxItems; ++it) {
        const unsigned int fb = __ballot_sync(0xFFFFFFFFu, (fmask >> it) & 1u);
        if ((fmask >> it) & 1u) {
          const uint32_t off = __popc(fb & lt);
          if (fslot + off < n) Qn[fslot + off] = tv[it];
          else atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
          if (md.approx) {
            if (xslot + off < n) w.fresh[xslot + off] = tv[it];
            else atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
          }
        }
        fslot += __popc(fb);
        xslot += __popc(fb);
      }
    }
    if (any_far) {
#pragma unroll
      for (int it = 0; it < kRelaxItems; ++it) {
        const uint32_t slot = app[it] & (kNfRing - 1);
        const unsigned int b0 = __shfl_sync(0xFFFFFFFFu, lb0, slot & 31);
        const unsigned int b1 = __shfl_sync(0xFFFFFFFFu, lb1, slot & 31);
        if ((lmask >> it) & 1u) {
          const uint32_t pos = (slot < 32 ? b0 : b1) + ((rankp >> (8 * it)) & 0xFFu);
          if (pos < nv.cap) nv.lists[(uint64_t)slot * nv.cap + pos] = tv[it];
          else unl = min(unl, app[it]);
        }
      }
      unl = __reduce_min_sync(0xFFFFFFFFu, unl);
      if (lane == 0 && unl != kInf32) atomicMin(nv.beyond, unl);
    }
    tile = next;
  }
  if (md.fused) block_min2_to_global(pd, po, &S1->min_d, md.use_out ? &S1->min_out : nullptr, sh.red);
  if (kNF) {  // far-part count: one atomic per block (the barrier above orders scratch reuse)
    uint32_t tf;
    block_exclusive_scan((uint32_t)dfar, sh.scan, &tf);
    if (tid == 0 && tf) atomicAdd(&ctl->far_count, tf);
  }
  if (!grp.sync()) return false;
  if (leader) {
    const uint32_t settled_now = ldcg_u32(&S0->settled_now);
    st.settled += settled_now;
    st.relaxed += E;
    st.phases = k;
    if (w.trace && k <= w.trace_cap) {
      const uint32_t code = ldcg_u32(&S0->arm);
      const bool in_dyn = md.use_in && w.cur_in != nullptr &&
                          ((code & 0x80u) ? ((code >> 8) >= 2) : arm.in_simple);
      sssp_phase_record r;
      r.frontier = ldcg_u32(&S0->fsize);
      r.settled = settled_now;
      r.min_d = md.fused ? min(ldcg_u64(&S0->min_d), ldcg_u64(&S0->a_min_d)) : ldcg_u64(&S0->a_min_d);
      r.min_out = md.use_out ? (md.fused ? min(ldcg_u64(&S0->min_out), ldcg_u64(&S0->a_min_out))
                                         : ldcg_u64(&S0->a_min_out))
                             : (md.approx ? ldcg_u64(&S0->a_min_apx) : kInf64);
      r.deg_settled = E;
      uint32_t c = p.crit & SSSP_CRITERIA_MASK;
      if (md.use_in) c = (c & ~(uint32_t)(SSSP_IN_STATIC | SSSP_IN_SIMPLE)) | (in_dyn ? SSSP_IN_SIMPLE : SSSP_IN_STATIC);
      r.criterion = c;
      r.arm = ldcg_u32(&S0->arm);
      r.t_start_ns = ldcg_u64(&S0->t_start);
      r.t_end_ns = globaltimer_ns();
      r.queued = ldcg_u32(&S0->qcount);
      r.select_ns = (uint32_t)(ldcg_u64(&S0->t_select) - r.t_start_ns);
      w.trace[k - 1] = r;
    }
  }
  return true;
}

// The policy's last choice in grid mode and the phase it was made in (per
// block; s_arm_k = ~0 at the start of every solve, see solve_body).
static __shared__ Arm s_arm_last;
static __shared__ unsigned long long s_arm_k;

__device__ __forceinline__ bool run_phase(const SolveParams& p, const Grp& grp, const Mode& md, uint64_t k,
                                          const NfView& nv, uint32_t nf_code, const PhaseHead& h, const Shared& sh,
                                          Stats& st) {
  Arm arm;
  if ((p.crit & SSSP_POLICY_LEARNED) && p.policy != nullptr) {
    // The network is evaluated in the first grid phase of a solve and then at
    // most every 4th phase (its forward pass sits on the phase's critical
    // path); the phases in between keep its last choice.  (The previous
    // phase's counts are its features.)  Every block evaluates the same inputs.
    if (nv.bound != kNoBound) {
      arm = choose_arm(p, k, h.nQ, 0, 0, 0, 0, true);  // split: the static sparse arm
    } else if (k <= s_arm_k || k - s_arm_k >= 4) {
      const PhaseSlot* prev = &p.ws.ctl->slot[(k + 3) % 4];
      arm = choose_arm(p, k, h.nQ, h.nQ + (md.nearfar ? h.far : 0u), (uint32_t)ldcg_u64(&prev->relax_packed),
                       ldcg_u32(&prev->settled_now), ldcg_u32(&prev->fsize), false);
      __syncthreads();
      if (threadIdx.x == 0) {
        s_arm_last = arm;
        s_arm_k = k;
      }
      __syncthreads();
    } else {
      arm = s_arm_last;
    }
  } else {
    arm = arm_for(p, h.nQ);
  }
  if (grp.rank == 0 && threadIdx.x == 0) p.ws.ctl->slot[k % 4].arm = arm_code(arm, grp.size == 1) | nf_code;
  if (!phase_select(p, grp, md, arm, k, h, sh, st)) return false;
  return nv.bound != kNoBound ? phase_relax<true>(p, grp, md, arm, k, nv, false, sh, st)
                              : phase_relax<false>(p, grp, md, arm, k, nv, false, sh, st);
}

// Relax step of a solo phase: the warps of the block stride over the relax
// list's edges; vertices new to the next queue get slots from a shared counter
// (slots past kSoloCap go to the global queue at the same index).
struct SoloRelax {
  const unsigned long long* sp_d;
  const uint32_t* sp_row;
  const uint32_t* sp_base;
  uint32_t nS, E;
  uint32_t* sqn;
  uint32_t* gqn;
  unsigned int* qn;
};

template <bool kNF>
__device__ __forceinline__ void solo_relax(const SolveParams& p, const Mode& md, const SoloRelax& r,
                                           const NfView& nv, unsigned long long& pd, unsigned long long& po,
                                           int& dfar) {
  const unsigned int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t eb = warp * 32; eb < r.E; eb += blockDim.x) {
    const uint32_t e = eb + lane;
    bool fresh = false;
    uint32_t t = 0, app = kNoBucket;
    if (e < r.E) {
      uint32_t a = 0, b = r.nS;
      while (b - a > 1) {
        const uint32_t mid = (a + b) >> 1;
        if (r.sp_base[mid] <= e) a = mid; else b = mid;
      }
      const uint2 ed = __ldg(&p.g.edges[r.sp_row[a] + (e - r.sp_base[a])]);
      t = ed.x;
      relax_edge<kNF>(p, md, t, ed.y, r.sp_d[a], nv, pd, po, fresh, dfar, app);
    }
    if (kNF) nf_list_append(nv, app, t);
    const unsigned int fmask = __ballot_sync(0xFFFFFFFFu, fresh);
    if (fmask) {
      unsigned int b0 = 0;
      if (lane == 0) b0 = atomicAdd(r.qn, (unsigned int)__popc(fmask));
      b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
      if (fresh) {
        const uint32_t slot = b0 + __popc(fmask & ((1u << lane) - 1u));
        if (slot < kSoloCap) r.sqn[slot] = t;
        else if (slot < p.g.n) r.gqn[slot] = t;
        else atomicCAS(&p.ws.ctl->err, 0, (int)SSSP_ERR_INTERNAL);
      }
    }
  }
}

// Solo episode (fused thresholds only): this block runs phases k, k+1, ...
// alone while |F| <= min(solo_max, kSoloCap).  The two fringe queues, the
// relax list, the counters and the thresholds live in shared memory; global
// memory is touched only for vertex records, status bytes, edges and distance
// updates.  Queue slots at or beyond kSoloCap go to the global queue at the
// same index.  If a phase's relax list has more than solo_edges edges and
// `can_handoff`, the episode stops after the selection and hands the relax step
// to the whole group (*handoff = true).
// Entry: global queue q[(k-1)&1] with slot[k%3].qcount entries, thresholds in
// slot[k%3].  Exit at phase k: the same state with slot[(k+1)%3] reset (no
// handoff), or the state after a grid selection step of phase k (handoff).
// All threads of the block call it.
__device__ __forceinline__ uint64_t solo_episode(const SolveParams& p, const Mode& md_shared, uint64_t k, const NfView& nv,
                                 uint32_t nf_code, unsigned char* smem, Stats& st_shared, bool can_handoff,
                                 bool* handoff) {
  const Mode md = md_shared;  // in registers for the episode (read in every step)
  const GraphView& g = p.g;
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x;
  const unsigned int lane = tid & 31, warp = tid >> 5;
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* sqa = reinterpret_cast<uint32_t*>(red + 64);
  uint32_t* sqb = sqa + kSoloCap;
  unsigned long long* sp_d = reinterpret_cast<unsigned long long*>(sqb + kSoloCap);
  uint32_t* sp_row = reinterpret_cast<uint32_t*>(sp_d + kSoloCap);
  uint32_t* sp_base = sp_row + kSoloCap;
  // (thread t loads the records of fringe entries t, t + blockDim, ... into
  // registers and decides those same entries: no block barrier between)
  static_assert(kSoloCap % kThreads == 0, "solo entries per thread");
  // per-phase counters, double-buffered by phase parity: the buffer of phase
  // k + 1 is cleared during phase k, after every thread has read it as phase
  // k - 1's
  __shared__ unsigned int s_qn[2], s_settled[2];
  __shared__ unsigned int s_wk[32], s_wr[32], s_we[32];  // per-warp counts
  __shared__ unsigned long long s_relax[2], s_thr_d[2], s_thr_o[2];
  __shared__ int s_dfar[2];
  *handoff = false;

  const uint32_t cap = p.solo_max < kSoloCap ? p.solo_max : kSoloCap;
  // counters of the previous phase (policy features)
  uint32_t e_prev = (uint32_t)ldcg_u64(&ctl->slot[(k + 3) % 4].relax_packed);
  uint32_t s_prev = ldcg_u32(&ctl->slot[(k + 3) % 4].settled_now);
  uint32_t f_prev = ldcg_u32(&ctl->slot[(k + 3) % 4].fsize);
  uint32_t nF = ldcg_u32(&ctl->slot[k % 4].qcount);
  const bool kNF = nv.bound != kNoBound;
  uint32_t far = kNF ? ldcg_u32(&ctl->far_count) : 0u;  // far part of F (not in the queues)
  Stats& st = st_shared;  // thread 0's running counters
  __shared__ unsigned long long s_t0, s_tsel;  // thread 0's trace stamps
  Arm arm{false, false, -1};
  unsigned int since_pick = 0;
  unsigned long long minD = min(ldcg_u64(&ctl->slot[k % 4].min_d), ldcg_u64(&ctl->slot[k % 4].a_min_d));
  unsigned long long minOut = min(ldcg_u64(&ctl->slot[k % 4].min_out), ldcg_u64(&ctl->slot[k % 4].a_min_out));
  {
    const uint32_t* gq = w.q[(k - 1) & 1];
    uint32_t* sq = ((k - 1) & 1) ? sqb : sqa;
    for (uint32_t i = tid; i < nF; i += nthr) sq[i] = ldcg_u32(gq + i);
  }
  if (tid < 2) {
    s_qn[tid] = 0;
    s_settled[tid] = 0;
    s_relax[tid] = 0;
    s_thr_d[tid] = s_thr_o[tid] = kInf64;
    s_dfar[tid] = 0;
  }
  __syncthreads();
  for (;;) {
    const int pb = (int)(k & 1);  // this phase's counter buffer
    const int cur = (int)((k - 1) & 1);
    const uint32_t* sq = cur ? sqb : sqa;
    uint32_t* sqn = cur ? sqa : sqb;
    uint32_t* gqn = w.q[cur ^ 1];
    // the policy is evaluated on the first phase of the episode and every 8th
    // phase after it (the choice is logged per phase either way)
    if (since_pick == 0) arm = choose_arm(p, k, nF, nF + far, e_prev, s_prev, f_prev, kNF);
    since_pick = (since_pick + 1) & 7u;
    const bool in_dyn = md.use_in && arm.in_simple && w.cur_in != nullptr;
    const uint32_t fs = nF + far;  // |F| at the start of the phase
    if (tid == 0 && w.trace) s_t0 = globaltimer_ns();
    // ---- B1: load the records of this thread's fringe entries (all in flight at once)
    constexpr int kIt = kSoloCap / kThreads;
    VRec r[kIt];
#pragma unroll
    for (int j = 0; j < kIt; ++j) {
      const uint32_t i = tid + j * nthr;
      if (i < nF) r[j] = ldcg_vrec(&w.vrec[sq[i]]);
    }
    if (in_dyn) {
#pragma unroll
      for (int j = 0; j < kIt; ++j) {
        const uint32_t i = tid + j * nthr;
        if (i < nF) r[j].im = in_min_dynamic(g, w, sq[i], false);
      }
    }
    // IN-SIMPLE minima read status bytes that the selection below writes
    if (in_dyn) __syncthreads();
    // ---- B2: select.  Pass 1 decides and issues the row loads of the settled
    // vertices; one block scan of per-warp counts gives every warp its output
    // offsets; pass 2 writes the kept entries and the relax list (no shared
    // atomics on the hot counters).
    unsigned long long pd = kInf64, po = kInf64;
    uint32_t selm[kIt], keepm[kIt];
    uint2 rdj[kIt];
#pragma unroll
    for (int j = 0; j < kIt; ++j) {
      selm[j] = keepm[j] = 0;
      rdj[j] = make_uint2(0, 0);
      const uint32_t base = warp * 32 + j * nthr;
      if (base < nF) {
        const uint32_t i = base + lane;
        const bool valid = i < nF;
        bool sel = false;
        if (valid) {
          const unsigned long long dv = r[j].d;
          if (md.use_in) {
            const uint32_t im = r[j].im;
            sel = (im == kInf32) || dv <= minD + im;
          }
          if (!sel && md.use_out) sel = dv <= minOut;
          const uint32_t v = sq[i];
          if (sel) {
            if (status_live(md, kNF)) w.status[v] = kS;
            w.vrec[v].d = dv | kSettledBit;
            if (w.settle_phase) w.settle_phase[v] = (uint32_t)k;
            rdj[j] = __ldg(&g.rowdeg[v]);
          } else {
            pd = dv < pd ? dv : pd;
            const uint32_t om = r[j].om;
            if (om != kInf32) {
              const unsigned long long x = dv + om;
              po = x < po ? x : po;
            }
          }
        }
        selm[j] = __ballot_sync(0xFFFFFFFFu, sel);
        keepm[j] = __ballot_sync(0xFFFFFFFFu, valid && !sel);
      }
    }
    uint32_t wk = 0, wr = 0, we = 0, ws = 0;
#pragma unroll
    for (int j = 0; j < kIt; ++j) {
      if (warp * 32 + j * nthr >= nF) break;  // (warp-uniform) the rest of the steps are empty
      const bool rl = ((selm[j] >> lane) & 1u) && rdj[j].y > 0;
      wk += __popc(keepm[j]);
      ws += __popc(selm[j]);
      wr += __popc(__ballot_sync(0xFFFFFFFFu, rl));
      we += __reduce_add_sync(0xFFFFFFFFu, rl ? rdj[j].y : 0u);
    }
    if (lane == 0) {
      s_wk[warp] = wk;
      s_wr[warp] = wr;
      s_we[warp] = we;
      if (ws) atomicAdd(&s_settled[pb], ws);
    }
    pd = warp_min_u64(pd);
    po = warp_min_u64(po);
    if (lane == 0) {
      if (pd != kInf64) atomicMin(&s_thr_d[pb], pd);
      if (po != kInf64 && md.use_out) atomicMin(&s_thr_o[pb], po);
    }
    __syncthreads();
    if (tid == 0) {  // the next phase's counters (every thread has read them as the last phase's)
      s_qn[pb ^ 1] = 0;
      s_settled[pb ^ 1] = 0;
      s_relax[pb ^ 1] = 0;
      s_thr_d[pb ^ 1] = s_thr_o[pb ^ 1] = kInf64;
      s_dfar[pb ^ 1] = 0;
    }
    {
      // every warp scans the per-warp counts itself: its offsets and the totals
      const unsigned int nw = nthr >> 5;
      const uint32_t a = lane < nw ? s_wk[lane] : 0, b = lane < nw ? s_wr[lane] : 0, c = lane < nw ? s_we[lane] : 0;
      const uint32_t ia = warp_inclusive_scan(a), ib = warp_inclusive_scan(b), ic = warp_inclusive_scan(c);
      uint32_t koff = __shfl_sync(0xFFFFFFFFu, ia - a, warp);
      uint32_t roff = __shfl_sync(0xFFFFFFFFu, ib - b, warp);
      uint32_t eoff = __shfl_sync(0xFFFFFFFFu, ic - c, warp);
      if (warp == 0 && lane == 31) {
        s_qn[pb] = ia;
        s_relax[pb] = ((unsigned long long)ib << 32) | ic;
      }
      const unsigned int lt = (1u << lane) - 1u;
#pragma unroll
      for (int j = 0; j < kIt; ++j) {
        const uint32_t base = warp * 32 + j * nthr;
        if (base < nF) {
          const uint32_t i = base + lane;
          if ((keepm[j] >> lane) & 1u) {
            const uint32_t slot = koff + __popc(keepm[j] & lt);
            const uint32_t v = sq[i];
            if (slot < kSoloCap) sqn[slot] = v;
            else if (slot < n) gqn[slot] = v;
            else atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
          }
          koff += __popc(keepm[j]);
          const bool rl = ((selm[j] >> lane) & 1u) && rdj[j].y > 0;
          const unsigned int rm = __ballot_sync(0xFFFFFFFFu, rl);
          const uint32_t c = rl ? rdj[j].y : 0u;
          const uint32_t incl = warp_inclusive_scan(c);
          if (rl) {
            const uint32_t slot = roff + __popc(rm & lt);  // < |S'| <= nF <= kSoloCap
            sp_d[slot] = r[j].d;
            sp_row[slot] = rdj[j].x;
            sp_base[slot] = eoff + incl - c;
          }
          roff += __popc(rm);
          eoff += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
      }
    }
    __syncthreads();
    const unsigned long long packed = s_relax[pb];
    const uint32_t nS = (uint32_t)(packed >> 32), E = (uint32_t)packed;
    if (can_handoff && E > p.solo_edges) {
      // state of a grid selection step of phase k, in global memory
      for (uint32_t j = tid; j < nS; j += nthr) {
        *reinterpret_cast<ulonglong2*>(&w.sp[j]) =
            make_ulonglong2(sp_d[j], (unsigned long long)sp_row[j] | ((unsigned long long)sp_base[j] << 32));
        if (w.tile_owner) mark_tile_owner(w.tile_owner, j, sp_base[j], (j + 1 < nS ? sp_base[j + 1] : E) - sp_base[j]);
      }
      const uint32_t kept = s_qn[pb];
      const uint32_t nk = kept < kSoloCap ? kept : kSoloCap;
      for (uint32_t j = tid; j < nk; j += nthr) gqn[j] = sqn[j];
      if (tid == 0) {
        st.sum_f += fs;
        ctl->far_count = far;
        PhaseSlot* S0 = &ctl->slot[k % 4];
        PhaseSlot* S1 = &ctl->slot[(k + 1) % 4];
        reset_slot(S0);
        reset_slot(S1);
        reset_slot(&ctl->slot[(k + 2) % 4]);
        S0->qcount = nF;
        S0->fsize = fs;
        S0->min_d = minD;
        S0->min_out = minOut;
        S0->relax_packed = packed;
        S0->settled_now = s_settled[pb];
        S0->arm = arm_code(arm, true) | nf_code;
        S0->t_start = s_t0;
        S0->t_select = globaltimer_ns();
        S1->qcount = kept;
        S1->min_d = s_thr_d[pb];
        S1->min_out = s_thr_o[pb];
      }
      __threadfence();
      __syncthreads();
      *handoff = true;
      return k;
    }
    // ---- C: relax
    if (tid == 0 && w.trace) s_tsel = globaltimer_ns();
    pd = kInf64;
    po = kInf64;
    int dfar = 0;
    const SoloRelax sr{sp_d, sp_row, sp_base, nS, E, sqn, gqn, &s_qn[pb]};
    if (kNF) solo_relax<true>(p, md, sr, nv, pd, po, dfar);
    else solo_relax<false>(p, md, sr, nv, pd, po, dfar);
    pd = warp_min_u64(pd);
    po = warp_min_u64(po);
    if (kNF) dfar = __reduce_add_sync(0xFFFFFFFFu, dfar);
    if (lane == 0) {
      if (pd != kInf64) atomicMin(&s_thr_d[pb], pd);
      if (po != kInf64 && md.use_out) atomicMin(&s_thr_o[pb], po);
      if (dfar) atomicAdd(&s_dfar[pb], dfar);
    }
    __syncthreads();
    const uint32_t nFn = s_qn[pb];
    const uint32_t settled_now = s_settled[pb];
    if (tid == 0) {
      st.phases = k;
      st.sum_f += fs;
      st.settled += settled_now;
      st.relaxed += E;
      ctl->heartbeat = k;
      if (w.trace && k <= w.trace_cap) {
        sssp_phase_record r;
        r.frontier = fs;
        r.settled = settled_now;
        r.min_d = minD;
        r.min_out = md.use_out ? minOut : kInf64;
        r.deg_settled = E;
        uint32_t c = p.crit & SSSP_CRITERIA_MASK;
        if (md.use_in) c = (c & ~(uint32_t)(SSSP_IN_STATIC | SSSP_IN_SIMPLE)) | (in_dyn ? SSSP_IN_SIMPLE : SSSP_IN_STATIC);
        r.criterion = c;
        r.arm = arm_code(arm, true) | nf_code;
        r.t_start_ns = s_t0;
        r.t_end_ns = globaltimer_ns();
        r.queued = nF;
        r.select_ns = (uint32_t)(s_tsel - s_t0);
        w.trace[k - 1] = r;
      }
    }
    nf_code &= ~(kArmNfRefill | kArmNfPull);  // a refill, pull or split only runs before the episode
    minD = s_thr_d[pb];
    minOut = s_thr_o[pb];
    e_prev = E;
    s_prev = settled_now;
    f_prev = fs;
    nF = nFn;
    if (kNF) far += (uint32_t)s_dfar[pb];
    ++k;
    if (nF == 0 || nF > cap || k > (uint64_t)n + 1) break;
    // thresholds above the bound are exact only after the far part is scanned
    if (kNF && far > 0 && (md.use_out ? minOut : minD) > nv.bound) break;
  }
  // hand the state back in global memory for phase k
  {
    const uint32_t* sq = ((k - 1) & 1) ? sqb : sqa;
    uint32_t* gq = w.q[(k - 1) & 1];
    const uint32_t ns = nF < kSoloCap ? nF : kSoloCap;
    for (uint32_t i = tid; i < ns; i += nthr) gq[i] = sq[i];
  }
  if (tid == 0) {
    PhaseSlot* S0 = &ctl->slot[k % 4];
    reset_slot(S0);
    reset_slot(&ctl->slot[(k + 1) % 4]);
    ctl->far_count = far;
    S0->qcount = nF;
    S0->min_d = minD;
    S0->min_out = minOut;
    PhaseSlot* Sp = &ctl->slot[(k + 3) % 4];  // the last solo phase, for the policy's features
    Sp->relax_packed = e_prev;
    Sp->settled_now = (uint32_t)s_prev;
    Sp->fsize = (uint32_t)f_prev;
  }
  __threadfence();
  __syncthreads();
  return k;
}

// ---------------------------------------------------------------------------
// Near/far split of the fringe (static criteria).  key(v) = d(v) - inmin(v).
// Invariant: a fringe vertex is far (kFarBit set, not in the queue) iff
// key(v) > B; the queue holds exactly the near fringe.  A vertex that any
// criterion settles has key(v) <= T, where T = minOut with an OUT criterion,
// else minD (IN: key <= minD; OUT: key <= d <= minOut; minD <= minOut).  A far
// vertex has d >= key > B, so whenever the thresholds accumulated over the near
// part and the relaxations satisfy T <= B they are the thresholds of the whole
// fringe and every vertex the phase settles is in the queue.  When T > B (and
// the far part is not empty) a refill first computes the exact minima over the
// far part and raises B to at least T.  The selections, and so every result,
// are those of the unsplit fringe.

// Histogram bin of x >= 0: bins 0..3 hold x itself, then 4 bins per octave.
__device__ __forceinline__ int nf_bin(unsigned long long x) {
  if (x < 4) return (int)x;
  const int m = 63 - __clzll((long long)x);
  return 4 * (m - 1) + (int)((x >> (m - 2)) & 3u);
}

// Largest x of bin b (saturated at kNoBound).
__device__ __forceinline__ unsigned long long nf_bin_upper(int b) {
  if (b < 4) return (unsigned long long)b;
  const int m = b / 4 + 1, s = b & 3;
  if (m >= 61) return kNoBound;
  return (1ull << m) + ((unsigned long long)(s + 1) << (m - 2)) - 1;
}

__device__ __forceinline__ unsigned long long nf_key(const VRec& r, unsigned long long d) {
  return (r.im == kInf32 || d <= r.im) ? 0ull : d - r.im;
}

// Near-part size to aim at when the bound is set: the tuning's value, else
// about sqrt(n * settled per phase), which balances the per-phase scan of the
// near queue against the dense refill pass; never more than 1/8 of the fringe,
// so that the bound lands well inside the fringe's keys.
__device__ __forceinline__ uint32_t nf_target(const SolveParams& p, uint64_t k, uint32_t fringe) {
  uint32_t t = p.nf_target;
  if (t == 0) {
    const uint32_t s_prev = ldcg_u32(&p.ws.ctl->slot[(k + 3) % 4].settled_now);
    if (p.ws.nf_list) {
      // listed buckets: raising B costs a pass over the pulled lists only, so
      // the near part is kept at a few phases' worth of settled vertices
      t = s_prev > 2048u ? 4u * s_prev : 8192u;
    } else {
      const float s = (float)(s_prev > 256u ? s_prev : 256u);
      const float x = 2.0f * sqrtf((float)p.g.n * s);
      t = x < 4096.0f ? 4096u : (x > (float)p.g.n ? p.g.n : (uint32_t)x);
    }
  }
  const uint32_t cap = fringe / 8 > 0 ? fringe / 8 : 1u;
  return t < cap ? t : cap;
}

// Adds one to bin `bin` (>= 0) of a shared histogram for every lane that has
// one; lanes with bin < 0 add nothing.  Lanes with the same bin are counted by
// one atomic (keys crowd into few bins).  All 32 lanes of the warp call it.
__device__ __forceinline__ void nf_hist_add(uint32_t* sh_hist, int bin) {
  const unsigned int peers = __match_any_sync(0xFFFFFFFFu, bin);
  if (bin >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&sh_hist[bin], (uint32_t)__popc(peers));
}

// Block-local histogram in shared memory, flushed to the group's histogram.
__device__ __forceinline__ void nf_hist_clear(uint32_t* sh_hist) {
  for (int b = threadIdx.x; b < kNfBins; b += blockDim.x) sh_hist[b] = 0;
  __syncthreads();
}
__device__ __forceinline__ void nf_hist_flush(const uint32_t* sh_hist, unsigned int* gh) {
  __syncthreads();
  for (int b = threadIdx.x; b < kNfBins; b += blockDim.x)
    if (sh_hist[b]) atomicAdd(&gh[b], sh_hist[b]);
}

// Smallest bin whose cumulative count reaches `target` (kNfBins if none),
// read from the group's histogram after a barrier.  Every block computes the
// same answer.  All threads of the block call it.
__device__ __forceinline__ int nf_pick_bin(const unsigned int* gh, uint32_t target, const Shared& sh) {
  __shared__ int s_bin;
  const uint32_t v = threadIdx.x < kNfBins ? ldcg_u32(&gh[threadIdx.x]) : 0u;
  if (threadIdx.x == 0) s_bin = kNfBins;
  uint32_t total;
  const uint32_t excl = block_exclusive_scan(v, sh.scan, &total);
  if (threadIdx.x < kNfBins && excl < target && excl + v >= target) s_bin = (int)threadIdx.x;
  __syncthreads();
  const int b = s_bin;
  __syncthreads();
  return b;
}

// Bucket geometry set by a split or a full refill: bound B, bucket width 2^s
// with 2^s <= e + 1 (e: the key offset above the old bound holding about
// `target` vertices), origin O = B + 1 - 2^s (the near part is bucket 0 and
// below), cursor 0.
__device__ __forceinline__ NfView nf_geometry(const NfView& nv, unsigned long long B, unsigned long long e) {
  NfView v = nv;
  v.bound = B;
  v.cursor = 0;
  v.origin = 0;
  v.shift = 0;
  if (B < kNoBound) {
    const unsigned long long w1 = (e < B ? e : B) + 1;
    v.shift = 63u - (uint32_t)__clzll((long long)w1);
    v.origin = B + 1 - (1ull << v.shift);
  }
  return v;
}

// Empties the bucket lists before a split or a full refill lists the far
// part anew (block rank 0 of the group; ordered before any listing by the
// group barrier that follows).
__device__ __forceinline__ void nf_lists_reset(const Grp& grp, Ctl* ctl) {
  if (grp.rank == 0) {
    if (threadIdx.x < kNfRing) ctl->nf_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) ctl->nf_beyond = kInf32;
  }
}

// First split (B = kNoBound, no far vertex, so the phase-k thresholds are
// exact): B = T + the key offset below which about `target` queue entries lie;
// entries above B are marked far and the queue is compacted.  Leaves B as is
// when the whole fringe fits the target.  Every block of the group calls it.
__device__ __noinline__ bool nf_split(const SolveParams& p, const Grp& grp, const Mode& md, uint64_t k, const Shared& sh,
                                      NfView& nv, uint32_t& uses) {
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x;
  const uint64_t gthreads = (uint64_t)grp.size * nthr;
  const uint64_t gtid = (uint64_t)grp.rank * nthr + tid;
  const bool leader = grp.rank == 0 && tid == 0;
  PhaseSlot* S0 = &ctl->slot[k % 4];
  uint32_t* Q = w.q[(k - 1) & 1];
  const uint32_t nF = ldcg_u32(&S0->qcount);
  const unsigned long long T = md.use_out ? ldcg_u64(&S0->min_out) : ldcg_u64(&S0->min_d);
  if (T >= kNoBound) return true;
  unsigned int* gh = ctl->hist[uses & 1];
  uint32_t* hist = sh.s_base;
  nf_hist_clear(hist);
  for (uint64_t c0 = (uint64_t)grp.rank * nthr; c0 < nF; c0 += gthreads) {  // warp-uniform trips
    const uint64_t i = c0 + tid;
    int bin = -1;
    if (i < nF) {
      const VRec r = ldcg_vrec(&w.vrec[ldcg_u32(&Q[i])]);
      const unsigned long long key = nf_key(r, r.d);
      bin = nf_bin(key > T ? key - T : 0ull);
    }
    nf_hist_add(hist, bin);
  }
  nf_hist_flush(hist, gh);
  if (leader) ctl->nf_tmp = 0;
  if (tid < kNfBins && grp.rank == 0) ctl->hist[(uses + 1) & 1][tid] = 0;  // the next use's histogram
  nf_lists_reset(grp, ctl);
  ++uses;
  if (!grp.sync()) return false;
  const int b = nf_pick_bin(gh, nf_target(p, k, nF), sh);
  if (b >= kNfBins) return true;
  const unsigned long long e = nf_bin_upper(b);
  const unsigned long long B = e >= kNoBound - T ? kNoBound : T + e;
  if (B >= kNoBound) return true;
  const NfView v2 = nf_geometry(nv, B, e);
  // keep the entries with key <= B (compacted into the relax-list buffer),
  // mark the others far and list them in their buckets
  uint32_t* tmp = reinterpret_cast<uint32_t*>(w.sp);
  uint32_t demoted = 0;
  for (uint64_t c0 = (uint64_t)grp.rank * nthr; c0 < nF; c0 += gthreads) {
    const uint64_t i = c0 + tid;
    bool keep = false;
    uint32_t v = 0, app = kNoBucket;
    if (i < nF) {
      v = ldcg_u32(&Q[i]);
      const VRec r = ldcg_vrec(&w.vrec[v]);
      keep = nf_key(r, r.d) <= B;
      if (!keep) {
        w.vrec[v].d = r.d | kFarBit;
        ++demoted;
        if (v2.lists) app = nf_bucket(v2, r.d, r.im);
      }
    }
    nf_list_append(v2, app, v);
    uint32_t tk;
    const uint32_t pk = block_exclusive_scan(keep ? 1u : 0u, sh.scan, &tk);
    if (tid == 0) sh.bases[0] = tk ? atomicAdd(&ctl->nf_tmp, tk) : 0u;
    __syncthreads();
    if (keep) tmp[(uint32_t)sh.bases[0] + pk] = v;
    __syncthreads();
  }
  uint32_t td;
  block_exclusive_scan(demoted, sh.scan, &td);
  if (tid == 0 && td) atomicAdd(&ctl->far_count, td);
  if (!grp.sync()) return false;
  const uint32_t kept = ldcg_u32(&ctl->nf_tmp);
  for (uint64_t i = gtid; i < kept; i += gthreads) Q[i] = ldcg_u32(&tmp[i]);
  if (leader) S0->qcount = kept;
  if (tid == 0) nv = v2;  // (published to the block by the barrier below)
  return grp.sync();
}

// Refill (far part not empty, accumulated T > B).  R1: every block scans its
// own contiguous range of vertex records (kNfItems loads in flight per
// thread, no block barrier inside the loop), takes the exact minima of d and
// d + outmin over the far vertices and a histogram of their keys above B, and
// writes each far vertex as {d, v, inmin} into its own range of the relax-list
// buffer.  After a group barrier, B' = max(T, B + the offset below which about
// `target` far vertices lie).  R2: every block reads back only its own far
// entries and moves those with key <= B' to the queue of phase k.  Every block
// of the group calls it.
constexpr int kNfItems = 8;

__device__ __noinline__ bool nf_refill(const SolveParams& p, const Grp& grp, const Mode& md, uint64_t k, const Shared& sh,
                                       NfView& nv, uint32_t& uses) {
  const GraphView& g = p.g;
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const bool leader = grp.rank == 0 && tid == 0;
  PhaseSlot* S0 = &ctl->slot[k % 4];
  uint32_t* Q = w.q[(k - 1) & 1];
  unsigned int* gh = ctl->hist[uses & 1];
  uint32_t* hist = sh.s_base;
  ulonglong2* tmp = reinterpret_cast<ulonglong2*>(w.sp);
  __shared__ unsigned int s_fcnt;
  // |F| now: read before the first barrier, since R2 of faster blocks changes
  // both counts while slower ones still pick the bin (every block must pick
  // the same B)
  const uint32_t fringe = ldcg_u32(&S0->qcount) + ldcg_u32(&ctl->far_count);
  const unsigned long long bound = nv.bound;
  // this block's vertex range [lo, hi)
  const uint64_t per = ((uint64_t)n + grp.size - 1) / grp.size;
  const uint64_t lo = (uint64_t)grp.rank * per;
  const uint64_t hi = lo + per < n ? lo + per : n;
  if (tid == 0) s_fcnt = 0;
  nf_hist_clear(hist);  // (its barrier also publishes s_fcnt)
  unsigned long long lmin_d = kInf64, lmin_o = kInf64;
  const uint64_t chunk = (uint64_t)nthr * kNfItems;
  for (uint64_t c0 = lo; c0 < hi; c0 += chunk) {
    VRec rr[kNfItems];
#pragma unroll
    for (int j = 0; j < kNfItems; ++j) {
      const uint64_t v = c0 + (uint64_t)j * nthr + tid;
      rr[j].d = kUnexplored;
      if (v < hi) rr[j] = ldcg_vrec(&w.vrec[v]);
    }
#pragma unroll
    for (int j = 0; j < kNfItems; ++j) {
      const bool far = rr[j].d != kUnexplored && (rr[j].d >> 62) == 1u;  // bit 62 set, bit 63 clear
      const unsigned long long d = rr[j].d & ~kFarBit;
      int bin = -1;
      if (far) {
        lmin_d = d < lmin_d ? d : lmin_d;
        if (rr[j].om != kInf32) {
          const unsigned long long x = d + rr[j].om;
          lmin_o = x < lmin_o ? x : lmin_o;
        }
        bin = nf_bin(nf_key(rr[j], d) - bound);
      }
      nf_hist_add(hist, bin);
      const unsigned int fm = __ballot_sync(0xFFFFFFFFu, far);
      if (fm) {
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(&s_fcnt, (unsigned int)__popc(fm));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (far) {
          const uint32_t v = (uint32_t)(c0 + (uint64_t)j * nthr + tid);
          tmp[lo + base + __popc(fm & ((1u << lane) - 1u))] =
              make_ulonglong2(d, (unsigned long long)v | ((unsigned long long)rr[j].im << 32));
        }
      }
    }
  }
  block_min2_to_global(lmin_d, lmin_o, &S0->a_min_d, md.use_out ? &S0->a_min_out : nullptr, sh.red);
  const uint32_t cnt = s_fcnt;  // this block's far entries (the barrier above published it)
  nf_hist_flush(hist, gh);
  if (tid < kNfBins && grp.rank == 0) ctl->hist[(uses + 1) & 1][tid] = 0;
  nf_lists_reset(grp, ctl);
  ++uses;
  if (!grp.sync()) return false;
  const unsigned long long a_d = ldcg_u64(&S0->min_d), f_d = ldcg_u64(&S0->a_min_d);
  const unsigned long long a_o = ldcg_u64(&S0->min_out), f_o = ldcg_u64(&S0->a_min_out);
  const unsigned long long minD = a_d < f_d ? a_d : f_d;
  const unsigned long long minOut = a_o < f_o ? a_o : f_o;
  const unsigned long long T = md.use_out ? minOut : minD;
  const int b = nf_pick_bin(gh, nf_target(p, k, fringe), sh);
  const unsigned long long e = b >= kNfBins ? kNoBound : nf_bin_upper(b);
  unsigned long long B = e >= kNoBound - bound ? kNoBound : bound + e;
  if (B < T) B = T >= kNoBound ? kNoBound : T;
  const NfView v2 = nf_geometry(nv, B, e);
  uint32_t moved = 0;
  const uint32_t rchunk = nthr * kSelItems;
  for (uint32_t c0 = 0; c0 < cnt; c0 += rchunk) {
    uint32_t mv = 0;
    uint32_t vv[kSelItems], app[kSelItems];
#pragma unroll
    for (int j = 0; j < kSelItems; ++j) {
      const uint32_t i = c0 + j * nthr + tid;
      vv[j] = 0;
      app[j] = kNoBucket;
      if (i < cnt) {
        const ulonglong2 t = __ldcg(&tmp[lo + i]);
        const uint32_t im = (uint32_t)(t.y >> 32);
        const unsigned long long key = (im == kInf32 || t.x <= im) ? 0ull : t.x - im;
        vv[j] = (uint32_t)t.y;
        if (key <= B) {
          w.vrec[vv[j]].d = t.x;
          mv |= 1u << j;
        } else if (v2.lists) {
          app[j] = nf_bucket(v2, t.x, im);
        }
      }
    }
    nf_list_append_n<kSelItems>(v2, app, vv);
    uint32_t tm;
    const uint32_t pm = block_exclusive_scan(__popc(mv), sh.scan, &tm);
    if (tid == 0) sh.bases[0] = tm ? atomicAdd(&S0->qcount, tm) : 0u;
    __syncthreads();
    uint32_t slot = (uint32_t)sh.bases[0] + pm;
#pragma unroll
    for (int j = 0; j < kSelItems; ++j)
      if ((mv >> j) & 1u) {
        if (slot < n) Q[slot] = vv[j];
        else atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
        ++slot;
      }
    moved += __popc(mv);
    __syncthreads();
  }
  uint32_t tm;
  block_exclusive_scan(moved, sh.scan, &tm);
  if (tid == 0 && tm) atomicSub(&ctl->far_count, tm);
  if (leader) {  // the exact thresholds of the whole fringe (idempotent with what every block read)
    S0->min_d = minD;
    S0->min_out = minOut;
  }
  __syncthreads();
  if (tid == 0) nv = v2;  // (published to the block by the barrier below)
  return grp.sync();
}

// Pull (far part listed, accumulated T > B): raise B to the end of the bucket
// holding T -- further, bucket by bucket, while the pulled lists hold fewer
// than `target` entries -- and move every far vertex of the pulled lists whose
// key is now <= B' to the queue of phase k (the one thread whose atomicAnd
// clears the far bit moves it; stale and duplicate entries are skipped),
// taking the minima of d and d + outmin over the moved vertices into the
// phase's thresholds.  The vertex attaining T is among them or in the queue,
// every far vertex left has key > B' >= T, so the thresholds stay exact.  Sets
// *need_full (and changes nothing) when a full refill is needed instead: the
// bucket holding T lies past the ring or at or after the lowest bucket with an
// unlisted vertex.  Every block of the group calls it.
__device__ __noinline__ bool nf_pull(const SolveParams& p, const Grp& grp, const Mode& md, uint64_t k, const Shared& sh,
                                     NfView& nv, bool* need_full) {
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = p.g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  PhaseSlot* S0 = &ctl->slot[k % 4];
  uint32_t* Q = w.q[(k - 1) & 1];
  __shared__ uint32_t s_pre[kNfRing + 1];
  __shared__ uint32_t s_nb;
  __shared__ unsigned long long s_newb;
  // inputs no block changes before the barrier below (moved vertices' minima
  // and count go to scratch fields first), so every block computes the same B'
  const unsigned long long T = md.use_out ? ldcg_u64(&S0->min_out) : ldcg_u64(&S0->min_d);
  const uint32_t beyond = ldcg_u32(&ctl->nf_beyond);
  const uint32_t target = nf_target(p, k, kInf32);
  const uint32_t c = nv.cursor;
  if (tid == 0) {
    s_nb = 0;
    const unsigned long long bt = T >= kNoBound ? ~0ull : (T - nv.origin) >> nv.shift;  // T > B >= O
    if (bt <= (unsigned long long)c + kNfRing && bt < beyond) {
      uint32_t c1 = (uint32_t)bt;
      uint64_t tot = 0;
      s_pre[0] = 0;
      for (uint32_t i = c + 1; i <= c1; ++i) {
        const uint32_t f = ldcg_u32(&ctl->nf_cnt[i & (kNfRing - 1)]);
        tot += f < nv.cap ? f : nv.cap;
        s_pre[i - c] = (uint32_t)tot;
      }
      while (tot < target && c1 + 1 <= c + kNfRing && c1 + 1 < beyond) {
        ++c1;
        const uint32_t f = ldcg_u32(&ctl->nf_cnt[c1 & (kNfRing - 1)]);
        tot += f < nv.cap ? f : nv.cap;
        s_pre[c1 - c] = (uint32_t)tot;
      }
      // B' = O + (c1 + 1) * 2^s - 1, if it stays below kNoBound
      const unsigned long long span = (unsigned long long)(c1 + 1);
      if (nv.shift < 62 && span <= ((kNoBound - nv.origin) >> nv.shift)) {
        s_nb = c1 - c;
        s_newb = nv.origin + (span << nv.shift) - 1;
      }
    }
  }
  __syncthreads();
  const uint32_t nb = s_nb;
  if (nb == 0) {
    *need_full = true;
    return true;
  }
  const unsigned long long B1 = s_newb;
  const uint32_t total = s_pre[nb];
  unsigned long long lmin_d = kInf64, lmin_o = kInf64;
  uint32_t moved = 0;
  const uint64_t gwarps = (uint64_t)grp.size * (nthr >> 5);
  for (uint64_t i0 = ((uint64_t)grp.rank * (nthr >> 5) + warp) * 32; i0 < total; i0 += gwarps * 32) {
    const uint32_t i = (uint32_t)i0 + lane;
    bool mv = false;
    uint32_t v = 0;
    if (i < total) {
      uint32_t a = 0, b = nb;  // bucket j (0-based) with s_pre[j] <= i < s_pre[j + 1]
      while (b - a > 1) {
        const uint32_t mid = (a + b) >> 1;
        if (s_pre[mid] <= i) a = mid; else b = mid;
      }
      const uint32_t slot = (c + 1 + a) & (kNfRing - 1);
      v = ldcg_u32(&nv.lists[(uint64_t)slot * nv.cap + (i - s_pre[a])]);
      const VRec r = ldcg_vrec(&w.vrec[v]);
      if ((r.d >> 62) == 1u) {  // far (bit 62 set, bit 63 clear)
        const unsigned long long d = r.d & ~kFarBit;
        if (nf_key(r, d) <= B1) {
          const unsigned long long old = atomicAnd(&w.vrec[v].d, ~kFarBit);
          if (old & kFarBit) {
            mv = true;
            lmin_d = d < lmin_d ? d : lmin_d;
            if (r.om != kInf32) {
              const unsigned long long x = d + r.om;
              lmin_o = x < lmin_o ? x : lmin_o;
            }
          }
        }
      }
    }
    const unsigned int mm = __ballot_sync(0xFFFFFFFFu, mv);
    if (mm) {
      unsigned int base = 0;
      if (lane == 0) base = atomicAdd(&S0->qcount, (unsigned int)__popc(mm));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (mv) {
        const uint32_t slot = base + __popc(mm & ((1u << lane) - 1u));
        if (slot < n) Q[slot] = v;
        else atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
      }
      moved += __popc(mm);
    }
  }
  // the selection step takes min(min_d, a_min_d) and min(min_out, a_min_out)
  block_min2_to_global(lmin_d, lmin_o, &S0->a_min_d, md.use_out ? &S0->a_min_out : nullptr, sh.red);
  if (lane == 0 && moved) atomicAdd(&ctl->nf_moved, moved);
  if (!grp.sync()) return false;
  if (grp.rank == 0) {
    // the pulled slots start over as the buckets past the ring's far end (no
    // block lists a far vertex before the next selection step's barrier)
    if (tid >= 1 && tid <= nb) ctl->nf_cnt[(c + tid) & (kNfRing - 1)] = 0;
    if (tid == 0) {
      const uint32_t mv = ldcg_u32(&ctl->nf_moved);
      if (mv) atomicSub(&ctl->far_count, mv);
      ctl->nf_moved = 0;
    }
  }
  if (tid == 0) {
    nv.bound = B1;
    nv.cursor = c + nb;
  }
  __syncthreads();
  return true;
}

// Initialise, run all phases (switching to solo mode while the fringe is
// small), write the distances.  Every block of the group calls it.
// `p` is the block's shared copy of the parameters (what the out-of-line
// phase steps take); `pk` is the same parameters where the inlined solo
// episodes read them fastest (the kernel parameter bank of a single solve).
__device__ void solve_body(const SolveParams& p, const SolveParams& pk, const Grp& grp_in, unsigned char* smem) {
  const GraphView& g = p.g;
  const SolveWS& w = p.ws;
  Ctl* ctl = w.ctl;
  const uint32_t n = g.n;
  const unsigned int tid = threadIdx.x, nthr = blockDim.x;
  // The group, the shared-memory layout and the mode are the same for every
  // thread of the block: one copy in shared memory, which the steps read
  // through references (per-thread copies would live in local memory).
  __shared__ Grp s_grp;
  __shared__ Shared s_sh;
  __shared__ Mode s_md;
  if (tid == 0) {
    s_grp = grp_in;
    s_sh = carve(smem);
    s_md = mode_of(p);
  }
  __syncthreads();
  const Grp& grp = s_grp;
  const Shared& sh = s_sh;
  const Mode& md = s_md;
  const uint64_t gthreads = (uint64_t)grp.size * nthr;
  const uint64_t gtid = (uint64_t)grp.rank * nthr + tid;
  const bool leader = grp.rank == 0 && tid == 0;
  // Counters and the near/far bound live in shared memory: they are touched
  // once per phase at most, and keeping them out of registers leaves the
  // phase loops more room.
  __shared__ Stats s_st;
  __shared__ NfView s_nv;  // near/far bound and bucket geometry (same in every block)
  Stats& st = s_st;
  if (tid == 0) {
    s_st = Stats{0, 0, 0, 0};
    s_arm_k = ~0ull;
    s_nv.bound = kNoBound;
    s_nv.origin = 0;
    s_nv.shift = 0;
    s_nv.cursor = 0;
    s_nv.cap = w.nf_cap;
    s_nv.lists = w.nf_list;
    s_nv.cnt = ctl->nf_cnt;
    s_nv.beyond = &ctl->nf_beyond;
  }
  if ((p.crit & SSSP_POLICY_LEARNED) && p.policy) {  // (published by the first barrier below)
    float* pw = reinterpret_cast<float*>(smem + kPolicySmemOffset);
    for (int i = tid; i < kPolWeights; i += nthr) pw[i] = __ldg(&p.policy[i]);
  }

  for (uint64_t v = gtid; v < n; v += gthreads) {
    const uint32_t im = __ldg(&g.in_min[v]), om = __ldg(&g.out_min[v]);
    *reinterpret_cast<ulonglong2*>(&w.vrec[v]) =
        make_ulonglong2(kUnexplored, (unsigned long long)im | ((unsigned long long)om << 32));
    w.status[v] = kU;
    if (w.cur_out) w.cur_out[v] = (uint32_t)g.row_off[v];
    if (w.cur_in) w.cur_in[v] = (uint32_t)g.rrow_off[v];
    if (w.settle_phase) w.settle_phase[v] = 0;
  }
  // Small graphs: pull the edge array into L2 now (coalesced, all blocks)
  // instead of paying an HBM round trip on the first touch of every edge.
  if ((uint64_t)g.m * sizeof(uint2) + (uint64_t)n * (sizeof(VRec) + sizeof(uint2)) <= kL2PrefetchBytes) {
    const char* base = reinterpret_cast<const char*>(g.edges);
    const uint64_t lines = ((uint64_t)g.m * sizeof(uint2) + 127) / 128;
    for (uint64_t l = gtid; l < lines; l += gthreads)
      asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(base + l * 128));
  }
  if (leader) {
    for (int j = 0; j < 4; ++j) reset_slot(&ctl->slot[j]);
    ctl->heartbeat = 0;
    ctl->next_phase = 0;
    ctl->resume_relax = 0;
    ctl->far_count = 0;
    ctl->nf_tmp = 0;
  }
  if (grp.rank == 0)
    for (int b = tid; b < 2 * kNfBins; b += nthr) ctl->hist[b / kNfBins][b % kNfBins] = 0;
  if (!grp.sync()) return;
  if (leader) {
    w.vrec[p.source].d = 0;
    w.status[p.source] = kF;
    w.q[0][0] = p.source;
    PhaseSlot* s1 = &ctl->slot[1];
    s1->qcount = 1;
    s1->min_d = 0;
    const uint32_t om = __ldg(&g.out_min[p.source]);
    s1->min_out = om == kInf32 ? kInf64 : (unsigned long long)om;
  }
  if (!grp.sync()) return;

  const bool dense_forced = (p.crit & SSSP_FRONTIER_DENSE) != 0;
  const uint32_t solo_cap = p.solo_max < kSoloCap ? p.solo_max : kSoloCap;
  unsigned int episodes = 0;
  NfView& nv = s_nv;
  uint32_t nf_uses = 0;
  uint64_t k = 1;
  for (;;) {
    PhaseHead h = load_head(ctl, k, nv.bound != kNoBound);
    uint32_t nF = h.nQ;
    uint32_t nf_code = 0;
    if (k > (uint64_t)n + 1) {  // every phase settles a vertex: more phases mean a broken invariant
      if (leader) atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
      break;
    }
    if (md.nearfar) {
      const uint32_t far = h.far;
      if (nF == 0 && far == 0) break;
      const unsigned long long T = md.use_out ? h.min_out : h.min_d;
      if (far > 0 && T > nv.bound) {
        // raise B: from the bucket lists when they cover T, else by a full refill
        bool full = nv.lists == nullptr;
        if (!full && !nf_pull(p, grp, md, k, sh, nv, &full)) return;
        if (full) {
          if (!nf_refill(p, grp, md, k, sh, nv, nf_uses)) return;
          nf_code = kArmNfRefill;
        } else {
          nf_code = kArmNfPull;
        }
        h = load_head(ctl, k, nv.bound != kNoBound);
        nF = h.nQ;
        if (nF == 0) {  // a refill or pull always moves the vertex that attains T
          if (leader) atomicCAS(&ctl->err, 0, (int)SSSP_ERR_INTERNAL);
          break;
        }
      } else if (far == 0 && nv.bound == kNoBound && (uint64_t)nF >= (uint64_t)p.nf_min * grp.size &&
                 (uint64_t)nF * 256 >= (uint64_t)p.nf_share * n) {
        // (with a policy too: while the fringe is split, every phase runs
        // the static sparse arm, see choose_arm)
        if (!nf_split(p, grp, md, k, sh, nv, nf_uses)) return;
        h = load_head(ctl, k, nv.bound != kNoBound);
        nF = h.nQ;
        if (nv.bound != kNoBound) nf_code = kArmNfRefill;
      }
      if (nv.bound != kNoBound) nf_code |= kArmNfActive;
    } else if (nF == 0) {
      break;
    }
    const bool fast_solo = md.fused && !dense_forced && nF <= solo_cap;
    const bool generic_solo = !md.fused && grp.size > 1 && nF <= p.solo_max;
    if (fast_solo || generic_solo) {
      __shared__ unsigned long long s_next;
      __shared__ int s_ok, s_resume;
      bool resume_relax = false;
      if (grp.rank == 0) {
        if (fast_solo) {
          k = solo_episode(pk, md, k, nv, nf_code, smem, st, grp.size > 1, &resume_relax);
        } else {
          // three-step kind: the generic phase on this block alone
          const Grp solo{grp.bar, grp.err, grp.limit, 0, 1};
          while (nF != 0 && nF <= p.solo_max && k <= (uint64_t)n + 1) {
            run_phase(p, solo, md, k, nv, 0u, h, sh, st);
            ++k;
            if (tid == 0) ctl->heartbeat = k;
            h = load_head(ctl, k, nv.bound != kNoBound);
            nF = h.nQ;
          }
        }
        if (grp.size > 1) {
          __syncthreads();
          if (tid == 0) {
            ctl->next_phase = k;
            ctl->resume_relax = resume_relax ? 1u : 0u;
            __threadfence();
            red_release_gpu_add(&ctl->gate, 1u);
          }
          __syncthreads();
        }
      } else {
        if (tid == 0) {
          s_ok = bounded_wait_change(&ctl->gate, episodes, grp.limit, grp.err, &ctl->heartbeat) ? 1 : 0;
          s_next = ld_relaxed_gpu_u64(&ctl->next_phase);
          s_resume = (int)ldcg_u32(&ctl->resume_relax);
        }
        __syncthreads();
        if (!s_ok) return;
        k = s_next;
        resume_relax = s_resume != 0;
        __syncthreads();
      }
      ++episodes;
      if (resume_relax) {
        const Arm arm = arm_for(p, ldcg_u32(&ctl->slot[k % 4].qcount));
        const bool ok = nv.bound != kNoBound ? phase_relax<true>(p, grp, md, arm, k, nv, true, sh, st)
                                             : phase_relax<false>(p, grp, md, arm, k, nv, true, sh, st);
        if (!ok) return;
        ++k;
      }
      continue;
    }
    if (!run_phase(p, grp, md, k, nv, nf_code, h, sh, st)) return;
    ++k;
  }
  if (leader) {
    ctl->phases = st.phases;
    ctl->sum_f = st.sum_f;
    ctl->settled = st.settled;
    ctl->relaxed = st.relaxed;
  }
  if (!grp.sync()) return;
  for (uint64_t v = gtid; v < n; v += gthreads) {
    const unsigned long long d = ldcg_u64(&w.vrec[v].d) & ~kSettledBit;
    w.dist[v] = d == kUnexplored ? kInf64 : d;
  }
}

// The solve's parameters live in shared memory, one copy per block: every
// step reads them through a reference, and a per-thread copy in local memory
// would take L1 space (and L2 traffic) from the graph's data.
__global__ void __launch_bounds__(kThreads, 1) k_solve_grid(SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SolveParams s_p;
  grid_sync_init();
  if (threadIdx.x == 0) s_p = p;
  __syncthreads();
  const Grp grp{&s_p.ws.ctl->bar, &s_p.ws.ctl->err, s_p.wait_ns, blockIdx.x, gridDim.x};
  solve_body(s_p, p, grp, smem);
}

// Batched solver: the grid is split into groups of `bpg` blocks; the first
// block of a group takes the next solve from a device counter (descriptors
// sorted largest first by the host) and the group runs it to the end.
struct BatchItem {
  GraphView g;
  SolveWS ws;
  uint32_t source;
  uint32_t out_index;  // position of this solve in the caller's arrays
};

struct GroupSlot {
  GridBarrier bar;
  unsigned int item;
  unsigned int pad;
};

// Execution tuning of a batch launch (see sssp_tuning).
struct BatchTuning {
  uint32_t solo_max, solo_edges, nf_min, nf_target, nf_share;
};

__global__ void __launch_bounds__(kThreads) k_solve_batch(const BatchItem* items, uint32_t count,
                                                           unsigned int* next, GroupSlot* groups, uint32_t bpg,
                                                           uint32_t crit, BatchTuning tu,
                                                           unsigned long long wait_ns, int* err,
                                                           unsigned long long* phases_out, const float* policy) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int s_item;
  grid_sync_init();
  const unsigned int gidx = blockIdx.x / bpg, rank = blockIdx.x % bpg;
  GroupSlot* gs = &groups[gidx];
  const Grp grp{&gs->bar, err, wait_ns, rank, bpg};
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) gs->item = atomicAdd(next, 1u);
    if (!grp.sync()) return;
    if (threadIdx.x == 0) s_item = ldcg_u32(&gs->item);
    __syncthreads();
    const unsigned int it = s_item;
    if (!grp.sync()) return;  // everyone has read the mailbox before it is reused
    if (it >= count) break;
    __shared__ SolveParams p;  // one copy per block (see k_solve_grid)
    if (threadIdx.x == 0) {
      p.g = items[it].g;
      p.ws = items[it].ws;
      p.source = items[it].source;
      p.crit = crit;
      p.wait_ns = wait_ns;
      p.solo_max = tu.solo_max;
      p.solo_edges = tu.solo_edges;
      p.nf_min = tu.nf_min;
      p.nf_target = tu.nf_target;
      p.nf_share = tu.nf_share;
      p.policy = policy;
    }
    __syncthreads();
    solve_body(p, p, grp, smem);
    if (*(volatile int*)err != 0) return;
    if (rank == 0 && threadIdx.x == 0) {
      const int e = (int)ldcg_u32(reinterpret_cast<const uint32_t*>(&p.ws.ctl->err));
      if (e != 0) atomicCAS(err, 0, e);
      if (phases_out) phases_out[items[it].out_index] = p.ws.ctl->phases;
    }
  }
}

// ---------------------------------------------------------------------------
// host side

namespace {

// Co-resident blocks per SM of the solve kernels, per device ordinal (0 = not
// set up yet).  The first solve on a device sets the kernels' shared-memory
// attribute and measures the occupancy with that device current; the mutex
// makes concurrent first solves from several threads safe.
constexpr int kMaxDevices = 64;
std::atomic<int> g_blocks_per_sm[kMaxDevices];
std::mutex g_attr_mu;

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return dev;
}

sssp_status ensure_kernel_attrs() {
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices) return fail(SSSP_ERR_CUDA, "no usable current CUDA device (ordinal %d)", dev);
  if (g_blocks_per_sm[dev].load() > 0) return SSSP_OK;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (g_blocks_per_sm[dev].load() > 0) return SSSP_OK;
  SSSP_CUDA_TRY(cudaFuncSetAttribute(k_solve_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  SSSP_CUDA_TRY(cudaFuncSetAttribute(k_solve_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  int a = 0, b = 0;
  SSSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_solve_grid, kThreads, kSmemBytes));
  SSSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_solve_batch, kThreads, kSmemBytes));
  const int per_sm = std::min(a, b);
  if (per_sm < 1) return fail(SSSP_ERR_CUDA, "solve kernel cannot be resident");
  g_blocks_per_sm[dev].store(per_sm);
  return SSSP_OK;
}

// Co-resident blocks of the solve kernels on the current device (after
// ensure_kernel_attrs succeeded on it).
uint32_t resident_blocks() {
  const int dev = current_device();
  const int per_sm = dev >= 0 && dev < kMaxDevices ? g_blocks_per_sm[dev].load() : 0;
  return (uint32_t)std::max(1, per_sm * sm_count());
}

sssp_status check_crit(const sssp_graph* g, uint32_t crit) {
  const uint32_t known = SSSP_IN_STATIC | SSSP_OUT_STATIC | SSSP_IN_SIMPLE | SSSP_OUT_SIMPLE | SSSP_IN_FULL |
                         SSSP_OUT_WEAK | SSSP_DIJK | SSSP_APPROX | (63u << SSSP_APPROX_K_SHIFT) |
                         SSSP_FRONTIER_DENSE | SSSP_FRONTIER_AUTO | SSSP_POLICY_LEARNED;
  if ((crit & SSSP_CRITERIA_MASK) == 0) return fail(SSSP_ERR_INVALID_ARG, "criterion mask has no criterion bit");
  if (crit & ~known) return fail(SSSP_ERR_INVALID_ARG, "unknown criterion bits 0x%x", crit & ~known);
  if (crit & SSSP_POLICY_LEARNED) {
    if (!policy_weights()) return fail(SSSP_ERR_UNSUPPORTED, "no phase policy is loaded on this device");
    if ((crit & SSSP_CRITERIA_MASK) != (SSSP_IN_STATIC | SSSP_OUT_STATIC))
      return fail(SSSP_ERR_INVALID_ARG, "SSSP_POLICY_LEARNED takes IN_STATIC | OUT_STATIC as its fallback arm");
  }
  if ((crit & (63u << SSSP_APPROX_K_SHIFT)) && !(crit & SSSP_APPROX))
    return fail(SSSP_ERR_INVALID_ARG, "criterion bits 10..15 (k) are set without SSSP_APPROX");
  if ((crit & (SSSP_IN_SIMPLE | SSSP_IN_FULL | SSSP_APPROX)) && !g->rrow_off)
    return fail(SSSP_ERR_UNSUPPORTED, "IN-SIMPLE, IN (full) and APPROX need a graph built with SSSP_GRAPH_REVERSE");
  return SSSP_OK;
}

// Blocks for a single solve: enough to cover the vertices, at most all
// co-resident blocks.
int blocks_for(uint32_t n) {
  const int max_blocks = (int)resident_blocks();
  const uint64_t want = grid_blocks() ? grid_blocks() : ((uint64_t)n + kVertsPerBlock - 1) / kVertsPerBlock;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)max_blocks));
}

}  // namespace

void workspace_free(Workspace* ws) {
  if (!ws) return;
  dev_free(ws->vrec);
  dev_free(ws->status);
  dev_free(ws->q0);
  dev_free(ws->q1);
  dev_free(ws->sp);
  dev_free(ws->cur_out);
  dev_free(ws->cur_in);
  dev_free(ws->im_dyn);
  dev_free(ws->tile_owner);
  dev_free(ws->im_full);
  dev_free(ws->apx_in);
  dev_free(ws->apx_out);
  dev_free(ws->fresh);
  dev_free(ws->nf_list);
  dev_free(ws->dist);
  dev_free(ws->ctl);
  cudaFreeHost(ws->ctl_host);
  delete ws;
}

sssp_status workspace_alloc(uint32_t n, uint64_t m, bool want_cursors, bool want_dist, Workspace** out) {
  Workspace* ws = new (std::nothrow) Workspace();
  if (!ws) return fail(SSSP_ERR_OUT_OF_MEMORY, "host allocation failed");
  ws->n = n;
  sssp_status s = SSSP_OK;
  ws->nf_cap = std::max<uint32_t>(n / 32, 1024u);
  if ((s = dev_alloc(&ws->vrec, n)) || (s = dev_alloc(&ws->status, n)) || (s = dev_alloc(&ws->q0, n)) ||
      (s = dev_alloc(&ws->q1, n)) || (s = dev_alloc(&ws->sp, n)) || (s = dev_alloc(&ws->ctl, 1)) ||
      (s = dev_alloc(&ws->tile_owner, m / kTile + 2)) ||
      (n <= kNearFarMaxVertices && (s = dev_alloc(&ws->nf_list, (size_t)kNfRing * ws->nf_cap)))) {
    workspace_free(ws);
    return s;
  }
  if (want_cursors && ((s = dev_alloc(&ws->cur_out, n)) || (s = dev_alloc(&ws->cur_in, n)) ||
                       (s = dev_alloc(&ws->im_dyn, n)) || (s = dev_alloc(&ws->im_full, n)) ||
                       (s = dev_alloc(&ws->apx_in, n)) || (s = dev_alloc(&ws->apx_out, n)) ||
                       (s = dev_alloc(&ws->fresh, n)))) {
    workspace_free(ws);
    return s;
  }
  if (want_dist && (s = dev_alloc(&ws->dist, n))) {
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
    sssp_status s = workspace_alloc(g->n, g->m, true, true, &g->ws);
    if (s != SSSP_OK) return s;
  }
  *out = g->ws;
  return SSSP_OK;
}

namespace {

SolveWS ws_view(Workspace* ws, unsigned long long* dist, uint32_t crit, bool has_reverse) {
  SolveWS w;
  memset(&w, 0, sizeof w);
  w.vrec = ws->vrec;
  w.status = ws->status;
  w.q[0] = ws->q0;
  w.q[1] = ws->q1;
  w.sp = ws->sp;
  w.dist = dist ? dist : ws->dist;
  w.cur_out = (crit & (SSSP_OUT_SIMPLE | SSSP_OUT_WEAK | SSSP_APPROX)) ? ws->cur_out : nullptr;
  w.cur_in = ((crit & (SSSP_IN_SIMPLE | SSSP_IN_FULL | SSSP_APPROX | SSSP_POLICY_LEARNED)) && has_reverse)
                 ? ws->cur_in : nullptr;
  w.im_dyn = w.cur_in ? ws->im_dyn : nullptr;
  w.tile_owner = ws->tile_owner;
  w.im_full = ((crit & SSSP_IN_FULL) && has_reverse) ? ws->im_full : nullptr;
  const bool apx = (crit & SSSP_APPROX) && has_reverse;
  w.apx_in = apx ? ws->apx_in : nullptr;
  w.apx_out = apx ? ws->apx_out : nullptr;
  w.fresh = apx ? ws->fresh : nullptr;
  w.nf_list = ws->nf_list;
  w.nf_cap = ws->nf_list ? ws->nf_cap : 0;
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
  TmpBuf<uint32_t> sp_tmp(st);
  TmpBuf<sssp_phase_record> tr_tmp(st);
  if (settle_phase && !sp_dev && (s = sp_tmp.alloc(g->n)) != SSSP_OK) return s;
  if (trace && trace_cap && (s = tr_tmp.alloc(trace_cap)) != SSSP_OK) return s;
  uint32_t* sp_buf = sp_tmp.p;
  sssp_phase_record* tr_buf = tr_tmp.p;

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
  p.solo_max = solo_max();
  p.solo_edges = solo_edges();
  p.nf_min = nearfar_min();
  p.nf_target = nearfar_target();
  p.nf_share = nearfar_share();
  p.policy = (crit & SSSP_POLICY_LEARNED) ? policy_weights() : nullptr;

  const int blocks = blocks_for(g->n);
  SSSP_CUDA_TRY(cudaMemsetAsync(ws->ctl, 0, sizeof(Ctl), st));
  void* args[] = {&p};
  SSSP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_solve_grid, dim3(blocks), dim3(kThreads), args,
                                            kSmemBytes, st));
  SSSP_CUDA_TRY(cudaMemcpyAsync(ws->ctl_host, ws->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  if (!dist_dev)
    SSSP_CUDA_TRY(cudaMemcpyAsync(dist_out, ws->dist, g->n * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  if (sp_buf) SSSP_CUDA_TRY(cudaMemcpyAsync(settle_phase, sp_buf, g->n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
  const Ctl& c = *ws->ctl_host;
  if (c.err != 0) {
    return fail((sssp_status)c.err, c.err == SSSP_ERR_TIMEOUT ? "an in-kernel wait exceeded its limit"
                                                               : "device-side error %d", c.err);
  }
  if (tr_buf) {
    const uint64_t rec = std::min<uint64_t>(trace_cap, c.phases);
    if (rec) SSSP_CUDA_TRY(cudaMemcpy(trace, tr_buf, rec * sizeof(sssp_phase_record), cudaMemcpyDeviceToHost));
  }
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
  uint32_t bpg = 1;                    // blocks per solve
  uint32_t groups = 0;
  uint32_t max_groups = 0;             // gslots allocated (any bpg >= 1 fits)
  BatchItem* items = nullptr;          // device, largest graph first
  unsigned int* next = nullptr;        // device work counter
  GroupSlot* gslots = nullptr;         // device, one per group
  int* err = nullptr;                  // device
  std::vector<Workspace*> ws;          // one per solve
  std::vector<BatchItem> h_items;      // host copy of the descriptors (same order)
  unsigned long long* phases = nullptr;  // device [count], caller order
  bool own_phases = false;
  float* policy = nullptr;             // device copy of the policy network taken at creation
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
  dev_free(b->items);
  dev_free(b->next);
  dev_free(b->gslots);
  dev_free(b->err);
  dev_free(b->policy);
  if (b->own_phases) dev_free(b->phases);
  delete b;
}

// Queue the batch on `st`: reset the work counter, group slots and every
// control block, then one cooperative launch whose groups pull solves.
sssp_status batch_enqueue(sssp_batch* b, cudaStream_t st) {
  SSSP_CUDA_TRY(cudaMemsetAsync(b->next, 0, sizeof(unsigned int), st));
  SSSP_CUDA_TRY(cudaMemsetAsync(b->gslots, 0, b->groups * sizeof(GroupSlot), st));
  SSSP_CUDA_TRY(cudaMemsetAsync(b->err, 0, sizeof(int), st));
  for (Workspace* w : b->ws) SSSP_CUDA_TRY(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl), st));
  const int blocks = (int)(b->groups * b->bpg);
  BatchTuning tu{solo_max(), solo_edges(), nearfar_min(), nearfar_target(), nearfar_share()};
  unsigned long long wait = wait_limit_ns();
  void* args[] = {&b->items, &b->count, &b->next, &b->gslots, &b->bpg, &b->crit, &tu, &wait, &b->err, &b->phases,
                  &b->policy};
  SSSP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_solve_batch, dim3(blocks), dim3(kThreads), args,
                                            kSmemBytes, st));
  return SSSP_OK;
}

sssp_status batch_build(sssp_graph* const* graphs, const uint32_t* sources, uint32_t count, uint32_t crit,
                        uint64_t* const* dist_out, uint64_t* phases_dev, uint32_t bpg, cudaStream_t st,
                        sssp_batch** out) {
  if (!graphs || !sources || !dist_out || count == 0) return fail(SSSP_ERR_INVALID_ARG, "empty or NULL batch");
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
  const uint32_t resident = resident_blocks();
  if (bpg == 0) bpg = 1;
  if (bpg > resident) bpg = resident;
  sssp_batch* b = new (std::nothrow) sssp_batch();
  if (!b) return fail(SSSP_ERR_OUT_OF_MEMORY, "host allocation failed");
  b->count = count;
  b->crit = crit;
  b->bpg = bpg;
  b->groups = std::max<uint32_t>(1, std::min<uint32_t>(count, resident / bpg));
  b->max_groups = std::max<uint32_t>(1, std::min(count, resident));
  // Largest solves first, so the tail of the queue holds the short ones.
  std::vector<uint32_t> order(count);
  for (uint32_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
    return graphs[a]->m + graphs[a]->n > graphs[c]->m + graphs[c]->n;
  });
  std::vector<BatchItem> h(count);
  b->ws.assign(count, nullptr);
  const bool cursors = (crit & (SSSP_IN_SIMPLE | SSSP_OUT_SIMPLE | SSSP_IN_FULL | SSSP_APPROX | SSSP_POLICY_LEARNED)) != 0;
  for (uint32_t k = 0; k < count; ++k) {
    const uint32_t i = order[k];
    if ((s = workspace_alloc(graphs[i]->n, graphs[i]->m, cursors, false, &b->ws[k])) != SSSP_OK) {
      batch_free(b);
      return s;
    }
    h[k].g = view_of(graphs[i]);
    h[k].ws = ws_view(b->ws[k], reinterpret_cast<unsigned long long*>(dist_out[i]), crit, graphs[i]->rrow_off);
    h[k].source = sources[i];
    h[k].out_index = i;
  }
  if ((s = dev_alloc(&b->items, count)) != SSSP_OK || (s = dev_alloc(&b->next, 1)) != SSSP_OK ||
      (s = dev_alloc(&b->gslots, std::max<uint32_t>(1, std::min(count, resident)))) != SSSP_OK ||
      (s = dev_alloc(&b->err, 1)) != SSSP_OK) {
    batch_free(b);
    return s;
  }
  if (phases_dev) {
    b->phases = reinterpret_cast<unsigned long long*>(phases_dev);
  } else {
    b->own_phases = true;
    if ((s = dev_alloc(&b->phases, count)) != SSSP_OK) {
      batch_free(b);
      return s;
    }
  }
  if (crit & SSSP_POLICY_LEARNED) {  // the batch keeps the network loaded now, whatever is loaded later
    if ((s = dev_alloc(&b->policy, kPolWeights)) != SSSP_OK) {
      batch_free(b);
      return s;
    }
    if (cudaMemcpyAsync(b->policy, policy_weights(), kPolWeights * sizeof(float), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess) {
      batch_free(b);
      return fail(SSSP_ERR_CUDA, "copy of the policy network failed");
    }
  }
  if (cudaMemcpyAsync(b->items, h.data(), count * sizeof(BatchItem), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    batch_free(b);
    return fail(SSSP_ERR_CUDA, "copy of batch descriptors failed");
  }
  b->h_items = std::move(h);
  *out = b;
  return SSSP_OK;
}

// Capture the batch's launch (current blocks per solve) in a CUDA graph.
sssp_status batch_capture(sssp_batch* b) {
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
    return fail(SSSP_ERR_CUDA, "stream creation failed");
  sssp_status s = SSSP_OK;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    s = batch_enqueue(b, cap);
    e = cudaStreamEndCapture(cap, &b->graph);
  }
  if (e == cudaSuccess && s == SSSP_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cap);
  if (s != SSSP_OK) return s;
  if (e != cudaSuccess) return fail(SSSP_ERR_CUDA, "CUDA graph capture failed: %s", cudaGetErrorString(e));
  return SSSP_OK;
}

sssp_status batch_status(sssp_batch* b) {
  int e = 0;
  SSSP_CUDA_TRY(cudaMemcpy(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) return fail((sssp_status)e, "device-side error %d in a batched solve", e);
  return SSSP_OK;
}

// Blocks per solve for a batch: as many groups as solves while that keeps
// every resident block busy, fewer (larger) groups for few large solves.
uint32_t choose_bpg(sssp_graph* const* graphs, uint32_t count) {
  const uint32_t resident = resident_blocks();
  uint64_t maxn = 0;
  for (uint32_t i = 0; i < count; ++i) maxn = std::max<uint64_t>(maxn, graphs[i]->n);
  const uint32_t bpg = std::max<uint32_t>(1, resident / std::max<uint32_t>(1, count));
  const uint32_t useful = (uint32_t)std::max<uint64_t>(1, (maxn + kVertsPerBlock - 1) / kVertsPerBlock);
  return std::min(bpg, useful);
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
  sssp_status s = ensure_kernel_attrs();
  if (s != SSSP_OK) return s;
  if (!graphs || count == 0) return fail(SSSP_ERR_INVALID_ARG, "empty or NULL batch");
  for (uint32_t i = 0; i < count; ++i)
    if (!graphs[i]) return fail(SSSP_ERR_INVALID_ARG, "graph %u is NULL", i);
  sssp_batch* b = nullptr;
  const uint32_t bpg = batch_blocks_per_solve() ? batch_blocks_per_solve() : choose_bpg(graphs, count);
  s = batch_build(graphs, sources, count, criterion, dist_out, ph_dev ? phases_out : nullptr, bpg, st, &b);
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
  sssp_status s = ensure_kernel_attrs();
  if (s != SSSP_OK) return s;
  if (!graphs || count == 0) return fail(SSSP_ERR_INVALID_ARG, "empty or NULL batch");
  for (uint32_t i = 0; i < count; ++i)
    if (!graphs[i]) return fail(SSSP_ERR_INVALID_ARG, "graph %u is NULL", i);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  sssp_batch* b = nullptr;
  const uint32_t bpg = batch_blocks_per_solve() ? batch_blocks_per_solve() : choose_bpg(graphs, count);
  s = batch_build(graphs, sources, count, criterion, dist_out, phases_out, bpg, st, &b);
  if (s != SSSP_OK) return s;
  if ((s = batch_capture(b)) != SSSP_OK) {
    batch_free(b);
    return s;
  }
  *out = b;
  return SSSP_OK;
}

extern "C" sssp_status sssp_batch_autotune(sssp_batch* b, void* stream, uint32_t* bpg_out, float* ms_out) {
  clear_error();
  if (!b) return fail(SSSP_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t resident = resident_blocks();
  // candidates: 1, 2, 4, ..., all co-resident blocks, and the batch's own
  // choice.  The search starts at the batch's choice and walks up and then
  // down the ladder; a walk stops at the first candidate that is clearly
  // slower than the best so far (launch time is unimodal in practice, and a
  // launch with many blocks per solve can run for seconds on deep solves).
  // Each candidate's warm-up launch is timed too: one already kWarmCut times
  // the best median gets no timed runs.  Timed runs: kTimed, scored by the
  // median.
  constexpr int kTimed = 3;
  constexpr float kWarmCut = 1.5f, kStopCut = 1.1f, kKeepOwn = 0.97f;
  const uint32_t bpg0 = b->bpg;
  std::vector<uint32_t> ladder;
  for (uint32_t c = 1; c < resident; c *= 2) ladder.push_back(c);
  ladder.push_back(resident);
  if (std::find(ladder.begin(), ladder.end(), bpg0) == ladder.end()) ladder.push_back(bpg0);
  std::sort(ladder.begin(), ladder.end());
  const int i0 = (int)(std::find(ladder.begin(), ladder.end(), bpg0) - ladder.begin());
  cudaEvent_t ev[kTimed + 2];
  for (auto& e : ev) SSSP_CUDA_TRY(cudaEventCreate(&e));
  uint32_t best = bpg0;
  float best_ms = -1.0f, first_ms = -1.0f;
  sssp_status s = SSSP_OK;
  // times candidate c; returns its median launch time, or a negative value if
  // the warm-up alone was kWarmCut times the best median
  auto measure = [&](uint32_t c, float* out) -> sssp_status {
    b->bpg = c;
    b->groups = std::max<uint32_t>(1, std::min<uint32_t>(b->count, resident / c));
    sssp_status r = SSSP_OK;
    if (cudaEventRecord(ev[0], st) != cudaSuccess) return fail(SSSP_ERR_CUDA, "timing a batch launch failed");
    if ((r = batch_enqueue(b, st)) != SSSP_OK) return r;  // warm-up
    if (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess)
      return fail(SSSP_ERR_CUDA, "timing a batch launch failed");
    if ((r = batch_status(b)) != SSSP_OK) return r;
    float warm = 0.0f;
    cudaEventElapsedTime(&warm, ev[0], ev[1]);
    if (best_ms > 0.0f && warm > kWarmCut * best_ms) {
      *out = -1.0f;
      return SSSP_OK;
    }
    for (int i = 0; i < kTimed; ++i) {
      if ((r = batch_enqueue(b, st)) != SSSP_OK) return r;
      if (cudaEventRecord(ev[i + 2], st) != cudaSuccess) return fail(SSSP_ERR_CUDA, "timing a batch launch failed");
    }
    if (cudaEventSynchronize(ev[kTimed + 1]) != cudaSuccess) return fail(SSSP_ERR_CUDA, "timing a batch launch failed");
    if ((r = batch_status(b)) != SSSP_OK) return r;
    float t[kTimed];
    for (int i = 0; i < kTimed; ++i) cudaEventElapsedTime(&t[i], ev[i + 1], ev[i + 2]);
    std::sort(t, t + kTimed);
    *out = t[kTimed / 2];
    return SSSP_OK;
  };
  float ms = 0.0f;
  if ((s = measure(bpg0, &ms)) == SSSP_OK) {
    best_ms = first_ms = ms;
    for (int dir : {+1, -1}) {
      for (int i = i0 + dir; s == SSSP_OK && i >= 0 && i < (int)ladder.size(); i += dir) {
        if ((s = measure(ladder[i], &ms)) != SSSP_OK || ms < 0.0f) break;
        // another candidate replaces the batch's own choice only if clearly faster
        if (ms < best_ms && ms < kKeepOwn * first_ms) {
          best_ms = ms;
          best = ladder[i];
        }
        if (ms > kStopCut * best_ms) break;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  b->bpg = s == SSSP_OK ? best : bpg0;
  b->groups = std::max<uint32_t>(1, std::min<uint32_t>(b->count, resident / b->bpg));
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  const sssp_status sc = batch_capture(b);
  if (s != SSSP_OK) return s;
  if (sc != SSSP_OK) return sc;
  if (bpg_out) *bpg_out = best;
  if (ms_out) *ms_out = best_ms;
  return SSSP_OK;
}

extern "C" sssp_status sssp_batch_trace(sssp_batch* b, uint32_t i, sssp_phase_record* trace, uint64_t trace_cap,
                                        uint32_t* settle_phase, void* stream) {
  clear_error();
  if (!b) return fail(SSSP_ERR_INVALID_ARG, "batch is NULL");
  if (i >= b->count) return fail(SSSP_ERR_INVALID_ARG, "solve %u out of range (batch of %u)", i, b->count);
  if ((trace && trace_cap && !is_device_pointer(trace)) || (settle_phase && !is_device_pointer(settle_phase)))
    return fail(SSSP_ERR_INVALID_ARG, "trace and settle_phase of a batched solve must be device memory");
  uint32_t k = 0;
  while (k < b->count && b->h_items[k].out_index != i) ++k;
  if (k == b->count) return fail(SSSP_ERR_INTERNAL, "solve %u has no descriptor", i);
  BatchItem& it = b->h_items[k];
  it.ws.trace = trace_cap ? trace : nullptr;
  it.ws.trace_cap = trace ? trace_cap : 0;
  it.ws.settle_phase = settle_phase;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SSSP_CUDA_TRY(cudaMemcpyAsync(&b->items[k], &it, sizeof(BatchItem), cudaMemcpyHostToDevice, st));
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
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

// common.cuh -- device primitives and shared structures of the phase engine.
//
// Everything here is plain integer work: 64-bit min-reductions (warp shuffle ->
// block shared memory -> one global atomic), warp-aggregated queue appends, and
// barriers whose waits are bounded by %globaltimer so that a lost block can
// never hang the GPU (the wait gives up, records SSSP_ERR_TIMEOUT and returns).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sssp.h"

namespace sssp {

constexpr uint64_t kInf64 = ~0ull;
constexpr uint32_t kInf32 = 0xFFFFFFFFu;
// Tentative distances in the vertex records: an unexplored vertex holds
// kUnexplored (larger than any distance, which is < (2^31)(2^32) < 2^63); a
// settled vertex has kSettledBit set on top of its final distance, so one load
// of the record tells a relaxation both d and whether the target is settled.
constexpr uint64_t kUnexplored = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t kSettledBit = 0x8000000000000000ull;
// Near/far split of the fringe (n <= 2^30, so every distance is < 2^62): a
// fringe vertex with d(v) - inmin(v) above the bound B is "far" and stores
// d | kFarBit.  Whether the bit is set is a monotone function of d for a fixed
// vertex and B, so the stored words keep the order of the distances and
// atomicMin on them stays exact; every far word is below kUnexplored.
constexpr uint64_t kFarBit = 0x4000000000000000ull;
constexpr uint64_t kNoBound = 0x3FFFFFFFFFFFFFFFull;  // B when no vertex is far
constexpr uint32_t kNearFarMaxVertices = 1u << 30;
constexpr int kNfBins = 256;  // key histogram: 4 bins per octave
// Far vertices are also listed by key bucket: bucket i >= 1 holds keys in
// [O + i * 2^s, O + (i + 1) * 2^s) (O and s fixed by the last split or full
// refill, which set the bound B = O + 2^s - 1).  The near part is every bucket
// up to the cursor c (B = O + (c + 1) * 2^s - 1); buckets c+1 .. c+kNfRing have
// lists in a ring of kNfRing slots, so raising B moves just the listed
// vertices of the buckets it passes.
constexpr uint32_t kNfRing = 64;

// Vertex status: unexplored, fringe (queued), settled (Section 2's U, F, S).
enum : uint8_t { kU = 0, kF = 1, kS = 2 };

// Read-only device view of a preprocessed graph.
struct GraphView {
  uint32_t n;
  uint64_t m;
  const uint64_t* row_off;   // [n+1]
  const uint2* edges;        // [m] {target, cost}, each row sorted by (cost, target)
  const uint32_t* out_min;   // [n] static out-minimum, kInf32 if none
  const uint32_t* in_min;    // [n] static in-minimum, kInf32 if none
  const uint64_t* rrow_off;  // [n+1] in-edge CSR or nullptr
  const uint2* redges;       // [m] {source, cost}, rows sorted by (cost, source)
  const uint2* rowdeg;       // [n] {start of out-row, out-degree} (m < 2^32)
};

// Per-vertex record gathered by the selection and relax steps: the tentative
// distance (with the settled flag, see kSettledBit) and the minima the
// criteria compare it with, in one 16-byte load.  d is updated with 64-bit
// atomicMin / red.min.
//   im: static in-minimum
//   om: static out-minimum
struct __align__(16) VRec {
  unsigned long long d;
  uint32_t im;
  uint32_t om;
};

// Relax-list entry of a settled vertex with out-edges: its distance, the start
// of its out-row and the exclusive prefix of out-degrees over the list.
struct __align__(16) SpEnt {
  unsigned long long d;
  uint32_t row;
  uint32_t base;
};

// Bounded barrier over `size` blocks: one 32-bit counter.  Block 0 of the group
// adds 2^31 - (size - 1), the others add 1, so the top bit flips exactly when
// all have arrived (and the low bits return to their old value).
struct GridBarrier {
  unsigned int count;
  unsigned int pad;
};

// Per-phase accumulators in a ring of 4: slot k % 4 belongs to phase k.  It is
// reset at the top of phase k - 2, filled during phase k - 1 (the thresholds
// and queue of phase k) and phase k (relax list, counts), read in phase k and,
// for the policy's features, in phase k + 1.
struct PhaseSlot {
  unsigned long long min_d;       // fused thresholds of this phase (from phase k-1)
  unsigned long long min_out;
  unsigned long long a_min_d;     // thresholds recomputed by step A (three-step kind)
  unsigned long long a_min_out;
  unsigned long long relax_packed;  // (entries << 32) | edges of this phase's relax list
  unsigned int qcount;            // |F| of this phase
  unsigned int argmin;            // DIJK: lowest id of minimum d
  unsigned int settled_now;       // |S'| of this phase
  unsigned int arm;               // arm the phase ran with (policy index << 8 | dense)
  unsigned long long t_start;     // %globaltimer when the phase began (trace)
  unsigned int fsize;             // |F| at the start of the phase (queue + far part)
  unsigned int pad;
  unsigned long long t_select;    // %globaltimer when the selection step ended (trace)
  unsigned long long a_min_apx;   // APPROX's OUT threshold of this phase
  unsigned int fresh_count;       // vertices that entered F in the relax step before this phase
  unsigned int pad2;
};

// Per-solve control block in device memory (zeroed before each launch).
struct Ctl {
  PhaseSlot slot[4];
  unsigned long long phases, sum_f, settled, relaxed;
  int err;                  // sssp_status recorded by a device-side failure
  unsigned int gate;        // solo mode: bumped when the leader hands back to the group
  unsigned long long heartbeat;  // solo mode: phases done by the leader (progress for waiters)
  unsigned long long next_phase; // solo mode: phase the group resumes at
  unsigned int resume_relax;     // solo mode: 1 = the group resumes at the relax step of next_phase
  unsigned int pad;
  GridBarrier bar;
  // near/far split: far fringe vertices, a work counter and two key
  // histograms (use u fills hist[u & 1] while the other one is cleared)
  unsigned int far_count;
  unsigned int nf_tmp;
  unsigned int hist[2][kNfBins];
  // far-vertex buckets (see kNfRing; the geometry itself is computed alike in
  // every block): the lowest bucket with a far vertex that has no list entry
  // (kInf32 if none: past the ring when it was last lowered, or its list was
  // full), and the list fills
  unsigned int nf_beyond;
  unsigned int nf_moved;  // vertices a pull moved to the queue (summed before the far count drops)
  unsigned int nf_cnt[kNfRing];
};

// Mutable per-solve buffers.
struct SolveWS {
  VRec* vrec;              // [n]
  uint8_t* status;         // [n]
  uint32_t* q[2];          // [n] fringe queues (this phase / next phase)
  SpEnt* sp;               // [n] relax list
  uint32_t* cur_out;       // [n] out-row cursor (dynamic out-minimum), or nullptr
  uint32_t* cur_in;        // [n] in-row cursor (dynamic in-minimum), or nullptr
  uint32_t* im_dyn;        // [n] dynamic in-minimum of fringe vertices (IN-SIMPLE phases), or nullptr
  uint32_t* tile_owner;    // [m / tile + 2] relax-list entry holding each tile's first edge, or nullptr
  unsigned long long* im_full;  // [n] IN (full) minima of fringe vertices (IN_FULL phases), or nullptr
  unsigned long long* apx_in;   // [n] APPROX: approximate IN (full) values, or nullptr
  unsigned long long* apx_out;  // [n] APPROX: approximate OUT-WEAK values
  uint32_t* fresh;              // [n] APPROX: vertices that entered F in the last relax step
  uint32_t* nf_list;            // [kNfRing * nf_cap] far-vertex bucket lists, or nullptr (full refills only)
  uint32_t nf_cap;              // entries per bucket list
  unsigned long long* dist;  // [n] output distances
  Ctl* ctl;
  uint32_t* settle_phase;  // [n] optional
  sssp_phase_record* trace;  // optional
  uint64_t trace_cap;
};

// ---------------------------------------------------------------------------
// PTX helpers

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_min_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// L2-coherent loads of data that other blocks write during the kernel.
__device__ __forceinline__ unsigned long long ldcg_u64(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ldcg_u32(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint8_t ldcg_u8(const uint8_t* p) {
  return (uint8_t)__ldcg(reinterpret_cast<const unsigned char*>(p));
}
__device__ __forceinline__ VRec ldcg_vrec(const VRec* p) {
  const ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  VRec r;
  r.d = x.x;
  r.im = (uint32_t)x.y;
  r.om = (uint32_t)(x.y >> 32);
  return r;
}

__device__ __forceinline__ void red_min_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ SpEnt ldcg_sp(const SpEnt* p) {
  const ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  SpEnt r;
  r.d = x.x;
  r.row = (uint32_t)x.y;
  r.base = (uint32_t)(x.y >> 32);
  return r;
}

// ---------------------------------------------------------------------------
// Reductions and appends

// Minimum of a u64 over a full warp with two 32-bit warp reductions: the
// high words first, then the low words of the lanes that hold that high word.
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
  const uint32_t mh = __reduce_min_sync(0xFFFFFFFFu, hi);
  const uint32_t ml = __reduce_min_sync(0xFFFFFFFFu, hi == mh ? lo : 0xFFFFFFFFu);
  return ((unsigned long long)mh << 32) | ml;
}

// Inclusive prefix sum within a full warp.
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide min of two u64 values, then one atomicMin per block into dst0/dst1
// (skipped for a null destination or an infinite value).  Every thread of the
// block must call it.  scratch: 64 u64 of shared memory.
__device__ __forceinline__ void block_min2_to_global(unsigned long long a, unsigned long long b,
                                                     unsigned long long* dst0, unsigned long long* dst1,
                                                     unsigned long long* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  a = warp_min_u64(a);
  b = warp_min_u64(b);
  if (lane == 0) { scratch[warp] = a; scratch[32 + warp] = b; }
  __syncthreads();
  if (warp == 0) {
    a = lane < nwarps ? scratch[lane] : kInf64;
    b = lane < nwarps ? scratch[32 + lane] : kInf64;
    a = warp_min_u64(a);
    b = warp_min_u64(b);
    if (lane == 0) {
      if (a != kInf64 && dst0) atomicMin(dst0, a);
      if (b != kInf64 && dst1) atomicMin(dst1, b);
    }
  }
  __syncthreads();
}

// Block-wide exclusive prefix sum of one u32 per thread (blockDim.x a
// multiple of 32, at most 1024).  scratch: 33 u32 of shared memory.  Returns
// the thread's exclusive prefix; *total gets the block total (every thread).
// All threads of the block must call it.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* scratch, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t incl = warp_inclusive_scan(v);
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < nwarps ? scratch[lane] : 0u;
    const uint32_t wi = warp_inclusive_scan(w);
    if (lane < nwarps) scratch[lane] = wi - w;
    if (lane == 31) scratch[32] = wi;
  }
  __syncthreads();
  const uint32_t r = scratch[warp] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

// Warp-aggregated append: every lane of a full warp calls it; lanes with
// pred=true get consecutive slots of q (one atomicAdd per warp).  A slot at or
// beyond `cap` is not written; it records SSSP_ERR_INTERNAL in *err instead.
__device__ __forceinline__ void warp_append(uint32_t* q, unsigned int* count, bool pred, uint32_t val,
                                            uint32_t cap, int* err) {
  const unsigned int mask = __ballot_sync(0xFFFFFFFFu, pred);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned int)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (pred) {
    const unsigned int slot = base + __popc(mask & ((1u << lane) - 1u));
    if (slot < cap) q[slot] = val;
    else atomicCAS(err, 0, (int)SSSP_ERR_INTERNAL);
  }
}

// ---------------------------------------------------------------------------
// Bounded waits

// Spin until *addr != old.  Gives up after limit_ns of %globaltimer (recording
// SSSP_ERR_TIMEOUT in *err) or as soon as an error has been recorded.  When
// `progress` is given, the limit counts from the last change of *progress
// (a heartbeat another block advances while it works).  Returns true if the
// value changed.
__device__ __forceinline__ bool bounded_wait_change(const unsigned int* addr, unsigned int old,
                                                    unsigned long long limit_ns, int* err,
                                                    const unsigned long long* progress = nullptr) {
  unsigned long long t0 = globaltimer_ns();
  unsigned long long last = progress ? ld_relaxed_gpu_u64(progress) : 0;
  unsigned int spins = 0;
  while (ld_acquire_gpu(addr) == old) {
    if ((++spins & 15u) == 0) {
      if (*(volatile int*)err != 0) return false;
      const unsigned long long now = globaltimer_ns();
      if (progress) {
        const unsigned long long p = ld_relaxed_gpu_u64(progress);
        if (p != last) { last = p; t0 = now; }
      }
      if (now - t0 > limit_ns) {
        atomicCAS(err, 0, (int)SSSP_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// Group barriers this block has passed (shared memory; zeroed by
// grid_sync_init at kernel entry).  Every block of a group passes the same
// barriers, so the count tells each block what the counter's top bit will be
// once everyone has arrived at the next one.
static __shared__ unsigned int s_bar_gen;

__device__ __forceinline__ void grid_sync_init() {
  if (threadIdx.x == 0) s_bar_gen = 0;
  __syncthreads();
}

// Barrier over the `size` blocks of a group (all co-resident), on a counter
// that is zero when the kernel starts.  rank 0 adds 2^31 - (size - 1), the
// others 1, so the top bit flips exactly when all have arrived: after the g-th
// barrier it equals g & 1.  The arrival is a release reduction (no round trip
// back to the block), so every write of the block before the barrier (ordered
// by the block barrier in front of it) is visible to every block that has seen
// the flip with an acquire load.  Each wait is bounded; returns false in every
// thread of the block if it ran out or an error was recorded.  All threads must
// call it.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int rank, unsigned int size,
                                          unsigned long long limit_ns, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int add = rank == 0 ? 0x80000000u - (size - 1) : 1u;
    const unsigned int want = (++s_bar_gen & 1u) << 31;
    red_release_gpu_add(&bar->count, add);
    int ok = 1;
    unsigned long long t0 = 0;
    unsigned int spins = 0;
    while ((ld_acquire_gpu(&bar->count) & 0x80000000u) != want) {
      if ((++spins & 15u) == 0) {
        if (*(volatile int*)err != 0) { ok = 0; break; }
        const unsigned long long now = globaltimer_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > limit_ns) {
          atomicCAS(err, 0, (int)SSSP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace sssp

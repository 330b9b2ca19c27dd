// common.cuh -- device primitives and shared structures of the phase engine.
//
// Everything here is plain integer work: 64-bit min-reductions (warp shuffle ->
// block shared memory -> one global atomic), warp-aggregated queue appends, and a
// grid barrier whose waits are bounded by %globaltimer so that a lost block can
// never hang the GPU (the wait gives up, records SSSP_ERR_TIMEOUT and returns).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sssp.h"

namespace sssp {

constexpr uint64_t kInf64 = ~0ull;
constexpr uint32_t kInf32 = 0xFFFFFFFFu;

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
};

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// Per-solve control block in device memory.  Slots indexed [2] alternate by
// phase parity so the next phase's slot can be reset while this one is read.
struct Ctl {
  unsigned long long min_d[2];
  unsigned long long min_out[2];
  unsigned int argmin[2];
  unsigned int qcount[2];            // |F| of the queue with that parity
  unsigned long long relax_packed;   // (entries << 32) | edges of this phase's relax list
  unsigned int settled_now;          // |S'| of this phase (including degree-0 vertices)
  unsigned int pad0;
  unsigned long long phases, sum_f, settled, relaxed;
  int err;                           // sssp_status set by a device-side failure
  unsigned int done;
  GridBarrier bar;
  unsigned long long t_phase_start;
};

// Mutable per-solve buffers.
struct SolveWS {
  unsigned long long* d;   // [n] tentative distances
  uint8_t* status;         // [n]
  uint32_t* q[2];          // [n] fringe queues (current / next)
  uint32_t* sp_v;          // [n] relax list: settled vertices with out-degree > 0
  uint32_t* sp_base;       // [n] exclusive prefix of their out-degrees
  uint32_t* cur_out;       // [n] out-row cursor (dynamic out-minimum), or nullptr
  uint32_t* cur_in;        // [n] in-row cursor (dynamic in-minimum), or nullptr
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

// ---------------------------------------------------------------------------
// Reductions and appends

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = t < v ? t : v;
  }
  return v;
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
  return __reduce_add_sync(0xFFFFFFFFu, v);
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

// Block-wide min of two u64 values, then one atomicMin per block into dst0/dst1.
// Every thread of the block must call it.  scratch: 2 * 32 u64 of shared memory.
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
// Bounded wait: spin until *addr != old.  Gives up after limit_ns of
// %globaltimer (recording SSSP_ERR_TIMEOUT in *err) or as soon as another
// thread has recorded an error.  Returns true if the value changed.
__device__ __forceinline__ bool bounded_wait_change(const unsigned int* addr, unsigned int old,
                                                    unsigned long long limit_ns, int* err) {
  const unsigned long long t0 = globaltimer_ns();
  unsigned int spins = 0;
  while (ld_acquire_gpu(addr) == old) {
    if ((++spins & 15u) == 0) {
      if (*(volatile int*)err != 0) return false;
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicCAS(err, 0, (int)SSSP_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// Grid barrier for cooperative (co-resident) launches: one arrival counter and
// a generation word; the last block to arrive resets the counter and bumps the
// generation, the others wait with bounded_wait_change.  Returns false (in
// every thread of the block) if the wait ran out or any block recorded an
// error, so that all blocks leave the solve.  All threads must call it.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int nblocks, unsigned long long limit_ns,
                                          int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = ld_acquire_gpu(&bar->gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      red_release_gpu_add(&bar->gen, 1u);
    } else {
      ok = bounded_wait_change(&bar->gen, g, limit_ns, err) ? 1 : 0;
    }
    __threadfence();
    if (*(volatile int*)err != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace sssp

// engine.h -- launch interface of the persistent phase engine (engine.cu).
#pragma once

#include "common.cuh"

namespace sssp {

constexpr int kThreads = 512;
constexpr int kRelaxItems = 4;
constexpr int kTile = kThreads * kRelaxItems;
constexpr size_t kSmemBytes = 64 * sizeof(unsigned long long)                             // reduction scratch
                              + kTile * (2 * sizeof(uint32_t) + sizeof(unsigned long long))  // relax tile
                              + 16;
// Phases whose fringe has at most this many vertices run on one block alone.
constexpr uint32_t kSoloMaxDefault = 8192;

struct SolveParams {
  GraphView g;
  SolveWS ws;
  uint32_t source;
  uint32_t crit;
  unsigned long long wait_ns;
  uint32_t solo_max;  // 0 disables the single-block mode
  uint32_t pad;
};

// One whole solve per cooperative launch (all blocks co-resident), kThreads
// threads per block, kSmemBytes of dynamic shared memory.
__global__ void __launch_bounds__(kThreads) k_solve_grid(SolveParams p);

}  // namespace sssp

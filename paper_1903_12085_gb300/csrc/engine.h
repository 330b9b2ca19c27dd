// engine.h -- launch interface of the persistent phase engine (engine.cu).
#pragma once

#include "common.cuh"

namespace sssp {

constexpr int kThreads = 512;
constexpr int kRelaxItems = 4;
constexpr int kTile = kThreads * kRelaxItems;
constexpr size_t kSmemBytes = 64 * sizeof(unsigned long long)                             // reduction scratch
                              + kTile * (sizeof(uint32_t) + 2 * sizeof(unsigned long long))  // relax tile
                              + 16;

struct SolveParams {
  GraphView g;
  SolveWS ws;
  uint32_t source;
  uint32_t crit;
  unsigned long long wait_ns;
};

// One whole solve per cooperative launch (all blocks co-resident), kThreads
// threads per block, kSmemBytes of dynamic shared memory.
__global__ void __launch_bounds__(kThreads) k_solve_grid(SolveParams p);

}  // namespace sssp

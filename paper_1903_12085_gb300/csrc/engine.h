// engine.h -- launch interface of the persistent phase engine (engine.cu).
#pragma once

#include "common.cuh"

namespace sssp {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// Grid phases are warp-centric: a warp takes a chunk of 32 * kSelItems fringe
// entries in the selection step and a tile of kTile consecutive edges of the
// relax list in the relax step, with all of a lane's loads in flight together
// and no block barrier inside the loop.
constexpr int kRelaxItems = 4;  // edges per lane per relax tile
constexpr int kSelItems = 4;    // fringe entries per lane per selection chunk
constexpr int kTile = 32 * kRelaxItems;
// A single solve uses one block per this many vertices (at most all co-resident blocks).
constexpr uint32_t kVertsPerBlock = 1024;
// Solo mode (one block runs whole phases with its queues in shared memory):
// fringe and relax list hold at most kSoloCap entries.
constexpr uint32_t kSoloCap = 2048;
constexpr uint32_t kSoloMaxDefault = kSoloCap;     // fringe size limit
constexpr uint32_t kSoloEdgesDefault = 2048;       // relax edges above which a solo phase hands off
constexpr uint32_t kNearFarMinDefault = 8192;      // fringe size per block of the solve at which the near/far split starts
constexpr uint32_t kNearFarShareDefault = 8;       // ... and fringe share of n, in 256ths
constexpr size_t kGridSmem = 66 * sizeof(unsigned long long)                                         // reduction scratch, bases
                             + kWarps * kTile * (2 * sizeof(uint32_t) + sizeof(unsigned long long))  // relax tiles
                             + 36 * sizeof(uint32_t)                                                   // range, scan
                             + kWarps * kNfRing * sizeof(uint32_t);                                    // bucket counts
constexpr size_t kSoloSmem = 64 * sizeof(unsigned long long)                       // reduction scratch
                             + 2 * kSoloCap * sizeof(uint32_t)                     // two queues
                             + kSoloCap * (2 * sizeof(uint32_t) + sizeof(unsigned long long))  // relax list
                             + 16;
// Graphs whose edges and vertex records take at most this many bytes are
// prefetched into L2 when a solve starts (L2 holds 126 MiB).
constexpr uint64_t kL2PrefetchBytes = 96ull << 20;
// The phase layouts share one region; the policy network's weights follow it
// (staged once per solve, so an inference reads shared memory only).
constexpr size_t kPhaseSmem = kGridSmem > kSoloSmem ? kGridSmem : kSoloSmem;
constexpr size_t kPolicySmemOffset = (kPhaseSmem + 15) / 16 * 16;
constexpr size_t kSmemBytes = kPolicySmemOffset + 1476 * sizeof(float);

struct SolveParams {
  GraphView g;
  SolveWS ws;
  uint32_t source;
  uint32_t crit;
  unsigned long long wait_ns;
  uint32_t solo_max;    // largest fringe run by one block alone (0 = never)
  uint32_t solo_edges;  // relax edges above which a solo phase hands off to the group
  uint32_t nf_min;      // fringe size per block of the solve at which the near/far split starts (0 = never)
  uint32_t nf_target;   // near-part size aimed at when the bound is set (0 = automatic)
  uint32_t nf_share;    // the split also needs |F| >= nf_share * n / 256
  const float* policy;  // policy network weights (device) or nullptr
};

// One whole solve per cooperative launch (all blocks co-resident), kThreads
// threads per block, kSmemBytes of dynamic shared memory.
__global__ void __launch_bounds__(kThreads, 1) k_solve_grid(SolveParams p);

}  // namespace sssp

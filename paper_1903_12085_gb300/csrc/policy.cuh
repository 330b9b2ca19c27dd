// policy.cuh -- the per-phase policy network (device side, shared by the engine
// and the training kernels).
//
// A small MLP picks, at the start of every phase, which fused-threshold arm
// the phase runs with:
//   arm 0: IN-STATIC  | OUT-STATIC, sparse fringe queue
//   arm 1: IN-STATIC  | OUT-STATIC, dense scan of the status array
//   arm 2: IN-SIMPLE  | OUT-STATIC, sparse
//   arm 3: IN-SIMPLE  | OUT-STATIC, dense
// Every arm is a disjunction of sound criteria with a complete disjunct, so the
// choice never changes a distance (Section 3); it changes how many vertices a
// phase settles and what the phase costs.  The network maps 8 features of the
// phase-start state to 4 outputs, the predicted log2 of the phase time per
// settled vertex for each arm; the phase takes the arm with the smallest
// prediction if it beats arm 0 by a margin, else arm 0, the paper's IN+OUT
// (IN-SIMPLE arms only when the in-edge CSR exists; a non-finite prediction
// falls back to arm 0; while the engine keeps the fringe split into near and
// far parts, every phase takes arm 0 without asking the network).
//
// Features (float32, all cheap and identical in every block):
//   f0 = log2(1 + |F|) / 24          f4 = log2(1 + k) / 16     (k = phase index)
//   f1 = |F| / n                      f5 = log2(n) / 32
//   f2 = log2(1 + E_prev) / 24        f6 = (m / n) / 32
//   f3 = log2(1 + S_prev) / 24        f7 = S_prev / (1 + F_prev)
// where E_prev, S_prev, F_prev are the relaxed edges, settled vertices and
// fringe size of phase k-1 (0 for k = 1).
// Weights: one float array, W1[8][32], b1[32], W2[32][32], b2[32], W3[32][4],
// b3[4] (row-major, input index first), ReLU after the two hidden layers.
#pragma once

#include <cstdint>

namespace sssp {

constexpr int kPolFeat = 8;
constexpr int kPolHidden = 32;
constexpr int kPolArms = 4;
constexpr int kPolOffW1 = 0;
constexpr int kPolOffB1 = kPolOffW1 + kPolFeat * kPolHidden;
constexpr int kPolOffW2 = kPolOffB1 + kPolHidden;
constexpr int kPolOffB2 = kPolOffW2 + kPolHidden * kPolHidden;
constexpr int kPolOffW3 = kPolOffB2 + kPolHidden;
constexpr int kPolOffB3 = kPolOffW3 + kPolHidden * kPolArms;
constexpr int kPolWeights = kPolOffB3 + kPolArms;  // 1476

__host__ __device__ __forceinline__ void policy_features(float* f, uint64_t nF, uint64_t n, uint64_t m, uint64_t k,
                                                         uint64_t e_prev, uint64_t s_prev, uint64_t f_prev) {
  f[0] = log2f(1.0f + (float)nF) / 24.0f;
  f[1] = (float)nF / (float)n;
  f[2] = log2f(1.0f + (float)e_prev) / 24.0f;
  f[3] = log2f(1.0f + (float)s_prev) / 24.0f;
  f[4] = log2f(1.0f + (float)k) / 16.0f;
  f[5] = log2f((float)n) / 32.0f;
  f[6] = ((float)m / (float)n) / 32.0f;
  f[7] = (float)s_prev / (1.0f + (float)f_prev);
}

// Forward pass by one full warp: lane j owns hidden unit j of both layers.
// Returns the 4 outputs in lanes 0..3 (broadcast to every lane via out[]).
// `w` may point to global or shared memory (plain loads only).
__device__ __forceinline__ void policy_forward_warp(const float* __restrict__ w, const float* f, float* out) {
  const int lane = threadIdx.x & 31;
  float h1 = w[kPolOffB1 + lane];
#pragma unroll
  for (int i = 0; i < kPolFeat; ++i) h1 = fmaf(f[i], w[kPolOffW1 + i * kPolHidden + lane], h1);
  h1 = fmaxf(h1, 0.0f);
  float h2 = w[kPolOffB2 + lane];
#pragma unroll
  for (int i = 0; i < kPolHidden; ++i)
    h2 = fmaf(__shfl_sync(0xFFFFFFFFu, h1, i), w[kPolOffW2 + i * kPolHidden + lane], h2);
  h2 = fmaxf(h2, 0.0f);
#pragma unroll
  for (int a = 0; a < kPolArms; ++a) {
    float y = h2 * w[kPolOffW3 + lane * kPolArms + a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
    out[a] = y + w[kPolOffB3 + a];
  }
}

// Arm with the smallest prediction among the allowed ones (lowest index on
// ties), kept only if it beats arm 0 (the paper's IN+OUT on the sparse queue)
// by kPolicyMargin in log2 time per settled vertex -- the network was fitted on
// smaller graphs, and a switch it is unsure of tends to cost more than it
// saves; arm 0 if any allowed prediction is not finite.
constexpr float kPolicyMargin = 0.35f;

// allow_dense = false (a fringe below n/32) leaves out the dense arms: a scan of
// all n vertices then costs far more per settled vertex than on the small
// training graphs the network has seen.
__device__ __forceinline__ int policy_pick(const float* y, bool allow_simple, bool allow_dense) {
  const int na = allow_simple ? 4 : 2;
  int best = 0;
  for (int a = 0; a < na; ++a) {
    if (!isfinite(y[a])) return 0;
    if ((a & 1) && !allow_dense) continue;
    if (y[a] < y[best]) best = a;
  }
  return y[best] < y[0] - kPolicyMargin ? best : 0;
}

}  // namespace sssp

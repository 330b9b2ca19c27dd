// policy.cu -- storage of the per-phase policy network and its FP32 training
// kernels (forward, backward, Adam).  The network and its features are defined
// in policy.cuh.
//
// Training objective (masked mean squared error): for sample b, taken in a
// phase that ran with arm a_b and cost t_b (log2 of the phase time per settled
// vertex), loss = (1/B) sum_b (y_b[a_b] - t_b)^2 where y_b is the network output.
//
// Backward pass in two kernels:
//   k_mlp_samples      one thread per sample: forward, then the per-sample
//                      pre-activation gradients dZ1, dZ2, dY and the hidden
//                      activations H1, H2 (written to scratch);
//   k_mlp_grad_reduce  one block per weight row: dW[i][j] = sum_b A[b][i] G[b][j]
//                      (A = X, H1 or H2; G = dZ1, dZ2 or dY), bias rows sum G;
//                      fixed summation order, so gradients are deterministic.
#include <mutex>

#include "internal.h"
#include "policy.cuh"

namespace sssp {
namespace {

constexpr int kMaxDevices = 64;
float* g_policy[kMaxDevices] = {nullptr};
std::mutex g_policy_mu;

__global__ void k_mlp_forward(const float* __restrict__ w, const float* __restrict__ x, uint32_t batch,
                              float* __restrict__ y) {
  __shared__ float sw[kPolWeights];
  for (int i = threadIdx.x; i < kPolWeights; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    float h1[kPolHidden], h2[kPolHidden];
    for (int j = 0; j < kPolHidden; ++j) {
      float z = sw[kPolOffB1 + j];
      for (int i = 0; i < kPolFeat; ++i) z = fmaf(x[(size_t)b * kPolFeat + i], sw[kPolOffW1 + i * kPolHidden + j], z);
      h1[j] = fmaxf(z, 0.0f);
    }
    for (int j = 0; j < kPolHidden; ++j) {
      float z = sw[kPolOffB2 + j];
      for (int i = 0; i < kPolHidden; ++i) z = fmaf(h1[i], sw[kPolOffW2 + i * kPolHidden + j], z);
      h2[j] = fmaxf(z, 0.0f);
    }
    for (int a = 0; a < kPolArms; ++a) {
      float z = sw[kPolOffB3 + a];
      for (int i = 0; i < kPolHidden; ++i) z = fmaf(h2[i], sw[kPolOffW3 + i * kPolArms + a], z);
      y[(size_t)b * kPolArms + a] = z;
    }
  }
}

// Per-sample part of the backward pass.  Scratch layout per sample b:
// h1[32] dz1[32] h2[32] dz2[32] dy[4] se[1].
constexpr int kScr = 4 * kPolHidden + kPolArms + 1;

__global__ void k_mlp_samples(const float* __restrict__ w, const float* __restrict__ x,
                              const float* __restrict__ target, const uint32_t* __restrict__ arm, uint32_t batch,
                              float* __restrict__ scr) {
  __shared__ float sw[kPolWeights];
  for (int i = threadIdx.x; i < kPolWeights; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const float inv_b = 1.0f / (float)batch;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    float z1[kPolHidden], h1[kPolHidden], z2[kPolHidden], h2[kPolHidden];
    for (int j = 0; j < kPolHidden; ++j) {
      float z = sw[kPolOffB1 + j];
      for (int i = 0; i < kPolFeat; ++i) z = fmaf(x[(size_t)b * kPolFeat + i], sw[kPolOffW1 + i * kPolHidden + j], z);
      z1[j] = z;
      h1[j] = fmaxf(z, 0.0f);
    }
    for (int j = 0; j < kPolHidden; ++j) {
      float z = sw[kPolOffB2 + j];
      for (int i = 0; i < kPolHidden; ++i) z = fmaf(h1[i], sw[kPolOffW2 + i * kPolHidden + j], z);
      z2[j] = z;
      h2[j] = fmaxf(z, 0.0f);
    }
    const uint32_t a = arm[b] < kPolArms ? arm[b] : 0;
    float ya = sw[kPolOffB3 + a];
    for (int i = 0; i < kPolHidden; ++i) ya = fmaf(h2[i], sw[kPolOffW3 + i * kPolArms + a], ya);
    const float err = ya - target[b];
    const float dya = 2.0f * err * inv_b;  // d loss / d y_b[a]
    float* s = scr + (size_t)b * kScr;
    float dz2[kPolHidden];
    for (int i = 0; i < kPolHidden; ++i) dz2[i] = z2[i] > 0.0f ? sw[kPolOffW3 + i * kPolArms + a] * dya : 0.0f;
    for (int j = 0; j < kPolHidden; ++j) {
      float g = 0.0f;
      for (int i = 0; i < kPolHidden; ++i) g = fmaf(sw[kPolOffW2 + j * kPolHidden + i], dz2[i], g);
      s[kPolHidden + j] = z1[j] > 0.0f ? g : 0.0f;  // dz1
      s[j] = h1[j];
      s[2 * kPolHidden + j] = h2[j];
      s[3 * kPolHidden + j] = dz2[j];
    }
    for (int k = 0; k < kPolArms; ++k) s[4 * kPolHidden + k] = k == (int)a ? dya : 0.0f;
    s[4 * kPolHidden + kPolArms] = err * err * inv_b;
  }
}

// Block r computes gradient row r.  Rows: 0..7 W1 rows (A = x[i], G = dz1),
// 8..39 W2 rows (A = h1[i], G = dz2), 40..71 W3 rows (A = h2[i], G = dy),
// 72 b1 (G = dz1), 73 b2 (G = dz2), 74 b3 (G = dy), 75 loss (sum of se).
__global__ void k_mlp_grad_reduce(const float* __restrict__ x, const float* __restrict__ scr, uint32_t batch,
                                  float* __restrict__ grad, float* __restrict__ loss) {
  const int r = blockIdx.x;
  int cols, gofs, outofs, aidx = -1;
  bool ax = false;
  if (r < 8) { ax = true; aidx = r; gofs = kPolHidden; cols = kPolHidden; outofs = kPolOffW1 + r * kPolHidden; }
  else if (r < 40) { aidx = r - 8; gofs = 3 * kPolHidden; cols = kPolHidden; outofs = kPolOffW2 + (r - 8) * kPolHidden; }
  else if (r < 72) { aidx = 2 * kPolHidden + (r - 40); gofs = 4 * kPolHidden; cols = kPolArms; outofs = kPolOffW3 + (r - 40) * kPolArms; }
  else if (r == 72) { gofs = kPolHidden; cols = kPolHidden; outofs = kPolOffB1; }
  else if (r == 73) { gofs = 3 * kPolHidden; cols = kPolHidden; outofs = kPolOffB2; }
  else if (r == 74) { gofs = 4 * kPolHidden; cols = kPolArms; outofs = kPolOffB3; }
  else { gofs = 4 * kPolHidden + kPolArms; cols = 1; outofs = -1; }
  float acc[kPolHidden];
  for (int c = 0; c < kPolHidden; ++c) acc[c] = 0.0f;
  for (uint32_t b = threadIdx.x; b < batch; b += blockDim.x) {
    const float* s = scr + (size_t)b * kScr;
    const float av = aidx < 0 ? 1.0f : (ax ? x[(size_t)b * kPolFeat + aidx] : s[aidx]);
    for (int c = 0; c < cols; ++c) acc[c] = fmaf(av, s[gofs + c], acc[c]);
  }
  __shared__ float red[256];
  for (int c = 0; c < cols; ++c) {
    red[threadIdx.x] = acc[c];
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (outofs >= 0) grad[outofs + c] = red[0];
      else if (loss) *loss = red[0];
    }
    __syncthreads();
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, uint32_t count, float lr, float beta1, float beta2, float eps,
                       float c1, float c2) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = beta1 * m1[i] + (1.0f - beta1) * gi;
    const float b = beta2 * m2[i] + (1.0f - beta2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

}  // namespace

// Device pointer of the policy loaded on the current device (nullptr if none).
const float* policy_weights() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_policy_mu);
  return g_policy[dev];
}

}  // namespace sssp

using namespace sssp;

extern "C" sssp_status sssp_policy_load(const float* weights, size_t count) {
  clear_error();
  if (!weights || count != (size_t)kPolWeights)
    return fail(SSSP_ERR_INVALID_ARG, "policy needs %d weights (got %zu)", kPolWeights, count);
  int dev = 0;
  SSSP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(SSSP_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_policy_mu);
  if (!g_policy[dev]) {
    sssp_status s = dev_alloc(&g_policy[dev], kPolWeights);
    if (s != SSSP_OK) return s;
  }
  SSSP_CUDA_TRY(cudaMemcpy(g_policy[dev], weights, kPolWeights * sizeof(float),
                           is_device_pointer(weights) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  return SSSP_OK;
}

extern "C" sssp_status sssp_policy_clear(void) {
  int dev = 0;
  SSSP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_policy_mu);
  if (dev >= 0 && dev < kMaxDevices && g_policy[dev]) {
    dev_free(g_policy[dev]);
    g_policy[dev] = nullptr;
  }
  return SSSP_OK;
}

extern "C" sssp_status sssp_policy_features(uint64_t frontier, uint64_t n, uint64_t m, uint64_t phase,
                                            uint64_t edges_prev, uint64_t settled_prev, uint64_t frontier_prev,
                                            float* out8) {
  if (!out8 || n == 0) return fail(SSSP_ERR_INVALID_ARG, "bad feature arguments");
  policy_features(out8, frontier, n, m, phase, edges_prev, settled_prev, frontier_prev);
  return SSSP_OK;
}

extern "C" sssp_status sssp_mlp_forward(const float* w, const float* x, uint32_t batch, float* y, void* stream) {
  clear_error();
  if (!w || !x || !y) return fail(SSSP_ERR_INVALID_ARG, "NULL argument");
  if (batch == 0) return SSSP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = (int)std::min<uint32_t>((batch + 127) / 128, 1024);
  k_mlp_forward<<<blocks, 128, 0, st>>>(w, x, batch, y);
  SSSP_CUDA_TRY(cudaGetLastError());
  return SSSP_OK;
}

extern "C" sssp_status sssp_mlp_backward(const float* w, const float* x, const float* target, const uint32_t* arm,
                                         uint32_t batch, float* grad, float* loss, void* stream) {
  clear_error();
  if (!w || !x || !target || !arm || !grad || batch == 0) return fail(SSSP_ERR_INVALID_ARG, "NULL or empty argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TmpBuf<float> sbuf(st);
  sssp_status s = sbuf.alloc((size_t)batch * kScr);
  if (s != SSSP_OK) return s;
  float* scr = sbuf.p;
  const int blocks = (int)std::min<uint32_t>((batch + 127) / 128, 1024);
  k_mlp_samples<<<blocks, 128, 0, st>>>(w, x, target, arm, batch, scr);
  k_mlp_grad_reduce<<<76, 256, 0, st>>>(x, scr, batch, grad, loss);
  SSSP_CUDA_TRY(cudaGetLastError());
  return SSSP_OK;
}

extern "C" sssp_status sssp_mlp_adam(float* w, const float* grad, float* m1, float* m2, uint32_t count, float lr,
                                     float beta1, float beta2, float eps, uint32_t step, void* stream) {
  clear_error();
  if (!w || !grad || !m1 || !m2 || step == 0) return fail(SSSP_ERR_INVALID_ARG, "bad Adam arguments");
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_adam<<<(int)std::min<uint32_t>((count + 255) / 256, 1024), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      w, grad, m1, m2, count, lr, beta1, beta2, eps, c1, c2);
  SSSP_CUDA_TRY(cudaGetLastError());
  return SSSP_OK;
}

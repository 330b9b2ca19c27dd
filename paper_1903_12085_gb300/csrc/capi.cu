// capi.cu -- error reporting and small utilities behind the C ABI.
#include <atomic>
#include <cstdarg>
#include <cstdio>

#include "engine.h"
#include "internal.h"

namespace sssp {

namespace {
thread_local char t_err[512] = "";
std::atomic<uint64_t> g_wait_ns{2000000000ull};
std::atomic<uint32_t> g_solo_max{kSoloMaxDefault};
std::atomic<uint32_t> g_batch_bpg{0};
std::atomic<uint32_t> g_grid_blocks{0};
std::atomic<uint32_t> g_solo_edges{kSoloEdgesDefault};
std::atomic<uint32_t> g_nf_min{kNearFarMinDefault};
std::atomic<uint32_t> g_nf_target{0};
std::atomic<uint32_t> g_nf_share{kNearFarShareDefault};
}  // namespace

uint32_t solo_max() { return g_solo_max.load(); }
uint32_t batch_blocks_per_solve() { return g_batch_bpg.load(); }
uint32_t grid_blocks() { return g_grid_blocks.load(); }
uint32_t solo_edges() { return g_solo_edges.load(); }
uint32_t nearfar_min() { return g_nf_min.load(); }
uint32_t nearfar_target() { return g_nf_target.load(); }
uint32_t nearfar_share() { return g_nf_share.load(); }

sssp_status fail(sssp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof t_err, fmt, ap);
  va_end(ap);
  return st;
}

void clear_error() { t_err[0] = '\0'; }

uint64_t wait_limit_ns() { return g_wait_ns.load(); }

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int sm_count() {
  // per device ordinal (a process may switch devices between calls)
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cached[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = dev >= 0 && dev < kMaxDevices ? dev : 0;
  int c = cached[slot].load();
  if (c <= 0) {
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    if (c <= 0) c = 1;
    cached[slot].store(c);
  }
  return c;
}

}  // namespace sssp

namespace sssp {
namespace {
// Waits on a word that nothing writes: the wait must run out.
__global__ void k_selftest_wait(const unsigned int* flag, unsigned long long limit_ns, int* err) {
  if (threadIdx.x == 0) bounded_wait_change(flag, 0u, limit_ns, err);
}
}  // namespace
}  // namespace sssp

extern "C" sssp_status sssp_selftest_wait(uint64_t limit_ns) {
  sssp::clear_error();
  unsigned int* words = nullptr;  // [0] the flag nothing writes, [1] the error word
  int herr = 0;
  {
    sssp_status s = sssp::dev_alloc(&words, 2);
    if (s != SSSP_OK) return s;
  }
  cudaError_t e = cudaMemset(words, 0, 2 * sizeof(unsigned int));
  if (e == cudaSuccess) {
    sssp::k_selftest_wait<<<1, 32>>>(words, limit_ns, reinterpret_cast<int*>(words + 1));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&herr, words + 1, sizeof(int), cudaMemcpyDeviceToHost);
  sssp::dev_free(words);
  if (e != cudaSuccess) return sssp::fail(SSSP_ERR_CUDA, "self-test wait: %s", cudaGetErrorString(e));
  if (herr != 0) return sssp::fail((sssp_status)herr, "bounded wait gave up as designed");
  return SSSP_OK;
}

extern "C" sssp_status sssp_set_tuning(const sssp_tuning* t) {
  if (!t) {
    sssp::g_solo_max.store(sssp::kSoloMaxDefault);
    sssp::g_batch_bpg.store(0);
    sssp::g_grid_blocks.store(0);
    sssp::g_solo_edges.store(sssp::kSoloEdgesDefault);
    sssp::g_nf_min.store(sssp::kNearFarMinDefault);
    sssp::g_nf_target.store(0);
    sssp::g_nf_share.store(sssp::kNearFarShareDefault);
    return SSSP_OK;
  }
  sssp::g_solo_max.store(t->solo_max_frontier);
  sssp::g_batch_bpg.store(t->batch_blocks_per_solve);
  sssp::g_grid_blocks.store(t->grid_blocks);
  sssp::g_solo_edges.store(t->solo_max_edges);
  sssp::g_nf_min.store(t->nearfar_min_frontier);
  sssp::g_nf_target.store(t->nearfar_target);
  sssp::g_nf_share.store(t->nearfar_min_share);
  return SSSP_OK;
}

extern "C" sssp_status sssp_get_tuning(sssp_tuning* t) {
  if (!t) return sssp::fail(SSSP_ERR_INVALID_ARG, "tuning is NULL");
  *t = sssp_tuning{};
  t->solo_max_frontier = sssp::g_solo_max.load();
  t->batch_blocks_per_solve = sssp::g_batch_bpg.load();
  t->grid_blocks = sssp::g_grid_blocks.load();
  t->solo_max_edges = sssp::g_solo_edges.load();
  t->nearfar_min_frontier = sssp::g_nf_min.load();
  t->nearfar_target = sssp::g_nf_target.load();
  t->nearfar_min_share = sssp::g_nf_share.load();
  return SSSP_OK;
}

extern "C" sssp_status sssp_set_wait_limit_ns(uint64_t ns) {
  sssp::g_wait_ns.store(ns);
  return SSSP_OK;
}

extern "C" sssp_status sssp_set_l2_fetch_granularity(uint32_t bytes) {
  sssp::clear_error();
  if (bytes != 32 && bytes != 64 && bytes != 128)
    return sssp::fail(SSSP_ERR_INVALID_ARG, "L2 fetch granularity must be 32, 64 or 128 bytes (got %u)", bytes);
  SSSP_CUDA_TRY(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes));
  return SSSP_OK;
}

extern "C" const char* sssp_last_error(void) { return sssp::t_err; }

extern "C" const char* sssp_version(void) { return "sssp-gb300 0.1 (sm_103a)"; }

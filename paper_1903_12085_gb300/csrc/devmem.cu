// devmem.cu -- every device allocation the library makes, counted and
// optionally capped.
//
// Graph handles, solve workspaces, batches, the policy network and the
// temporaries of preprocessing and training all allocate through dev_malloc /
// dev_malloc_async and release through dev_free / dev_free_async.  The layer
// keeps the size of every live block, so sssp_device_memory_in_use reports
// what the library holds, and sssp_set_device_memory_limit makes any request
// that would exceed a cap fail with SSSP_ERR_OUT_OF_MEMORY before cudaMalloc is
// called.  The cap serves callers that share a device with other work, and it
// lets tests force an allocation failure at every point of graph creation,
// solve set-up and batch creation (out-of-memory injection on the host, with no
// GPU fault) and check that every failed call frees what it took.
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace sssp {
namespace {

std::mutex g_mu;
std::unordered_map<void*, size_t> g_live;  // live blocks -> bytes
uint64_t g_in_use = 0;
uint64_t g_limit = 0;  // 0 = no cap

// Reserves `bytes` against the cap (lock held by the caller).
sssp_status reserve_locked(size_t bytes) {
  if (g_limit != 0 && (bytes > g_limit || g_in_use > g_limit - bytes))
    return fail(SSSP_ERR_OUT_OF_MEMORY,
                "device memory limit of %llu bytes reached (%llu in use, %llu requested)",
                (unsigned long long)g_limit, (unsigned long long)g_in_use, (unsigned long long)bytes);
  return SSSP_OK;
}

void record(void* p, size_t bytes) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_live[p] = bytes;
  g_in_use += bytes;
}

void forget(void* p) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) return;
  g_in_use -= it->second;
  g_live.erase(it);
}

}  // namespace

sssp_status dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  bytes = bytes > 0 ? bytes : 1;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    sssp_status s = reserve_locked(bytes);
    if (s != SSSP_OK) return s;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY : SSSP_ERR_CUDA,
                "cudaMalloc of %llu bytes failed: %s", (unsigned long long)bytes, cudaGetErrorString(e));
  }
  record(*p, bytes);
  return SSSP_OK;
}

sssp_status dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  bytes = bytes > 0 ? bytes : 1;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    sssp_status s = reserve_locked(bytes);
    if (s != SSSP_OK) return s;
  }
  const cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY : SSSP_ERR_CUDA,
                "cudaMallocAsync of %llu bytes failed: %s", (unsigned long long)bytes, cudaGetErrorString(e));
  }
  record(*p, bytes);
  return SSSP_OK;
}

void dev_free(void* p) {
  if (!p) return;
  forget(p);
  cudaFree(p);
}

void dev_free_async(void* p, cudaStream_t st) {
  if (!p) return;
  forget(p);
  cudaFreeAsync(p, st);
}

}  // namespace sssp

extern "C" sssp_status sssp_set_device_memory_limit(uint64_t bytes) {
  sssp::clear_error();
  std::lock_guard<std::mutex> lock(sssp::g_mu);
  sssp::g_limit = bytes;
  return SSSP_OK;
}

extern "C" sssp_status sssp_device_memory_in_use(uint64_t* bytes) {
  sssp::clear_error();
  if (!bytes) return sssp::fail(SSSP_ERR_INVALID_ARG, "bytes is NULL");
  std::lock_guard<std::mutex> lock(sssp::g_mu);
  *bytes = sssp::g_in_use;
  return SSSP_OK;
}

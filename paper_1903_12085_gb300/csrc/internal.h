// internal.h -- host-side helpers shared by the library's translation units.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cuda_runtime.h>

#include "sssp.h"
#include "common.cuh"

namespace sssp {

// Records a message for sssp_last_error() and returns `st`.
sssp_status fail(sssp_status st, const char* fmt, ...);
void clear_error();

// Wait limit of in-kernel waits (ns).
uint64_t wait_limit_ns();

// Tuning knobs (sssp_set_tuning): largest fringe run by one block alone, and
// blocks per solve in batches (0 = chosen from the batch).
uint32_t solo_max();
uint32_t batch_blocks_per_solve();
uint32_t grid_blocks();
uint32_t solo_edges();
uint32_t nearfar_min();
uint32_t nearfar_target();
uint32_t nearfar_share();

// Policy network weights loaded on the current device, or nullptr.
const float* policy_weights();

// Returns true if p points to device (or managed) memory.
bool is_device_pointer(const void* p);

// Number of SMs of the current device.
int sm_count();

// Device allocations of the library (devmem.cu): counted, and refused with
// SSSP_ERR_OUT_OF_MEMORY beyond the cap of sssp_set_device_memory_limit.
sssp_status dev_malloc(void** p, size_t bytes);
sssp_status dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p);
void dev_free_async(void* p, cudaStream_t st);

template <class T>
sssp_status dev_alloc(T** p, size_t count) {
  return dev_malloc(reinterpret_cast<void**>(p), (count > 0 ? count : 1) * sizeof(T));
}

template <class T>
sssp_status dev_alloc_async(T** p, size_t count, cudaStream_t st) {
  return dev_malloc_async(reinterpret_cast<void**>(p), (count > 0 ? count : 1) * sizeof(T), st);
}

// A stream-ordered temporary that is released when it goes out of scope, so
// that every early return of a failing call frees it.
template <class T>
struct TmpBuf {
  T* p = nullptr;
  cudaStream_t st;
  explicit TmpBuf(cudaStream_t s) : st(s) {}
  TmpBuf(const TmpBuf&) = delete;
  TmpBuf& operator=(const TmpBuf&) = delete;
  sssp_status alloc(size_t count) { return dev_alloc_async(&p, count, st); }
  void release() {
    dev_free_async(p, st);
    p = nullptr;
  }
  ~TmpBuf() { release(); }
};

}  // namespace sssp

#define SSSP_CUDA_TRY(expr)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      return ::sssp::fail(e_ == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY           \
                                                          : SSSP_ERR_CUDA,                   \
                          "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                          __LINE__);                                                         \
    }                                                                                        \
  } while (0)

namespace sssp {
struct Workspace;
}

// Host-visible graph handle.
struct sssp_graph {
  uint32_t n;
  uint64_t m;
  uint32_t flags;
  int device;
  uint64_t* row_off;   // device [n+1]
  uint2* edges;        // device [m]
  uint32_t* out_min;   // device [n]
  uint32_t* in_min;    // device [n]
  uint2* rowdeg;       // device [n] {row start, out-degree}
  uint64_t* rrow_off;  // device [n+1] or nullptr
  uint2* redges;       // device [m] or nullptr
  // Lazily allocated solve workspace (shared by solves on this handle).
  sssp::Workspace* ws;
};

namespace sssp {

struct Workspace {
  uint32_t n;
  VRec* vrec;
  uint8_t* status;
  uint32_t* q0;
  uint32_t* q1;
  SpEnt* sp;
  uint32_t* cur_out;
  uint32_t* cur_in;
  uint32_t* im_dyn;
  uint32_t* tile_owner;      // [m / kTile + 2] relax-list entry holding the first edge of each tile
  unsigned long long* im_full;  // [n] IN (full) minima (allocated with the cursors)
  unsigned long long* apx_in;   // [n] APPROX values (allocated with the cursors)
  unsigned long long* apx_out;  // [n]
  uint32_t* fresh;              // [n]
  uint32_t* nf_list;            // [kNfRing * nf_cap] far-vertex bucket lists
  uint32_t nf_cap;
  unsigned long long* dist;  // used when the caller's distance buffer is host memory
  Ctl* ctl;
  Ctl* ctl_host;  // pinned mirror for read-back
};

GraphView view_of(const sssp_graph* g);
sssp_status workspace_get(sssp_graph* g, Workspace** out);
sssp_status workspace_alloc(uint32_t n, uint64_t m, bool want_cursors, bool want_dist, Workspace** out);
void workspace_free(Workspace* ws);

}  // namespace sssp

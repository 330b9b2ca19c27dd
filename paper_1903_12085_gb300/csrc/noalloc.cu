// noalloc.cu -- a solve entry point that allocates no memory at all.
//
// Some callers cannot call cudaMalloc at solve time: an application whose
// device memory is reserved up front by its own allocator (a framework's
// caching pool that owns the whole device), or a latency-critical service that
// cannot take cudaMalloc's implicit device-wide synchronisation in its request
// path.  sssp_solve_noalloc serves them: the caller passes the graph and the
// distance buffer in device memory, and every other buffer the solve needs
// lives in one file-scope __device__ array of fixed size, reserved when the
// library's module is loaded onto a GPU and held until the process exits.
//
// The array holds, for at most kNoallocMaxVertices vertices: the vertex
// status bytes, the two fringe queues, the relax list, the per-vertex
// distance/minima records, the static out/in minima, the out-row starts and
// degrees, and the control block.  Every call reuses
// it, so the control block is cleared at the start of each call (everything
// else is written before it is read).  Calls that overlap on the GPU race on
// the array.  The paper has no counterpart of this entry point.
#include <mutex>

#include "engine.h"
#include "internal.h"

namespace sssp {
namespace {

constexpr uint32_t kNoallocMaxVertices = SSSP_NOALLOC_MAX_VERTICES;
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffQ0 = align256(kOffStatus + kNoallocMaxVertices);
constexpr size_t kOffQ1 = align256(kOffQ0 + 4ull * kNoallocMaxVertices);
constexpr size_t kOffSp = align256(kOffQ1 + 4ull * kNoallocMaxVertices);
constexpr size_t kOffVrec = align256(kOffSp + sizeof(SpEnt) * kNoallocMaxVertices);
constexpr size_t kOffOutMin = align256(kOffVrec + sizeof(VRec) * kNoallocMaxVertices);
constexpr size_t kOffInMin = align256(kOffOutMin + 4ull * kNoallocMaxVertices);
constexpr size_t kOffRowDeg = align256(kOffInMin + 4ull * kNoallocMaxVertices);
constexpr size_t kOffCtl = align256(kOffRowDeg + 8ull * kNoallocMaxVertices);
constexpr size_t kScratchBytes = align256(kOffCtl + sizeof(Ctl));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-device set-up: the device address of the array (host code only sees a
// host-side stand-in for the symbol) and the co-resident block count.
struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;
  int max_blocks = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

sssp_status setup_for_current_device(DeviceSetup** out) {
  int dev = 0;
  SSSP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(SSSP_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    SSSP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    SSSP_CUDA_TRY(cudaFuncSetAttribute(k_solve_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    int per_sm = 0;
    SSSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_grid, kThreads, kSmemBytes));
    if (per_sm < 1) return fail(SSSP_ERR_CUDA, "solve kernel cannot be resident");
    s.base = static_cast<unsigned char*>(p);
    s.max_blocks = per_sm * sm_count();
    s.ready = true;
  }
  *out = &s;
  return SSSP_OK;
}

__global__ void k_noalloc_minima_init(uint32_t n, uint32_t* out_min, uint32_t* in_min) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    out_min[v] = kInf32;
    in_min[v] = kInf32;
  }
}

// Static minima over unsorted rows, plus validation of the caller's CSR
// (bad[0] set on an out-of-range target, a reserved cost or bad offsets).
__global__ void k_noalloc_minima(uint32_t n, uint64_t m, const uint64_t* __restrict__ ro,
                                 const uint2* __restrict__ edges, uint32_t* out_min, uint32_t* in_min,
                                 uint2* rowdeg, int* bad) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = warp0; u < n; u += nwarps) {
    const uint64_t b = ro[u], e = ro[u + 1];
    if (e < b || e > m || (u == 0 && b != 0) || (u == n - 1 && e != m)) {
      if (lane == 0) atomicExch(bad, 1);
      continue;
    }
    uint32_t best = kInf32;
    for (uint64_t i = b + lane; i < e; i += 32) {
      const uint2 ed = edges[i];
      if (ed.x >= n || ed.y == kInf32) {
        atomicExch(bad, 1);
        continue;
      }
      best = ed.y < best ? ed.y : best;
      red_min_u32(&in_min[ed.x], ed.y);
    }
    best = __reduce_min_sync(0xFFFFFFFFu, best);
    if (lane == 0) {
      out_min[u] = best;
      rowdeg[u] = make_uint2((uint32_t)b, (uint32_t)(e - b));
    }
  }
}

}  // namespace
}  // namespace sssp

using namespace sssp;

extern "C" sssp_status sssp_solve_noalloc(uint32_t n, uint64_t m, const uint64_t* row_offsets, const uint32_t* edges,
                                          uint32_t source, uint32_t criterion, uint64_t* dist_out,
                                          uint64_t* phases_out, void* stream) {
  clear_error();
  if (n == 0 || n > kNoallocMaxVertices)
    return fail(SSSP_ERR_INVALID_ARG, "sssp_solve_noalloc: n = %u is outside [1, %u]", n, kNoallocMaxVertices);
  if (m >= (1ull << 32)) return fail(SSSP_ERR_INVALID_ARG, "sssp_solve_noalloc: m must be < 2^32");
  if (source >= n) return fail(SSSP_ERR_INVALID_ARG, "source %u >= n = %u", source, n);
  const uint32_t allowed = SSSP_IN_STATIC | SSSP_OUT_STATIC | SSSP_DIJK | SSSP_FRONTIER_DENSE | SSSP_FRONTIER_AUTO;
  if ((criterion & SSSP_CRITERIA_MASK) == 0 || (criterion & ~allowed))
    return fail(SSSP_ERR_UNSUPPORTED, "sssp_solve_noalloc takes IN_STATIC, OUT_STATIC and DIJK only (mask 0x%x)",
                criterion);
  // The solve reads row_offsets and dist_out as 8-byte words and edges as
  // 8-byte {target, cost} pairs: a buffer that does not start on an 8-byte
  // boundary (a tensor slice at an odd 4-byte offset, say) would fault on the
  // GPU, so it is rejected here, before any CUDA call.
  if ((reinterpret_cast<uintptr_t>(row_offsets) & 7u) || (reinterpret_cast<uintptr_t>(edges) & 7u) ||
      (reinterpret_cast<uintptr_t>(dist_out) & 7u))
    return fail(SSSP_ERR_INVALID_ARG, "sssp_solve_noalloc: row_offsets, edges and dist_out must be 8-byte aligned");
  if (!row_offsets || !dist_out || (m > 0 && !edges) || !is_device_pointer(row_offsets) ||
      !is_device_pointer(dist_out) || (m > 0 && !is_device_pointer(edges)))
    return fail(SSSP_ERR_INVALID_ARG, "sssp_solve_noalloc: row_offsets, edges and dist_out must be device memory");
  DeviceSetup* dev = nullptr;
  sssp_status s = setup_for_current_device(&dev);
  if (s != SSSP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = dev->base;
  uint32_t* out_min = reinterpret_cast<uint32_t*>(base + kOffOutMin);
  uint32_t* in_min = reinterpret_cast<uint32_t*>(base + kOffInMin);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kOffCtl);
  uint2* rowdeg = reinterpret_cast<uint2*>(base + kOffRowDeg);
  const uint2* e2 = reinterpret_cast<const uint2*>(edges);

  // Clear the control block (barrier counters, error word), then the minima.
  SSSP_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
  const int blocks = dev->max_blocks;
  k_noalloc_minima_init<<<blocks, 256, 0, st>>>(n, out_min, in_min);
  k_noalloc_minima<<<blocks, 256, 0, st>>>(n, m, row_offsets, e2, out_min, in_min, rowdeg, &ctl->err);
  SSSP_CUDA_TRY(cudaGetLastError());
  int bad = 0;
  SSSP_CUDA_TRY(cudaMemcpyAsync(&bad, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
  if (bad) return fail(SSSP_ERR_INVALID_ARG, "sssp_solve_noalloc: invalid CSR (offsets, targets or costs)");
  SSSP_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));

  SolveParams p;
  memset(&p, 0, sizeof p);
  p.g.n = n;
  p.g.m = m;
  p.g.row_off = row_offsets;
  p.g.edges = e2;
  p.g.out_min = out_min;
  p.g.in_min = in_min;
  p.g.rowdeg = rowdeg;
  p.ws.dist = reinterpret_cast<unsigned long long*>(dist_out);
  p.ws.vrec = reinterpret_cast<VRec*>(base + kOffVrec);
  p.ws.status = base + kOffStatus;
  p.ws.q[0] = reinterpret_cast<uint32_t*>(base + kOffQ0);
  p.ws.q[1] = reinterpret_cast<uint32_t*>(base + kOffQ1);
  p.ws.sp = reinterpret_cast<SpEnt*>(base + kOffSp);
  p.ws.ctl = ctl;
  p.source = source;
  p.crit = criterion;
  p.wait_ns = wait_limit_ns();
  p.solo_max = solo_max();
  p.solo_edges = solo_edges();
  p.nf_min = nearfar_min();
  p.nf_target = nearfar_target();
  p.nf_share = nearfar_share();
  p.policy = nullptr;
  const uint64_t want = ((uint64_t)n + kVertsPerBlock - 1) / kVertsPerBlock;
  const int grid = (int)(want < (uint64_t)blocks ? (want > 0 ? want : 1) : blocks);
  void* args[] = {&p};
  SSSP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_solve_grid, dim3(grid), dim3(kThreads), args, kSmemBytes,
                                            st));
  Ctl h;
  SSSP_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.err != 0)
    return fail((sssp_status)h.err, h.err == SSSP_ERR_TIMEOUT ? "an in-kernel wait exceeded its limit"
                                                               : "device-side error %d", h.err);
  if (phases_out) *phases_out = h.phases;
  return SSSP_OK;
}

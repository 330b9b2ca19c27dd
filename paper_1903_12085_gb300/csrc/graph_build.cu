// graph_build.cu -- sssp_graph_create: device copy and preprocessing of a CSR graph.
//
// Preprocessing follows the paper's Section 5 ("Preprocessing: calculate the
// minimum outgoing/incoming edge for each vertex") together with the presorting
// of Proposition 3 (adjacency lists in increasing cost order, so that a minimum
// over the remaining edges is the first live element):
//   1. every out-row is sorted by (cost, target) -- an edge {target, cost} is
//      stored as one little-endian 64-bit word (cost << 32 | target), so sorting
//      the words sorts the row;
//   2. out_min[u] = cost of the first edge of row u;
//   3. in_min[v]  = red.min.u32 over all edges into v (the paper's atomic-min
//      scatter over out-edges, done with the native 32-bit min);
//   4. optionally the in-edge CSR: counting sort by target, rows then sorted by
//      (cost, source) the same way.
// Row sorts are segmented by length: <= 32 elements one warp (register bitonic
// network), <= 4096 one block (shared-memory bitonic), longer rows are sorted
// in 4096-element chunks and merged pairwise by rank (each element's output
// position = its index in its run + its rank in the sibling run).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace sssp {
namespace {

constexpr int kMidCap = 4096;   // longest row sorted inside one block's shared memory
constexpr int kSortThreads = 512;

__global__ void k_interleave(const uint32_t* __restrict__ col, const uint32_t* __restrict__ w, uint64_t m,
                             unsigned long long* __restrict__ keys) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    keys[i] = ((unsigned long long)w[i] << 32) | col[i];
}

// Device-side validation of the copied inputs.  bad[0] |= 1 offsets, 2 targets, 4 costs.
__global__ void k_validate(const uint64_t* __restrict__ ro, const uint32_t* __restrict__ col,
                           const uint32_t* __restrict__ w, uint32_t n, uint64_t m, unsigned int* bad) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += stride) {
    if (i == 0 && ro[0] != 0) atomicOr(bad, 1u);
    if (i == n && ro[n] != m) atomicOr(bad, 1u);
    if (i < n && ro[i] > ro[i + 1]) atomicOr(bad, 1u);
  }
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
    if (col[i] >= n) atomicOr(bad, 2u);
    if (w[i] == kInf32) atomicOr(bad, 4u);
  }
}

// Split rows by length into three lists.
__global__ void k_classify_rows(const uint64_t* __restrict__ ro, uint32_t n, uint32_t* small, uint32_t* mid,
                                uint32_t* large, unsigned int* counts) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const uint64_t deg = ro[u + 1] - ro[u];
    if (deg <= 1) continue;
    if (deg <= 32) small[atomicAdd(&counts[0], 1u)] = u;
    else if (deg <= kMidCap) mid[atomicAdd(&counts[1], 1u)] = u;
    else {
      large[atomicAdd(&counts[2], 1u)] = u;
      atomicMax(&counts[3], (unsigned int)deg);
    }
  }
}

// One warp per row of length 2..32: bitonic network across lanes.
__global__ void k_sort_small(const uint64_t* __restrict__ ro, const uint32_t* __restrict__ rows,
                             const unsigned int* __restrict__ count, unsigned long long* keys) {
  const unsigned int nrows = *count;
  const int lane = threadIdx.x & 31;
  const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp0; r < nrows; r += nwarps) {
    const uint32_t u = rows[r];
    const uint64_t b = ro[u], deg = ro[u + 1] - b;
    unsigned long long x = lane < (int)deg ? keys[b + lane] : kInf64;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, x, j);
        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
        const bool take_min = (lower == up);
        x = take_min ? (o < x ? o : x) : (o > x ? o : x);
      }
    }
    if (lane < (int)deg) keys[b + lane] = x;
  }
}

// Bitonic sort of `len` (<= kMidCap) keys in shared memory, padded to a power of two.
__device__ void block_bitonic(unsigned long long* s, int len) {
  int p2 = 1;
  while (p2 < len) p2 <<= 1;
  for (int i = threadIdx.x + len; i < p2; i += blockDim.x) s[i] = kInf64;
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = s[i], c = s[l];
          const bool up = (i & k) == 0;
          if ((a > c) == up) { s[i] = c; s[l] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// One block per (row) or per (row chunk of a long row): sort kMidCap-sized pieces.
__global__ void k_sort_mid(const uint64_t* __restrict__ ro, const uint32_t* __restrict__ rows,
                           const unsigned int* __restrict__ count, unsigned long long* keys) {
  __shared__ unsigned long long s[kMidCap];
  const unsigned int nrows = *count;
  for (unsigned int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const uint32_t u = rows[r];
    const uint64_t b = ro[u];
    const int len = (int)(ro[u + 1] - b);
    for (int i = threadIdx.x; i < len; i += blockDim.x) s[i] = keys[b + i];
    block_bitonic(s, len);
    for (int i = threadIdx.x; i < len; i += blockDim.x) keys[b + i] = s[i];
    __syncthreads();
  }
}

// Long rows: sort every kMidCap chunk (block per chunk, grid-strided over rows).
__global__ void k_sort_chunks(const uint64_t* __restrict__ ro, const uint32_t* __restrict__ rows,
                              const unsigned int* __restrict__ count, unsigned long long* keys) {
  __shared__ unsigned long long s[kMidCap];
  const unsigned int nrows = *count;
  for (unsigned int r = 0; r < nrows; ++r) {
    const uint32_t u = rows[r];
    const uint64_t b = ro[u], deg = ro[u + 1] - b;
    const uint64_t nchunks = (deg + kMidCap - 1) / kMidCap;
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
      const uint64_t cb = b + c * kMidCap;
      const int len = (int)(deg - c * kMidCap < (uint64_t)kMidCap ? deg - c * kMidCap : (uint64_t)kMidCap);
      for (int i = threadIdx.x; i < len; i += blockDim.x) s[i] = keys[cb + i];
      block_bitonic(s, len);
      for (int i = threadIdx.x; i < len; i += blockDim.x) keys[cb + i] = s[i];
      __syncthreads();
    }
  }
}

__device__ __forceinline__ uint64_t lower_bound_u64(const unsigned long long* a, uint64_t len,
                                                    unsigned long long x) {
  uint64_t lo = 0, hi = len;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ uint64_t upper_bound_u64(const unsigned long long* a, uint64_t len,
                                                    unsigned long long x) {
  uint64_t lo = 0, hi = len;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One merge pass over every long row: runs of width `width` are merged in
// pairs from src to dst (same offsets).  Equal keys are identical words, so
// ties between runs only need distinct positions (left run first).
__global__ void k_merge_pass(const uint64_t* __restrict__ ro, const uint32_t* __restrict__ rows,
                             const unsigned int* __restrict__ count, const unsigned long long* __restrict__ src,
                             unsigned long long* __restrict__ dst, uint64_t width) {
  const unsigned int nrows = *count;
  const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
  for (unsigned int r = 0; r < nrows; ++r) {
    const uint32_t u = rows[r];
    const uint64_t b = ro[u], deg = ro[u + 1] - b;
    for (uint64_t i = gtid; i < deg; i += gstride) {
      const uint64_t run = i / width, pair0 = (run & ~1ull) * width;
      const uint64_t lstart = pair0, lend = min(deg, pair0 + width);
      const uint64_t rstart = lend, rend = min(deg, pair0 + 2 * width);
      const unsigned long long x = src[b + i];
      uint64_t pos;
      if ((run & 1) == 0) pos = (i - lstart) + lower_bound_u64(src + b + rstart, rend - rstart, x);
      else pos = (i - rstart) + upper_bound_u64(src + b + lstart, lend - lstart, x);
      dst[b + pair0 + pos] = x;
    }
  }
}

__global__ void k_copy_rows(const uint64_t* __restrict__ ro, const uint32_t* __restrict__ rows,
                            const unsigned int* __restrict__ count, const unsigned long long* __restrict__ src,
                            unsigned long long* __restrict__ dst) {
  const unsigned int nrows = *count;
  const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
  for (unsigned int r = 0; r < nrows; ++r) {
    const uint32_t u = rows[r];
    const uint64_t b = ro[u], deg = ro[u + 1] - b;
    for (uint64_t i = gtid; i < deg; i += gstride) dst[b + i] = src[b + i];
  }
}

__global__ void k_fill_u32(uint32_t* p, uint64_t n, uint32_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_out_min(const uint64_t* __restrict__ ro, const uint2* __restrict__ edges, uint32_t n,
                          uint32_t* __restrict__ out_min, uint2* __restrict__ rowdeg) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    out_min[u] = ro[u + 1] > ro[u] ? edges[ro[u]].y : kInf32;
    rowdeg[u] = make_uint2((uint32_t)ro[u], (uint32_t)(ro[u + 1] - ro[u]));
  }
}

__global__ void k_in_min(const uint2* __restrict__ edges, uint64_t m, uint32_t* __restrict__ in_min) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint2 e = edges[i];
    red_min_u32(&in_min[e.x], e.y);
  }
}

__global__ void k_in_degree(const uint2* __restrict__ edges, uint64_t m, uint32_t* __restrict__ indeg) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&indeg[edges[i].x], 1u);
}

// Scatter every edge (u -> v, c) into the in-row of v as {u, c}.
__global__ void k_reverse_scatter(const uint64_t* __restrict__ ro, const uint2* __restrict__ edges, uint32_t n,
                                  const uint64_t* __restrict__ rro, unsigned int* __restrict__ fill,
                                  uint2* __restrict__ redges) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = warp0; u < n; u += nwarps) {
    for (uint64_t e = ro[u] + lane; e < ro[u + 1]; e += 32) {
      const uint2 ed = edges[e];
      const unsigned int slot = atomicAdd(&fill[ed.x], 1u);
      redges[rro[ed.x] + slot] = make_uint2((uint32_t)u, ed.y);
    }
  }
}

// ---- exclusive scan u32[n] -> u64[n+1] (three passes) ----
constexpr int kScanThreads = 1024, kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ uint64_t block_exclusive_scan_u64(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t y = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xFFFFFFFFu, y, o);
      if (lane >= o) y += t;
    }
    warp_tot[lane] = y;
  }
  __syncthreads();
  const uint64_t before = warp > 0 ? warp_tot[warp - 1] : 0;
  *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ tile_sum) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += base + k < n ? in[base + k] : 0;
  uint64_t tot;
  block_exclusive_scan_u64(s, &tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void k_scan_tile_sums(uint64_t* tile_sum, uint64_t ntiles) {
  uint64_t carry = 0;
  for (uint64_t b = 0; b < ntiles; b += blockDim.x) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < ntiles ? tile_sum[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan_u64(v, &tot);
    if (i < ntiles) tile_sum[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint64_t n, const uint64_t* __restrict__ tile_off,
                             uint64_t* __restrict__ out) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) { v[k] = base + k < n ? in[base + k] : 0; s += v[k]; }
  uint64_t tot;
  uint64_t run = tile_off[blockIdx.x] + block_exclusive_scan_u64(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_off[blockIdx.x] + tot;
}

int grid_for(uint64_t items, int threads) {
  const uint64_t want = (items + threads - 1) / threads;
  const uint64_t cap = (uint64_t)sm_count() * 16;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, cap));
}

sssp_status exclusive_scan(const uint32_t* in, uint64_t n, uint64_t* out, cudaStream_t st) {
  const uint64_t ntiles = std::max<uint64_t>(1, (n + kScanTile - 1) / kScanTile);
  TmpBuf<uint64_t> tbuf(st);
  sssp_status s = tbuf.alloc(ntiles);
  if (s != SSSP_OK) return s;
  uint64_t* tiles = tbuf.p;
  k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, tiles);
  k_scan_tile_sums<<<1, kScanThreads, 0, st>>>(tiles, ntiles);
  k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, tiles, out);
  SSSP_CUDA_TRY(cudaGetLastError());
  return SSSP_OK;
}

// Sort every row of (ro, keys) by key.  Temporary buffers come from the stream pool.
sssp_status sort_rows(const uint64_t* ro, uint32_t n, uint64_t m, unsigned long long* keys, cudaStream_t st) {
  if (m == 0) return SSSP_OK;
  TmpBuf<uint32_t> lbuf(st);
  TmpBuf<unsigned int> cbuf(st);
  sssp_status s = SSSP_OK;
  if ((s = lbuf.alloc(3ull * n)) != SSSP_OK || (s = cbuf.alloc(4)) != SSSP_OK) return s;
  uint32_t* lists = lbuf.p;
  unsigned int* counts = cbuf.p;
  SSSP_CUDA_TRY(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned int), st));
  uint32_t *small = lists, *mid = lists + n, *large = lists + 2ull * n;
  k_classify_rows<<<grid_for(n, 256), 256, 0, st>>>(ro, n, small, mid, large, counts);
  k_sort_small<<<grid_for(32ull * n, 256), 256, 0, st>>>(ro, small, counts + 0, keys);
  k_sort_mid<<<sm_count() * 8, kSortThreads, 0, st>>>(ro, mid, counts + 1, keys);
  unsigned int hc[4] = {0, 0, 0, 0};
  SSSP_CUDA_TRY(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st));
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
  const unsigned int nlarge = hc[2];
  const uint64_t maxdeg = hc[3];
  if (nlarge > 0) {
    k_sort_chunks<<<sm_count() * 4, kSortThreads, 0, st>>>(ro, large, counts + 2, keys);
    TmpBuf<unsigned long long> mbuf(st);
    if ((s = mbuf.alloc(m)) != SSSP_OK) return s;
    unsigned long long* tmp = mbuf.p;
    unsigned long long *src = keys, *dst = tmp;
    for (uint64_t width = kMidCap; width < maxdeg; width *= 2) {
      k_merge_pass<<<sm_count() * 4, 256, 0, st>>>(ro, large, counts + 2, src, dst, width);
      std::swap(src, dst);
    }
    if (src != keys) k_copy_rows<<<sm_count() * 4, 256, 0, st>>>(ro, large, counts + 2, src, keys);
    SSSP_CUDA_TRY(cudaGetLastError());
  }
  SSSP_CUDA_TRY(cudaGetLastError());
  return SSSP_OK;
}

// Host inputs: the offsets' two ends here, before anything is allocated; an
// edgeless graph's offsets too (all zero).  Everything else is checked by
// k_validate on the device copies (a failing build frees what it took).
sssp_status validate_host(uint32_t n, uint64_t m, const uint64_t* ro) {
  if (ro[0] != 0 || ro[n] != m) return fail(SSSP_ERR_INVALID_ARG, "row_offsets[0] must be 0 and row_offsets[n] = m");
  if (m == 0)
    for (uint32_t u = 0; u < n; ++u)
      if (ro[u] > ro[u + 1]) return fail(SSSP_ERR_INVALID_ARG, "row_offsets decrease at vertex %u", u);
  return SSSP_OK;
}

void free_graph(sssp_graph* g) {
  if (!g) return;
  if (g->ws) workspace_free(g->ws);
  dev_free(g->row_off);
  dev_free(g->edges);
  dev_free(g->out_min);
  dev_free(g->in_min);
  dev_free(g->rowdeg);
  dev_free(g->rrow_off);
  dev_free(g->redges);
  delete g;
}

sssp_status build(sssp_graph* g, const uint64_t* ro_in, const uint32_t* col_in, const uint32_t* w_in, int on_dev,
                  cudaStream_t st) {
  const uint32_t n = g->n;
  const uint64_t m = g->m;
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  sssp_status s = SSSP_OK;
  if ((s = dev_alloc(&g->row_off, n + 1ull)) != SSSP_OK || (s = dev_alloc(&g->edges, m)) != SSSP_OK ||
      (s = dev_alloc(&g->out_min, n)) != SSSP_OK || (s = dev_alloc(&g->in_min, n)) != SSSP_OK ||
      (s = dev_alloc(&g->rowdeg, n)) != SSSP_OK)
    return s;
  SSSP_CUDA_TRY(cudaMemcpyAsync(g->row_off, ro_in, (n + 1ull) * sizeof(uint64_t), kind, st));
  if (m > 0) {
    TmpBuf<uint32_t> tbuf(st);
    if ((s = tbuf.alloc(2 * m)) != SSSP_OK) return s;
    uint32_t* tmp = tbuf.p;
    SSSP_CUDA_TRY(cudaMemcpyAsync(tmp, col_in, m * sizeof(uint32_t), kind, st));
    SSSP_CUDA_TRY(cudaMemcpyAsync(tmp + m, w_in, m * sizeof(uint32_t), kind, st));
    {  // host inputs too: a device pass over the copies replaces a serial host loop over every edge
      TmpBuf<unsigned int> bbuf(st);
      if ((s = bbuf.alloc(1)) != SSSP_OK) return s;
      unsigned int* bad = bbuf.p;
      unsigned int hbad = 0;
      SSSP_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned int), st));
      k_validate<<<grid_for(m + n, 256), 256, 0, st>>>(g->row_off, tmp, tmp + m, n, m, bad);
      SSSP_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
      SSSP_CUDA_TRY(cudaStreamSynchronize(st));
      if (hbad) {
        return fail(SSSP_ERR_INVALID_ARG, "CSR is invalid (%s%s%s)", (hbad & 1) ? "offsets " : "",
                    (hbad & 2) ? "targets >= n " : "", (hbad & 4) ? "the reserved cost 0xFFFFFFFF" : "");
      }
    }
    k_interleave<<<grid_for(m, 256), 256, 0, st>>>(tmp, tmp + m, m, reinterpret_cast<unsigned long long*>(g->edges));
    SSSP_CUDA_TRY(cudaGetLastError());
  } else if (on_dev) {
    uint64_t h[2] = {0, 0};
    SSSP_CUDA_TRY(cudaMemcpyAsync(h, ro_in, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    SSSP_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0] != 0) return fail(SSSP_ERR_INVALID_ARG, "device CSR is invalid (offsets)");
  }
  s = sort_rows(g->row_off, n, m, reinterpret_cast<unsigned long long*>(g->edges), st);
  if (s != SSSP_OK) return s;
  k_out_min<<<grid_for(n, 256), 256, 0, st>>>(g->row_off, g->edges, n, g->out_min, g->rowdeg);
  k_fill_u32<<<grid_for(n, 256), 256, 0, st>>>(g->in_min, n, kInf32);
  if (m > 0) k_in_min<<<grid_for(m, 256), 256, 0, st>>>(g->edges, m, g->in_min);
  SSSP_CUDA_TRY(cudaGetLastError());
  if (g->flags & SSSP_GRAPH_REVERSE) {
    if ((s = dev_alloc(&g->rrow_off, n + 1ull)) != SSSP_OK || (s = dev_alloc(&g->redges, m)) != SSSP_OK) return s;
    TmpBuf<uint32_t> cbuf(st);
    if ((s = cbuf.alloc(n)) != SSSP_OK) return s;
    uint32_t* cnt = cbuf.p;
    SSSP_CUDA_TRY(cudaMemsetAsync(cnt, 0, n * sizeof(uint32_t), st));
    if (m > 0) k_in_degree<<<grid_for(m, 256), 256, 0, st>>>(g->edges, m, cnt);
    s = exclusive_scan(cnt, n, g->rrow_off, st);
    if (s != SSSP_OK) return s;
    SSSP_CUDA_TRY(cudaMemsetAsync(cnt, 0, n * sizeof(uint32_t), st));
    if (m > 0)
      k_reverse_scatter<<<grid_for(32ull * n, 256), 256, 0, st>>>(g->row_off, g->edges, n, g->rrow_off, cnt,
                                                                   g->redges);
    SSSP_CUDA_TRY(cudaGetLastError());
    cbuf.release();
    s = sort_rows(g->rrow_off, n, m, reinterpret_cast<unsigned long long*>(g->redges), st);
    if (s != SSSP_OK) return s;
  }
  SSSP_CUDA_TRY(cudaStreamSynchronize(st));
  return SSSP_OK;
}

}  // namespace

GraphView view_of(const sssp_graph* g) {
  GraphView v;
  v.n = g->n;
  v.m = g->m;
  v.row_off = g->row_off;
  v.edges = g->edges;
  v.out_min = g->out_min;
  v.in_min = g->in_min;
  v.rowdeg = g->rowdeg;
  v.rrow_off = g->rrow_off;
  v.redges = g->redges;
  return v;
}

}  // namespace sssp

using namespace sssp;

extern "C" sssp_status sssp_graph_create(uint32_t n, uint64_t m, const uint64_t* row_offsets, const uint32_t* col_idx,
                                         const uint32_t* weights, int inputs_on_device, uint32_t build_flags,
                                         void* stream, sssp_graph** out) {
  clear_error();
  if (!out) return fail(SSSP_ERR_INVALID_ARG, "out is NULL");
  if (n == 0 || n >= (1u << 31)) return fail(SSSP_ERR_INVALID_ARG, "n must satisfy 1 <= n < 2^31 (got %u)", n);
  if (m >= (1ull << 32)) return fail(SSSP_ERR_INVALID_ARG, "m must be < 2^32");
  if (!row_offsets || (m > 0 && (!col_idx || !weights))) return fail(SSSP_ERR_INVALID_ARG, "NULL CSR array");
  if (build_flags & ~(uint32_t)SSSP_GRAPH_REVERSE) return fail(SSSP_ERR_INVALID_ARG, "unknown build flag");
  if (!inputs_on_device) {
    sssp_status s = validate_host(n, m, row_offsets);
    if (s != SSSP_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  sssp_graph* g = new (std::nothrow) sssp_graph();
  if (!g) return fail(SSSP_ERR_OUT_OF_MEMORY, "host allocation failed");
  g->n = n;
  g->m = m;
  g->flags = build_flags;
  cudaGetDevice(&g->device);
  sssp_status s = build(g, row_offsets, col_idx, weights, inputs_on_device, st);
  if (s != SSSP_OK) {
    cudaStreamSynchronize(st);
    free_graph(g);
    return s;
  }
  *out = g;
  return SSSP_OK;
}

extern "C" void sssp_graph_destroy(sssp_graph* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  free_graph(g);
}

extern "C" sssp_status sssp_graph_info(const sssp_graph* g, uint32_t* n, uint64_t* m, uint32_t* flags) {
  if (!g) return fail(SSSP_ERR_INVALID_ARG, "graph is NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (flags) *flags = g->flags;
  return SSSP_OK;
}

extern "C" sssp_status sssp_graph_device_arrays(const sssp_graph* g, const uint64_t** row_off, const uint32_t** edges,
                                                const uint32_t** out_min, const uint32_t** in_min,
                                                const uint64_t** rrow_off, const uint32_t** redges) {
  if (!g) return fail(SSSP_ERR_INVALID_ARG, "graph is NULL");
  if (row_off) *row_off = g->row_off;
  if (edges) *edges = reinterpret_cast<const uint32_t*>(g->edges);
  if (out_min) *out_min = g->out_min;
  if (in_min) *in_min = g->in_min;
  if (rrow_off) *rrow_off = g->rrow_off;
  if (redges) *redges = reinterpret_cast<const uint32_t*>(g->redges);
  return SSSP_OK;
}

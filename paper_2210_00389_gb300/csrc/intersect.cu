// Intersection + count-once rule (a4) and reduction (a5); plain count (a6).
//
// Cover path, Alg. 1 and Thm. 2 of Bader et al., "Triangle
// Counting Through Cover-Edges": for each cover edge (u, v), u < v,
// c_uv = |{ w in N(u) ∩ N(v) : L(w) != L(u)  or  w > v }|, T = sum c_uv.
// Plain path, the direction-oriented edge iterator (Sec. I, Sec. V-A): for
// each edge u < v, |{ w in N(u) ∩ N(v) : w > v }|.
//
// Intersection by binary search of the shorter list in the longer one
// (Sec. V-A, "binary-search algorithms"), one warp per edge: every lane
// takes elements of the short list.  Warp-shuffle reduction to one 64-bit
// atomic per block; counts are exact integers, so the order is irrelevant.
#include "internal.cuh"

namespace tc {

constexpr int kIsThreads = 256;

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* __restrict__ a, int64_t len,
                                                   uint32_t x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  return x;
}

__device__ __forceinline__ void block_add(unsigned long long x, unsigned long long* out) {
  __shared__ unsigned long long ws[kIsThreads / 32];
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    x = lane < kIsThreads / 32 ? ws[lane] : 0ull;
    x = warp_sum(x);
    if (lane == 0 && x) atomicAdd(out, x);
  }
}

// One warp per cover edge.
__global__ void __launch_bounds__(kIsThreads)
k_cover_bsearch(const uint2* __restrict__ H, int64_t nh, const int64_t* __restrict__ off,
                const uint32_t* __restrict__ cols, const uint32_t* __restrict__ L,
                uint32_t* __restrict__ per_edge, unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long acc = 0, matches = 0;
  for (int64_t i = warp; i < nh; i += nwarps) {
    const uint2 e = H[i];
    const uint32_t u = e.x, v = e.y;
    const int64_t bu = off[u], du = off[u + 1] - bu;
    const int64_t bv = off[v], dv = off[v + 1] - bv;
    const uint32_t* A = cols + (du <= dv ? bu : bv);
    const uint32_t* B = cols + (du <= dv ? bv : bu);
    const int64_t la = du <= dv ? du : dv, lb = du <= dv ? dv : du;
    const uint32_t lvl = L[u];
    unsigned c = 0, m = 0;
    for (int64_t k = lane; k < la; k += 32) {
      const uint32_t x = A[k];
      const int64_t p = lower_bound_u32(B, lb, x);
      if (p < lb && B[p] == x) {
        ++m;
        if (L[x] != lvl || x > v) ++c;
      }
    }
    unsigned long long cs = warp_sum(c);
    matches += m;
    if (lane == 0) {
      if (per_edge) per_edge[i] = (uint32_t)cs;
      acc += cs;
    }
  }
  block_add(acc, &ctrl[kCtrlCount]);
  __syncthreads();
  block_add(matches, &ctrl[kCtrlMatches]);
}

// ustart[v] = index (into cols) of the first neighbour of v greater than v.
__global__ void k_upper_start(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                              uint32_t n, int64_t* __restrict__ ustart) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; v < (int64_t)n; v += stride) {
    const int64_t b = off[v];
    ustart[v] = b + lower_bound_u32(cols + b, off[v + 1] - b, (uint32_t)v + 1u);
  }
}

// One warp per CSR entry (u, v) with u < v: |N(u) ∩ N(v) ∩ (v, inf)|, where
// both suffixes start after v (N(u) right after the entry itself).
__global__ void __launch_bounds__(kIsThreads)
k_plain_bsearch(const uint32_t* __restrict__ erow, int64_t nnz, const int64_t* __restrict__ off,
                const uint32_t* __restrict__ cols, const int64_t* __restrict__ ustart,
                unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long acc = 0;
  for (int64_t e = warp; e < nnz; e += nwarps) {
    const uint32_t u = erow[e], v = cols[e];
    if (u >= v) continue;
    const int64_t au = e + 1, du = off[u + 1] - au;
    const int64_t av = ustart[v], dv = off[v + 1] - av;
    const uint32_t* A = cols + (du <= dv ? au : av);
    const uint32_t* B = cols + (du <= dv ? av : au);
    const int64_t la = du <= dv ? du : dv, lb = du <= dv ? dv : du;
    unsigned c = 0;
    for (int64_t k = lane; k < la; k += 32) {
      const uint32_t x = A[k];
      const int64_t p = lower_bound_u32(B, lb, x);
      if (p < lb && B[p] == x) ++c;
    }
    acc += c;
  }
  block_add(acc, &ctrl[kCtrlCount]);
}

int count_cover(tc_graph* g, uint32_t* per_edge_out, uint64_t* total) {
  cudaStream_t s = g->stream;
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlCount, 0, sizeof(unsigned long long), s));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlMatches, 0, sizeof(unsigned long long), s));
  cudaEventRecord(g->ev[4], s);
  if (g->num_cover > 0) {
    launch(k_cover_bsearch, grid_for(g->num_cover * 32, kIsThreads, 8), kIsThreads, 0, s, 
        g->cover.p, g->num_cover, g->off, g->cols, g->levels.p, per_edge_out, g->ctrl.p);
    TC_CUDA(cudaGetLastError());
  }
  cudaEventRecord(g->ev[5], s);
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  *total = g->ctrl_host[kCtrlCount];
  g->stats.matches = g->ctrl_host[kCtrlMatches];
  g->stats.edges_intersected = g->num_cover;
  cudaEventElapsedTime(&g->stats.ms_intersect, g->ev[4], g->ev[5]);
  return TC_OK;
}

int count_plain(tc_graph* g, uint64_t* total) {
  cudaStream_t s = g->stream;
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlCount, 0, sizeof(unsigned long long), s));
  if (g->nnz > 0) {
    DevBuf<int64_t> ustart;
    TC_TRY(ustart.alloc(g->n, s));
    launch(k_upper_start, grid_for(g->n, kIsThreads), kIsThreads, 0, s, g->off, g->cols, g->n,
                                                                     ustart.p);
    cudaEventRecord(g->ev[4], s);
    launch(k_plain_bsearch, grid_for(g->nnz * 32, kIsThreads, 8), kIsThreads, 0, s, 
        g->erow.p, g->nnz, g->off, g->cols, ustart.p, g->ctrl.p);
    TC_CUDA(cudaGetLastError());
    cudaEventRecord(g->ev[5], s);
  }
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  *total = g->ctrl_host[kCtrlCount];
  g->stats.edges_intersected = g->nnz / 2;
  if (g->nnz > 0) cudaEventElapsedTime(&g->stats.ms_intersect, g->ev[4], g->ev[5]);
  return TC_OK;
}

}  // namespace tc

// Cover-edge extraction (a2): Thm. 1 and Alg. 1 of Bader et al.,
// "Triangle Counting Through Cover-Edges".  The horizontal edges, both ends
// on one BFS level, form a cover-edge set; each is kept once as (u, v) with
// u < v, in CSR order (ascending u, then v).
//
// Stream compaction over the CSR entries: pass 1 counts kept entries per
// tile of kTile entries, a device-wide exclusive scan turns the counts into
// tile offsets, pass 2 re-evaluates the predicate and writes each kept pair
// at tile offset + (warp ballot / popc rank within the tile).
#include "internal.cuh"

namespace tc {

constexpr int kCovThreads = 256;
constexpr int kCovItems = 8;
constexpr int kCovTile = kCovThreads * kCovItems;

__device__ __forceinline__ bool is_cover(const uint32_t* __restrict__ erow,
                                         const uint32_t* __restrict__ cols,
                                         const uint32_t* __restrict__ L, int64_t e, int64_t nnz,
                                         uint32_t* pu, uint32_t* pv) {
  if (e >= nnz) return false;
  uint32_t u = erow[e], v = cols[e];
  *pu = u;
  *pv = v;
  return u < v && L[u] == L[v];
}

__global__ void __launch_bounds__(kCovThreads)
k_cover_count(const uint32_t* __restrict__ erow, const uint32_t* __restrict__ cols,
              const uint32_t* __restrict__ L, int64_t nnz, unsigned long long* tile_counts) {
  const int64_t base = (int64_t)blockIdx.x * kCovTile;
  int c = 0;
#pragma unroll
  for (int k = 0; k < kCovItems; ++k) {
    uint32_t u, v;
    c += is_cover(erow, cols, L, base + k * kCovThreads + threadIdx.x, nnz, &u, &v) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
  __shared__ int ws[kCovThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kCovThreads / 32; ++w) t += ws[w];
    tile_counts[blockIdx.x] = (unsigned long long)t;
  }
}

__global__ void __launch_bounds__(kCovThreads)
k_cover_write(const uint32_t* __restrict__ erow, const uint32_t* __restrict__ cols,
              const uint32_t* __restrict__ L, int64_t nnz,
              const unsigned long long* __restrict__ tile_offsets, uint2* __restrict__ H) {
  constexpr int kWarps = kCovThreads / 32;
  __shared__ int pre[kCovItems * kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kCovTile;
  unsigned masks[kCovItems];
  uint32_t us[kCovItems], vs[kCovItems];
#pragma unroll
  for (int k = 0; k < kCovItems; ++k) {
    bool f = is_cover(erow, cols, L, base + k * kCovThreads + threadIdx.x, nnz, &us[k], &vs[k]);
    masks[k] = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) pre[k * kWarps + wid] = __popc(masks[k]);
  }
  __syncthreads();
  // entry order inside the tile is (k, warp, lane): exclusive scan of the
  // kCovItems * kWarps warp counts in that order
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < kCovItems * kWarps; ++i) {
      int x = pre[i];
      pre[i] = run;
      run += x;
    }
  }
  __syncthreads();
  const unsigned long long t0 = tile_offsets[blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kCovItems; ++k) {
    if (masks[k] & (1u << lane)) {
      unsigned long long pos = t0 + pre[k * kWarps + wid] + __popc(masks[k] & lt);
      H[pos] = make_uint2(us[k], vs[k]);
    }
  }
}

int compute_cover(tc_graph* g) {
  cudaStream_t s = g->stream;
  if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  g->cover.release();
  g->num_cover = 0;
  if (g->nnz == 0) return TC_OK;
  const int64_t tiles = (g->nnz + kCovTile - 1) / kCovTile;
  DevBuf<unsigned long long> offs;
  TC_TRY(offs.alloc((size_t)tiles, s));
  launch(k_cover_count, (unsigned)tiles, kCovThreads, 0, s, g->erow.p, g->cols, g->levels.p, g->nnz,
                                                        offs.p);
  TC_TRY(exclusive_scan_u64(offs.p, tiles, g->ctrl.p + kCtrlTmp, s));
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host + kCtrlTmp, g->ctrl.p + kCtrlTmp, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  const int64_t h = (int64_t)g->ctrl_host[kCtrlTmp];
  TC_TRY(g->cover.alloc((size_t)h, s));
  if (h > 0)
    launch(k_cover_write, (unsigned)tiles, kCovThreads, 0, s, g->erow.p, g->cols, g->levels.p, g->nnz,
                                                          offs.p, g->cover.p);
  TC_CUDA(cudaGetLastError());
  g->num_cover = h;
  return TC_OK;
}

}  // namespace tc

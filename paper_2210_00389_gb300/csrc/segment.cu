// Level-segmented adjacency and cover-edge extraction (a2).
//
// After the BFS every neighbour w of x sits on level L(x)-1, L(x) or L(x)+1
// (levels are BFS distances, Def. 2 of Bader et al., "Triangle Counting
// Through Cover-Edges").  Each row of the CSR is stably partitioned into
// those three segments (each stays sorted), and the same-level segment is
// split at x:
//
//   scols[off[x] ..            off[x]+seg.x)   neighbours on level L(x)-1
//   scols[off[x]+seg.x ..      off[x]+seg.y)   same level, id < x
//   scols[off[x]+seg.y ..      off[x]+seg.z)   same level, id > x
//   scols[off[x]+seg.z ..      off[x+1])       neighbours on level L(x)+1
//
// The paper's cost analysis (Sec. III) budgets O(m) for rewriting the
// neighbour sets after the BFS; this is that step here.  It makes the
// count-once rule of Alg. 1 / Thm. 2 a property of which segments are
// intersected, so no level is read per common neighbour.
//
// The cover-edge set H (Thm. 1) is then, for every u, the segment
// "same level, id > u": its size is seg.z - seg.y, so H is written by an
// exclusive scan over vertices followed by a copy of those segments, in
// ascending (u, v) order.  hoff[u] (kept with H) is the index of u's first
// cover edge, so cover edge i = (u, v) sits at position i - hoff[u] of u's
// "same level, id > u" run.
#include "internal.cuh"

namespace tc {

constexpr int kSegThreads = 256;

// Warp per row; each chunk of 32 entries is classified, and warp ballots
// give each entry's rank inside its segment.
__global__ void __launch_bounds__(kSegThreads)
k_segment_rows(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
               const uint32_t* __restrict__ L, uint32_t n, uint32_t* __restrict__ scols,
               uint4* __restrict__ seg) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = warp; x < (int64_t)n; x += nwarps) {
    const int64_t b = off[x], e = off[x + 1];
    const uint32_t lx = L[x];
    // pass 1: segment sizes
    unsigned cb = 0, cs_lo = 0, cs_hi = 0;
    for (int64_t i = b + lane; i < e; i += 32) {
      const uint32_t w = cols[i];
      const uint32_t lw = L[w];
      cb += lw < lx;
      if (lw == lx) {
        if (w < (uint32_t)x) ++cs_lo; else ++cs_hi;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      cb += __shfl_xor_sync(0xFFFFFFFFu, cb, o);
      cs_lo += __shfl_xor_sync(0xFFFFFFFFu, cs_lo, o);
      cs_hi += __shfl_xor_sync(0xFFFFFFFFu, cs_hi, o);
    }
    // pass 2: stable scatter into the four runs
    int64_t p0 = b, p1 = b + cb, p2 = b + cb + cs_lo, p3 = b + cb + cs_lo + cs_hi;
    for (int64_t base = b; base < e; base += 32) {
      const int64_t i = base + lane;
      uint32_t w = 0;
      int cls = -1;
      if (i < e) {
        w = cols[i];
        const uint32_t lw = L[w];
        cls = lw < lx ? 0 : (lw == lx ? (w < (uint32_t)x ? 1 : 2) : 3);
      }
      const unsigned m0 = __ballot_sync(0xFFFFFFFFu, cls == 0);
      const unsigned m1 = __ballot_sync(0xFFFFFFFFu, cls == 1);
      const unsigned m2 = __ballot_sync(0xFFFFFFFFu, cls == 2);
      const unsigned m3 = __ballot_sync(0xFFFFFFFFu, cls == 3);
      if (cls == 0) scols[p0 + __popc(m0 & lt)] = w;
      else if (cls == 1) scols[p1 + __popc(m1 & lt)] = w;
      else if (cls == 2) scols[p2 + __popc(m2 & lt)] = w;
      else if (cls == 3) scols[p3 + __popc(m3 & lt)] = w;
      p0 += __popc(m0);
      p1 += __popc(m1);
      p2 += __popc(m2);
      p3 += __popc(m3);
    }
    if (lane == 0) seg[x] = make_uint4(cb, cb + cs_lo, cb + cs_lo + cs_hi, 0u);
  }
}

__global__ void k_cover_counts(const uint4* __restrict__ seg, uint32_t n,
                               unsigned long long* __restrict__ cnt) {
  int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; x < (int64_t)n; x += stride) {
    const uint4 s = seg[x];
    cnt[x] = (unsigned long long)(s.z - s.y);
  }
}

// Warp per vertex: copy the "same level, id > u" segment of u into H.
__global__ void __launch_bounds__(kSegThreads)
k_cover_gather(const int64_t* __restrict__ off, const uint32_t* __restrict__ scols,
               const uint4* __restrict__ seg, const unsigned long long* __restrict__ hoff,
               uint32_t n, uint2* __restrict__ H) {
  const int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < (int64_t)n; u += nwarps) {
    const uint4 s = seg[u];
    const int64_t len = (int64_t)(s.z - s.y);
    if (len == 0) continue;
    const uint32_t* src = scols + off[u] + s.y;
    const unsigned long long dst = hoff[u];
    for (int64_t k = lane; k < len; k += 32) H[dst + k] = make_uint2((uint32_t)u, src[k]);
  }
}

int compute_segments(tc_graph* g) {
  cudaStream_t s = g->stream;
  if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  if (g->seg_valid) return TC_OK;
  TC_TRY(g->scols.reserve((size_t)g->nnz, s));
  TC_TRY(g->seg.reserve(g->n, s));
  if (g->n > 0)
    launch(k_segment_rows, grid_for((int64_t)g->n * 32, kSegThreads, 16), kSegThreads, 0, s,
           g->off, g->cols, g->levels.p, g->n, g->scols.p, g->seg.p);
  TC_CUDA(cudaGetLastError());
  g->seg_valid = true;
  return TC_OK;
}

int compute_cover(tc_graph* g) {
  cudaStream_t s = g->stream;
  TC_TRY(compute_segments(g));
  g->cover.release();
  g->num_cover = 0;
  if (g->nnz == 0) return TC_OK;
  DevBuf<unsigned long long>& hoff = g->hoff;
  TC_TRY(hoff.reserve(g->n, s));
  launch(k_cover_counts, grid_for(g->n, kSegThreads), kSegThreads, 0, s, g->seg.p, g->n, hoff.p);
  TC_TRY(exclusive_scan_u64(hoff.p, g->n, g->ctrl.p + kCtrlTmp, s));
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host + kCtrlTmp, g->ctrl.p + kCtrlTmp, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  const int64_t h = (int64_t)g->ctrl_host[kCtrlTmp];
  TC_TRY(g->cover.alloc((size_t)h, s));
  if (h > 0)
    launch(k_cover_gather, grid_for((int64_t)g->n * 32, kSegThreads, 16), kSegThreads, 0, s,
           g->off, g->scols.p, g->seg.p, hoff.p, g->n, g->cover.p);
  TC_CUDA(cudaGetLastError());
  g->num_cover = h;
  return TC_OK;
}

}  // namespace tc

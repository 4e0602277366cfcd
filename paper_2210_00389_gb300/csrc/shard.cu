// Work-balanced shards of the edge index space (multi-GPU plan: the CSR
// and the levels are replicated, each GPU counts one contiguous slice of the
// cover edges and the per-GPU counts are summed).
//
// Cover edges are independent units once the levels exist (Alg. 1 of Bader
// et al., "Triangle Counting Through Cover-Edges": the count is a sum over
// H of per-edge terms, Thm. 2), so any partition of H gives partial counts
// whose sum is T.  The plain count is a sum over CSR entries u < v in the
// same way.  A slice's cost is estimated per edge as the lookups the hash
// intersection makes for it plus a fixed per-edge overhead.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace tc {

constexpr int kShardChunk = 4096;  // bounds fall on multiples of this
constexpr int kShardThreads = 256;

// Estimated cost of one edge: the lookups the hash intersection makes for
// it plus a fixed per-edge overhead (descriptor, work grab, reduction).
// The probe side is the endpoint of smaller degree (u on ties, as in the
// bucketing); its lookups are its relevant neighbours -- cover: its level
// l-1 segment and its level-l and level-l+1 neighbours above v (the
// segmented row [l-1 | l, id < x | l, id > x | l+1] of segment.cu); plain:
// its neighbours above v.
constexpr unsigned long long kEdgeOverhead = 32;

__device__ __forceinline__ int64_t first_above(const uint32_t* __restrict__ cols, int64_t lo,
                                               int64_t hi, uint32_t x) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cols[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Block per chunk: its edges' estimated work.
__global__ void __launch_bounds__(kShardThreads)
k_chunk_work(int mode, const uint2* __restrict__ H, const unsigned long long* __restrict__ hoff,
             const uint4* __restrict__ seg, const uint32_t* __restrict__ erow,
             const uint32_t* __restrict__ cols, const int64_t* __restrict__ off, int64_t nidx,
             unsigned long long* __restrict__ cw) {
  __shared__ unsigned long long red[kShardThreads / 32];
  const int64_t nch = (nidx + kShardChunk - 1) / kShardChunk;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    unsigned long long acc = 0;
    const int64_t e = min(nidx, (c + 1) * kShardChunk);
    for (int64_t i = c * kShardChunk + threadIdx.x; i < e; i += kShardThreads) {
      uint32_t u, v;
      if (mode == TC_MODE_COVER) {
        const uint2 h = H[i];
        u = h.x;
        v = h.y;
      } else {
        u = erow[i];
        v = cols[i];
        if (u >= v) continue;
      }
      const int64_t du = off[u + 1] - off[u], dv = off[v + 1] - off[v];
      const bool pu = dv > du;  // the probe side is u
      int64_t work;
      if (mode == TC_MODE_COVER) {
        const uint32_t p = pu ? u : v;
        const uint4 sg = seg[p];
        const int64_t dp = pu ? du : dv;
        const int64_t cut = pu ? (int64_t)sg.y + (i - (int64_t)hoff[u]) + 1 : (int64_t)sg.y;
        work = (int64_t)sg.x + (dp - cut);
      } else {
        work = pu ? off[u + 1] - (i + 1) : off[v + 1] - first_above(cols, off[v], off[v + 1], v);
      }
      acc += (unsigned long long)work + kEdgeOverhead;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int k = 0; k < kShardThreads / 32; ++k) t += red[k];
      cw[c] = t;
    }
    __syncthreads();
  }
}

// Thread k (1 <= k < P): bound k = the first chunk whose exclusive work
// prefix reaches k / P of the total, as an edge index.
__global__ void k_shard_bounds(const unsigned long long* __restrict__ prefix, int64_t nch,
                               const unsigned long long* __restrict__ total, int32_t P,
                               int64_t nidx, int64_t* __restrict__ bounds) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > P) return;
  if (k == 0) { bounds[0] = 0; return; }
  if (k == P) { bounds[P] = nidx; return; }
  // target k * W / P without overflow for W < 2^64
  const unsigned long long W = *total;
  const unsigned long long tgt = (W / P) * k + ((W % P) * k) / P;
  int64_t lo = 0, hi = nch;  // first c with prefix[c] >= tgt
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] < tgt) lo = mid + 1; else hi = mid;
  }
  bounds[k] = min(nidx, lo * (int64_t)kShardChunk);
}

int shard_bounds(tc_graph* g, int mode, int32_t P, int64_t* bounds_host) {
  cudaStream_t s = g->stream;
  int64_t nidx;
  if (mode == TC_MODE_COVER) {
    if (g->num_cover < 0) TC_TRY(compute_cover(g));
    nidx = g->num_cover;
  } else {
    TC_TRY(ensure_erow(g));
    nidx = g->nnz;
  }
  const int64_t nch = (nidx + kShardChunk - 1) / kShardChunk;
  DevBuf<unsigned long long> cw, total;
  DevBuf<int64_t> dbounds;
  TC_TRY(cw.alloc((size_t)std::max<int64_t>(nch, 1), s));
  TC_TRY(total.alloc(1, s));
  TC_TRY(dbounds.alloc((size_t)P + 1, s));
  TC_CUDA(cudaMemsetAsync(total.p, 0, sizeof(unsigned long long), s));
  if (nch > 0) {
    launch(k_chunk_work, (int)std::min<int64_t>(nch, (int64_t)sm_count() * 8), kShardThreads, 0,
           s, mode, g->cover.p, g->hoff.p, g->seg.p, g->erow.p, g->cols, g->off, nidx, cw.p);
    TC_TRY(exclusive_scan_u64(cw.p, nch, total.p, s));
  }
  launch(k_shard_bounds, (P + 1 + 127) / 128, 128, 0, s, cw.p, nch, total.p, P, nidx, dbounds.p);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaMemcpyAsync(bounds_host, dbounds.p, sizeof(int64_t) * ((size_t)P + 1),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  return TC_OK;
}

}  // namespace tc

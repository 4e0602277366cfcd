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
#include <algorithm>

#include "internal.cuh"

namespace tc {

constexpr int kSegThreads = 256;

// Segment of neighbour w (level lw) in the row of x (level lx): 0 = level
// below, 1 = same level and id < x, 2 = same level and id > x, 3 = above.
__device__ __forceinline__ int seg_class(uint32_t w, uint32_t lw, uint32_t x, uint32_t lx) {
  return lw < lx ? 0 : (lw == lx ? (w < x ? 1 : 2) : 3);
}

// Warp per row (rows of at most kLongRow entries); each chunk of 32 entries
// is classified, and warp ballots give each entry's rank inside its
// segment.  A row of at most 32 entries takes one pass; a longer one counts
// its segments first.
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
    if (e - b > kLongRow) continue;  // chunked: k_segment_chunks
    const uint32_t lx = L[x];
    unsigned c0, c1, c2;
    if (e - b <= 32) {
      const int64_t i = b + lane;
      uint32_t w = 0;
      int cls = -1;
      if (i < e) {
        w = cols[i];
        cls = seg_class(w, L[w], (uint32_t)x, lx);
      }
      const unsigned m0 = __ballot_sync(0xFFFFFFFFu, cls == 0);
      const unsigned m1 = __ballot_sync(0xFFFFFFFFu, cls == 1);
      const unsigned m2 = __ballot_sync(0xFFFFFFFFu, cls == 2);
      const unsigned m3 = __ballot_sync(0xFFFFFFFFu, cls == 3);
      c0 = __popc(m0);
      c1 = __popc(m1);
      c2 = __popc(m2);
      if (cls == 0) scols[b + __popc(m0 & lt)] = w;
      else if (cls == 1) scols[b + c0 + __popc(m1 & lt)] = w;
      else if (cls == 2) scols[b + c0 + c1 + __popc(m2 & lt)] = w;
      else if (cls == 3) scols[b + c0 + c1 + c2 + __popc(m3 & lt)] = w;
    } else {
      // pass 1: segment sizes
      c0 = 0; c1 = 0; c2 = 0;
      for (int64_t i = b + lane; i < e; i += 32) {
        const uint32_t w = cols[i];
        const int cls = seg_class(w, L[w], (uint32_t)x, lx);
        c0 += cls == 0;
        c1 += cls == 1;
        c2 += cls == 2;
      }
      for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xFFFFFFFFu, c0, o);
        c1 += __shfl_xor_sync(0xFFFFFFFFu, c1, o);
        c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
      }
      // pass 2: stable scatter into the four runs
      int64_t p0 = b, p1 = b + c0, p2 = b + c0 + c1, p3 = b + c0 + c1 + c2;
      for (int64_t base = b; base < e; base += 32) {
        const int64_t i = base + lane;
        uint32_t w = 0;
        int cls = -1;
        if (i < e) {
          w = cols[i];
          cls = seg_class(w, L[w], (uint32_t)x, lx);
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
    }
    if (lane == 0) seg[x] = make_uint4(c0, c0 + c1, c0 + c1 + c2, 0u);
  }
}

// Long rows, pass 1: CTA per chunk, the chunk's segment sizes.
__global__ void __launch_bounds__(kChunk)
k_segment_chunk_counts(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                       const uint32_t* __restrict__ L, const uint2* __restrict__ lchunks,
                       int64_t nch, uint4* __restrict__ ccnt) {
  __shared__ unsigned red[3][kChunk / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const uint32_t x = ch.x, lx = L[x];
    const int64_t b = off[x], e = off[x + 1];
    const int64_t i = b + (int64_t)ch.y * kChunk + threadIdx.x;
    int cls = -1;
    if (i < e) {
      const uint32_t w = cols[i];
      cls = seg_class(w, L[w], x, lx);
    }
    const unsigned m0 = __ballot_sync(0xFFFFFFFFu, cls == 0);
    const unsigned m1 = __ballot_sync(0xFFFFFFFFu, cls == 1);
    const unsigned m2 = __ballot_sync(0xFFFFFFFFu, cls == 2);
    if (lane == 0) {
      red[0][wid] = __popc(m0);
      red[1][wid] = __popc(m1);
      red[2][wid] = __popc(m2);
    }
    __syncthreads();
    if (wid == 0) {
      unsigned a0 = red[0][lane], a1 = red[1][lane], a2 = red[2][lane];
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xFFFFFFFFu, a0, o);
        a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, o);
        a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, o);
      }
      if (lane == 0) ccnt[c] = make_uint4(a0, a1, a2, 0u);
    }
    __syncthreads();
  }
}

// Long rows, pass 2: CTA per chunk.  The row's segment sizes and the
// chunk's offset inside each segment are sums over the row's chunk counts
// (the row's chunks are contiguous in lchunks); then a stable scatter of
// the chunk, ranked by warp ballots and a scan over the CTA's warps.  The
// row's first chunk writes seg.
__global__ void __launch_bounds__(kChunk)
k_segment_chunks(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                 const uint32_t* __restrict__ L, const uint2* __restrict__ lchunks, int64_t nch,
                 const uint4* __restrict__ ccnt, uint32_t* __restrict__ scols,
                 uint4* __restrict__ seg) {
  constexpr int kW = kChunk / 32;
  __shared__ unsigned s_tot[2][3][kW];   // [before this chunk / whole row][segment][warp]
  __shared__ unsigned s_wc[4][kW];       // per segment and warp: entries before this warp
  __shared__ unsigned s_base[2][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const uint32_t x = ch.x, lx = L[x];
    const int64_t b = off[x], e = off[x + 1];
    const uint32_t nrow = (uint32_t)((e - b + kChunk - 1) / kChunk);
    const int64_t first = c - ch.y;
    // row totals and this chunk's prefix
    unsigned t[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (uint32_t k = threadIdx.x; k < nrow; k += kChunk) {
      const uint4 q = ccnt[first + k];
      t[1][0] += q.x; t[1][1] += q.y; t[1][2] += q.z;
      if (k < ch.y) { t[0][0] += q.x; t[0][1] += q.y; t[0][2] += q.z; }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        unsigned v = t[h][j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) s_tot[h][j][wid] = v;
      }
    // classify this thread's entry
    const int64_t i = b + (int64_t)ch.y * kChunk + threadIdx.x;
    uint32_t w = 0;
    int cls = -1;
    if (i < e) {
      w = cols[i];
      cls = seg_class(w, L[w], x, lx);
    }
    unsigned m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) m[j] = __ballot_sync(0xFFFFFFFFu, cls == j);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) s_wc[j][wid] = __popc(m[j]);
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          unsigned v = s_tot[h][j][lane];
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
          if (lane == 0) s_base[h][j] = v;
        }
    } else if (wid <= 4) {
      // exclusive scan over the warps of segment wid - 1's counts
      const int j = wid - 1;
      const unsigned x = s_wc[j][lane];
      unsigned v = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
      }
      __syncwarp();
      s_wc[j][lane] = v - x;
    }
    __syncthreads();
    if (cls >= 0) {
      // segment start in the row + entries of this segment in earlier
      // chunks + in earlier warps of this chunk + rank in the warp
      const unsigned R0 = s_base[1][0], R1 = s_base[1][1], R2 = s_base[1][2];
      unsigned start = cls == 0 ? 0u : (cls == 1 ? R0 : (cls == 2 ? R0 + R1 : R0 + R1 + R2));
      unsigned before;
      if (cls < 3) {
        before = s_base[0][cls];
      } else {
        // earlier chunks' entries above the level: their size minus the rest
        before = ch.y * (unsigned)kChunk - s_base[0][0] - s_base[0][1] - s_base[0][2];
      }
      scols[b + start + before + s_wc[cls][wid] + __popc(m[cls] & lt)] = w;
    }
    if (ch.y == 0 && threadIdx.x == 0) {
      const unsigned R0 = s_base[1][0], R1 = s_base[1][1], R2 = s_base[1][2];
      seg[x] = make_uint4(R0, R0 + R1, R0 + R1 + R2, 0u);
    }
    __syncthreads();
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
// Long rows are copied by k_cover_gather_chunks.
__global__ void __launch_bounds__(kSegThreads)
k_cover_gather(const int64_t* __restrict__ off, const uint32_t* __restrict__ scols,
               const uint4* __restrict__ seg, const unsigned long long* __restrict__ hoff,
               uint32_t n, uint2* __restrict__ H) {
  const int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < (int64_t)n; u += nwarps) {
    const int64_t b = off[u];
    if (off[u + 1] - b > kLongRow) continue;
    const uint4 s = seg[u];
    const int64_t len = (int64_t)(s.z - s.y);
    if (len == 0) continue;
    const uint32_t* src = scols + b + s.y;
    const unsigned long long dst = hoff[u];
    for (int64_t k = lane; k < len; k += 32) H[dst + k] = make_uint2((uint32_t)u, src[k]);
  }
}

// CTA per chunk of a long row: the part of the row's cover run that falls
// in the chunk's entry range.
__global__ void __launch_bounds__(kChunk)
k_cover_gather_chunks(const int64_t* __restrict__ off, const uint32_t* __restrict__ scols,
                      const uint4* __restrict__ seg, const unsigned long long* __restrict__ hoff,
                      const uint2* __restrict__ lchunks, int64_t nch, uint2* __restrict__ H) {
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const uint32_t u = ch.x;
    const uint4 s = seg[u];
    const uint32_t k = ch.y * (uint32_t)kChunk + threadIdx.x;  // entry within the row
    if (k >= s.y && k < s.z) H[hoff[u] + (k - s.y)] = make_uint2(u, scols[off[u] + k]);
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
  if (g->nlchunks > 0) {
    DevBuf<uint4> ccnt;
    TC_TRY(ccnt.alloc((size_t)g->nlchunks, s));
    const int grid = (int)std::min<int64_t>(g->nlchunks, (int64_t)sm_count() * 2);
    launch(k_segment_chunk_counts, grid, kChunk, 0, s, g->off, g->cols, g->levels.p,
           g->lchunks.p, g->nlchunks, ccnt.p);
    launch(k_segment_chunks, grid, kChunk, 0, s, g->off, g->cols, g->levels.p, g->lchunks.p,
           g->nlchunks, ccnt.p, g->scols.p, g->seg.p);
  }
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
  if (h > 0) {
    launch(k_cover_gather, grid_for((int64_t)g->n * 32, kSegThreads, 16), kSegThreads, 0, s,
           g->off, g->scols.p, g->seg.p, hoff.p, g->n, g->cover.p);
    if (g->nlchunks > 0)
      launch(k_cover_gather_chunks, (int)std::min<int64_t>(g->nlchunks, (int64_t)sm_count() * 2),
             kChunk, 0, s, g->off, g->scols.p, g->seg.p, hoff.p, g->lchunks.p, g->nlchunks,
             g->cover.p);
  }
  TC_CUDA(cudaGetLastError());
  g->num_cover = h;
  return TC_OK;
}

}  // namespace tc

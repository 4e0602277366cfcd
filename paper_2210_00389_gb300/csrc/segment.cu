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
// and seg.w = L(x).
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
// A neighbour's level differs from x's by at most one (levels are BFS
// distances), so the levels are needed only modulo 256: lw may come from a
// byte copy of the levels (LT = uint8_t), which stays resident in L2 where
// the 32-bit levels of a large graph do not.
__device__ __forceinline__ int seg_class(uint32_t w, uint32_t lw, uint32_t x, uint32_t lx) {
  const uint32_t d = (lw - lx) & 0xFFu;
  return d == 0u ? (w < x ? 1 : 2) : (d == 1u ? 3 : 0);
}

constexpr int kTinyRow = 8;  // rows this short are partitioned by one thread
constexpr int kSegUnroll = 4;
constexpr int kSegBlock = 32 * kSegUnroll;  // entries a warp loads at once

// Entries [base, base + kSegBlock) of a row ending at e: lane entries
// base + 32 k + lane with their segment class (-1 past the row).
template <class LT>
__device__ __forceinline__ void seg_load_block(const uint32_t* __restrict__ cols,
                                               const LT* __restrict__ B, int64_t base,
                                               int64_t e, uint32_t x, uint32_t lx,
                                               uint32_t (&w)[kSegUnroll], int (&cls)[kSegUnroll]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kSegUnroll; ++k) {
    const int64_t i = base + 32 * k + lane;
    w[k] = i < e ? cols[i] : 0u;
  }
#pragma unroll
  for (int k = 0; k < kSegUnroll; ++k) {
    const int64_t i = base + 32 * k + lane;
    cls[k] = i < e ? seg_class(w[k], B[w[k]], x, lx) : -1;
  }
}

// Rows of at most kLongRow entries.  A warp takes 32 consecutive rows: each
// lane partitions its own row if it has at most kTinyRow entries (all its
// loads issued at once); the longer rows are then taken one at a time by
// the whole warp, in blocks of kSegBlock entries classified and ranked
// inside their segment by warp ballots.  A row of one block takes one pass;
// a longer one counts its segments first.  L: levels; B: the levels read for
// neighbours (L itself, or its byte copy).
template <class LT>
__global__ void __launch_bounds__(kSegThreads)
k_segment_rows(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
               const uint32_t* __restrict__ L, const LT* __restrict__ B, uint32_t n,
               uint32_t* __restrict__ scols, uint4* __restrict__ seg) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t gbase = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; gbase < (int64_t)n;
       gbase += gstride) {
    const int64_t xl = gbase + lane;
    int64_t bl = 0, el = 0;
    if (xl < (int64_t)n) {
      bl = off[xl];
      el = off[xl + 1];
    }
    const int64_t dl = el - bl;
    if (xl < (int64_t)n && dl <= kTinyRow) {
      const uint32_t lx = L[xl];
      uint32_t w[kTinyRow];
      int cls[kTinyRow];
#pragma unroll
      for (int k = 0; k < kTinyRow; ++k) w[k] = k < dl ? cols[bl + k] : 0u;
#pragma unroll
      for (int k = 0; k < kTinyRow; ++k)
        cls[k] = k < dl ? seg_class(w[k], B[w[k]], (uint32_t)xl, lx) : -1;
      unsigned c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
      for (int k = 0; k < kTinyRow; ++k) {
        c0 += cls[k] == 0;
        c1 += cls[k] == 1;
        c2 += cls[k] == 2;
      }
      int64_t p0 = bl, p1 = bl + c0, p2 = bl + c0 + c1, p3 = bl + c0 + c1 + c2;
#pragma unroll
      for (int k = 0; k < kTinyRow; ++k) {
        if (cls[k] == 0) scols[p0++] = w[k];
        else if (cls[k] == 1) scols[p1++] = w[k];
        else if (cls[k] == 2) scols[p2++] = w[k];
        else if (cls[k] == 3) scols[p3++] = w[k];
      }
      seg[xl] = make_uint4(c0, c0 + c1, c0 + c1 + c2, lx);
    }
    // rows for the whole warp (long rows are chunked: k_segment_chunks)
    unsigned rows = __ballot_sync(0xFFFFFFFFu, xl < (int64_t)n && dl > kTinyRow && dl <= kLongRow);
    while (rows) {
      const int r = __ffs(rows) - 1;
      rows &= rows - 1;
      const int64_t x = gbase + r;
      const int64_t b = __shfl_sync(0xFFFFFFFFu, bl, r), e = __shfl_sync(0xFFFFFFFFu, el, r);
      const uint32_t lx = L[x];
      // blocks of kSegBlock entries, all loads of a block issued together
      unsigned c0 = 0, c1 = 0, c2 = 0;
      if (e - b > kSegBlock) {
        // pass 1: segment sizes (a row of one block counts from its ballots)
        for (int64_t base = b; base < e; base += kSegBlock) {
          uint32_t w[kSegUnroll];
          int cls[kSegUnroll];
          seg_load_block(cols, B, base, e, (uint32_t)x, lx, w, cls);
#pragma unroll
          for (int k = 0; k < kSegUnroll; ++k) {
            c0 += cls[k] == 0;
            c1 += cls[k] == 1;
            c2 += cls[k] == 2;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          c0 += __shfl_xor_sync(0xFFFFFFFFu, c0, o);
          c1 += __shfl_xor_sync(0xFFFFFFFFu, c1, o);
          c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
        }
      }
      // pass 2: stable scatter into the four runs
      int64_t p0 = b, p1 = b + c0, p2 = b + c0 + c1, p3 = b + c0 + c1 + c2;
      for (int64_t base = b; base < e; base += kSegBlock) {
        uint32_t w[kSegUnroll];
        int cls[kSegUnroll];
        seg_load_block(cols, B, base, e, (uint32_t)x, lx, w, cls);
        if (e - b <= kSegBlock) {
          // one block: the segment sizes are its ballot counts
#pragma unroll
          for (int k = 0; k < kSegUnroll; ++k) {
            c0 += __popc(__ballot_sync(0xFFFFFFFFu, cls[k] == 0));
            c1 += __popc(__ballot_sync(0xFFFFFFFFu, cls[k] == 1));
            c2 += __popc(__ballot_sync(0xFFFFFFFFu, cls[k] == 2));
          }
          p1 = b + c0;
          p2 = b + c0 + c1;
          p3 = b + c0 + c1 + c2;
        }
        // ballots taken per round and used at once (few masks live)
#pragma unroll
        for (int k = 0; k < kSegUnroll; ++k) {
          const unsigned m0 = __ballot_sync(0xFFFFFFFFu, cls[k] == 0);
          const unsigned m1 = __ballot_sync(0xFFFFFFFFu, cls[k] == 1);
          const unsigned m2 = __ballot_sync(0xFFFFFFFFu, cls[k] == 2);
          const unsigned m3 = __ballot_sync(0xFFFFFFFFu, cls[k] == 3);
          if (cls[k] == 0) scols[p0 + __popc(m0 & lt)] = w[k];
          else if (cls[k] == 1) scols[p1 + __popc(m1 & lt)] = w[k];
          else if (cls[k] == 2) scols[p2 + __popc(m2 & lt)] = w[k];
          else if (cls[k] == 3) scols[p3 + __popc(m3 & lt)] = w[k];
          p0 += __popc(m0);
          p1 += __popc(m1);
          p2 += __popc(m2);
          p3 += __popc(m3);
        }
      }
      if (lane == 0) seg[x] = make_uint4(c0, c0 + c1, c0 + c1 + c2, lx);
    }
  }
}

// Long rows: a CTA of kChunkThreads threads per chunk of kChunk entries,
// kChunkPer entries per thread (entry s * kChunkThreads + thread), all of a
// thread's loads issued before they are used.
constexpr int kChunkThreads = 256;
constexpr int kChunkPer = kChunk / kChunkThreads;
constexpr int kChunkWarps = kChunkThreads / 32;
static_assert(kChunkPer * kChunkWarps == 32, "one warp scans a chunk's (sub-chunk, warp) counts");

// Long rows, pass 1: the chunk's segment sizes.
template <class LT>
__global__ void __launch_bounds__(kChunkThreads)
k_segment_chunk_counts(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                       const uint32_t* __restrict__ L, const LT* __restrict__ B,
                       const uint2* __restrict__ lchunks, int64_t nch, uint4* __restrict__ ccnt) {
  __shared__ unsigned red[3][kChunkWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const uint32_t x = ch.x, lx = L[x];
    const int64_t e = off[x + 1];
    const int64_t i0 = off[x] + (int64_t)ch.y * kChunk + threadIdx.x;
    uint32_t w[kChunkPer];
#pragma unroll
    for (int k = 0; k < kChunkPer; ++k) {
      const int64_t i = i0 + k * kChunkThreads;
      w[k] = i < e ? cols[i] : kUnvisited;
    }
    unsigned a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int k = 0; k < kChunkPer; ++k) {
      if (w[k] != kUnvisited) {
        const int cls = seg_class(w[k], B[w[k]], x, lx);
        a0 += cls == 0;
        a1 += cls == 1;
        a2 += cls == 2;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xFFFFFFFFu, a0, o);
      a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, o);
      a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, o);
    }
    if (lane == 0) {
      red[0][wid] = a0;
      red[1][wid] = a1;
      red[2][wid] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      for (int k = 0; k < kChunkWarps; ++k) {
        q.x += red[0][k];
        q.y += red[1][k];
        q.z += red[2][k];
      }
      ccnt[c] = q;
    }
    __syncthreads();
  }
}

// Long rows, pass 2.  The row's segment sizes and the chunk's offset inside
// each segment are sums over the row's chunk counts (the row's chunks are
// contiguous in lchunks); then a stable scatter of the chunk, ranked by
// __match_any_sync inside a warp and a scan over the chunk's (sub-chunk,
// warp) counts.  The row's first chunk writes seg.
template <class LT>
__global__ void __launch_bounds__(kChunkThreads)
k_segment_chunks(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                 const uint32_t* __restrict__ L, const LT* __restrict__ B,
                 const uint2* __restrict__ lchunks, int64_t nch, const uint4* __restrict__ ccnt,
                 uint32_t* __restrict__ scols, uint4* __restrict__ seg) {
  __shared__ unsigned s_tot[2][3][kChunkWarps];  // [before this chunk / whole row][segment][warp]
  __shared__ unsigned s_cnt[4][32];  // [segment][sub-chunk * warps + warp]: then exclusive scan
  __shared__ unsigned s_base[2][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const uint32_t x = ch.x, lx = L[x];
    const int64_t b = off[x], e = off[x + 1];
    const uint32_t nrow = (uint32_t)((e - b + kChunk - 1) / kChunk);
    const int64_t first = c - ch.y;
    // this thread's entries (loads first)
    const int64_t i0 = b + (int64_t)ch.y * kChunk + threadIdx.x;
    uint32_t w[kChunkPer];
    int cls[kChunkPer];
#pragma unroll
    for (int k = 0; k < kChunkPer; ++k) {
      const int64_t i = i0 + k * kChunkThreads;
      w[k] = i < e ? cols[i] : kUnvisited;
    }
    // row totals and this chunk's prefix
    unsigned t[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (uint32_t k = threadIdx.x; k < nrow; k += kChunkThreads) {
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
#pragma unroll
    for (int k = 0; k < kChunkPer; ++k)
      cls[k] = w[k] != kUnvisited ? seg_class(w[k], B[w[k]], x, lx) : -1;
    unsigned rank[kChunkPer];
#pragma unroll
    for (int k = 0; k < kChunkPer; ++k) {
      rank[k] = __popc(__match_any_sync(0xFFFFFFFFu, cls[k]) & lt);
      const unsigned m0 = __ballot_sync(0xFFFFFFFFu, cls[k] == 0);
      const unsigned m1 = __ballot_sync(0xFFFFFFFFu, cls[k] == 1);
      const unsigned m2 = __ballot_sync(0xFFFFFFFFu, cls[k] == 2);
      const unsigned m3 = __ballot_sync(0xFFFFFFFFu, cls[k] == 3);
      if (lane == 0) {
        const int slot = k * kChunkWarps + wid;
        s_cnt[0][slot] = __popc(m0);
        s_cnt[1][slot] = __popc(m1);
        s_cnt[2][slot] = __popc(m2);
        s_cnt[3][slot] = __popc(m3);
      }
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          unsigned v = lane < kChunkWarps ? s_tot[h][j][lane] : 0u;
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
          if (lane == 0) s_base[h][j] = v;
        }
    } else if (wid <= 4) {
      // exclusive scan of segment (wid - 1)'s counts in (sub-chunk, warp) order
      const int j = wid - 1;
      const unsigned v0 = s_cnt[j][lane];
      unsigned v = v0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
      }
      __syncwarp();
      s_cnt[j][lane] = v - v0;
    }
    __syncthreads();
    const unsigned R0 = s_base[1][0], R1 = s_base[1][1], R2 = s_base[1][2];
#pragma unroll
    for (int k = 0; k < kChunkPer; ++k) {
      const int cl = cls[k];
      if (cl < 0) continue;
      // segment start in the row + entries of this segment in earlier
      // chunks + in earlier (sub-chunk, warp) groups + rank in the warp
      const unsigned start = cl == 0 ? 0u : (cl == 1 ? R0 : (cl == 2 ? R0 + R1 : R0 + R1 + R2));
      // earlier chunks' entries above the level: their size minus the rest
      const unsigned before =
          cl < 3 ? s_base[0][cl]
                 : ch.y * (unsigned)kChunk - s_base[0][0] - s_base[0][1] - s_base[0][2];
      scols[b + start + before + s_cnt[cl][k * kChunkWarps + wid] + rank[k]] = w[k];
    }
    if (ch.y == 0 && threadIdx.x == 0) seg[x] = make_uint4(R0, R0 + R1, R0 + R1 + R2, lx);
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

// Copy the "same level, id > u" segment of every u into H.  A warp takes 32
// consecutive vertices: a lane copies its own vertex's run if it has at
// most kTinyRow entries; longer runs are copied by the whole warp, one at a
// time.  Long rows are copied by k_cover_gather_chunks.
__global__ void __launch_bounds__(kSegThreads)
k_cover_gather(const int64_t* __restrict__ off, const uint32_t* __restrict__ scols,
               const uint4* __restrict__ seg, const unsigned long long* __restrict__ hoff,
               uint32_t n, uint2* __restrict__ H) {
  const int lane = threadIdx.x & 31;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t gbase = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; gbase < (int64_t)n;
       gbase += gstride) {
    const int64_t u = gbase + lane;
    bool mine = false, warp_run = false;
    int64_t src = 0;
    uint32_t len = 0;
    unsigned long long dst = 0;
    if (u < (int64_t)n) {
      const int64_t b = off[u];
      if (off[u + 1] - b <= kLongRow) {
        const uint4 sg = seg[u];
        len = sg.z - sg.y;
        if (len > 0) {
          src = b + sg.y;
          dst = hoff[u];
          mine = len <= kTinyRow;
          warp_run = !mine;
        }
      }
    }
    if (mine) {
      uint32_t w[kTinyRow];
#pragma unroll
      for (int k = 0; k < kTinyRow; ++k) w[k] = k < (int)len ? scols[src + k] : 0u;
#pragma unroll
      for (int k = 0; k < kTinyRow; ++k)
        if (k < (int)len) H[dst + k] = make_uint2((uint32_t)u, w[k]);
    }
    unsigned runs = __ballot_sync(0xFFFFFFFFu, warp_run);
    while (runs) {
      const int r = __ffs(runs) - 1;
      runs &= runs - 1;
      const int64_t s0 = __shfl_sync(0xFFFFFFFFu, src, r);
      const uint32_t l0 = __shfl_sync(0xFFFFFFFFu, len, r);
      const unsigned long long d0 = __shfl_sync(0xFFFFFFFFu, dst, r);
      const uint32_t ur = (uint32_t)(gbase + r);
      for (uint32_t k = lane; k < l0; k += 32) H[d0 + k] = make_uint2(ur, scols[s0 + k]);
    }
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

__global__ void k_levels_u8(const uint32_t* __restrict__ L, uint32_t n, uint8_t* __restrict__ B) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride) B[i] = (uint8_t)L[i];
}

// Graphs with more vertices than this read neighbour levels from a byte copy
// (n bytes instead of 4n: at R-MAT scale 26 67 MB, which L2 holds).
constexpr uint32_t kByteLevelsMin = 1u << 23;

template <class LT>
static void launch_segments(tc_graph* g, const LT* B, uint4* ccnt) {
  cudaStream_t s = g->stream;
  if (g->n > 0)
    launch(k_segment_rows<LT>, grid_for((int64_t)g->n * 32, kSegThreads, 16), kSegThreads, 0, s,
           g->off, g->cols, g->levels.p, B, g->n, g->scols.p, g->seg.p);
  if (g->nlchunks > 0) {
    const int grid = (int)std::min<int64_t>(g->nlchunks, (int64_t)sm_count() * 8);
    launch(k_segment_chunk_counts<LT>, grid, kChunkThreads, 0, s, g->off, g->cols, g->levels.p, B,
           g->lchunks.p, g->nlchunks, ccnt);
    launch(k_segment_chunks<LT>, grid, kChunkThreads, 0, s, g->off, g->cols, g->levels.p, B,
           g->lchunks.p, g->nlchunks, ccnt, g->scols.p, g->seg.p);
  }
}

int compute_segments(tc_graph* g) {
  cudaStream_t s = g->stream;
  if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  if (g->seg_valid) return TC_OK;
  TC_TRY(g->scols.reserve((size_t)g->nnz, s));
  TC_TRY(g->seg.reserve(g->n, s));
  DevBuf<uint4> ccnt;
  if (g->nlchunks > 0) TC_TRY(ccnt.alloc((size_t)g->nlchunks, s));
  if (g->n > kByteLevelsMin) {
    DevBuf<uint8_t> b;
    TC_TRY(b.alloc(g->n, s));
    launch(k_levels_u8, grid_for(g->n, kSegThreads), kSegThreads, 0, s, g->levels.p, g->n, b.p);
    launch_segments<uint8_t>(g, b.p, ccnt.p);
  } else {
    launch_segments<uint32_t>(g, g->levels.p, ccnt.p);
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

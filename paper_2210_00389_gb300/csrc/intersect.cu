// Intersection + count-once rule (a4), reduction (a5), plain count (a6).
//
// Cover path (Alg. 1 and Thm. 2 of Bader et al., "Triangle Counting Through
// Cover-Edges"): for a cover edge (u, v), u < v, on level l,
//   c_uv = |{ w in N(u) ∩ N(v) : L(w) != l  or  w > v }|.
// A common neighbour lies on level l-1, l or l+1, so with the level-segmented
// rows of segment.cu
//   c_uv = |N_{l-1}(u) ∩ N_{l-1}(v)| + |N_{l+1}(u) ∩ N_{l+1}(v)|
//        + |N_l(u) ∩ (v,inf)  ∩  N_l(v) ∩ (v,inf)|.
// Plain path (direction-oriented edge iterator, Sec. I and Sec. V-A): for an
// edge u < v, |N(u) ∩ (v,inf) ∩ N(v) ∩ (v,inf)|.
//
// Both paths share one warp-cooperative intersection of two sorted lists
// (warp_intersect): a windowed merge that streams both lists 32 elements at
// a time (merge-path, Sec. V-A) when their lengths are within a factor
// kSkew, else a binary search of the shorter list in the longer one
// (binary-search intersection, Sec. V-A).  Edges are handed to warps in
// chunks from an atomic work counter (dynamic load balance; consecutive
// edges share an endpoint, so its rows stay in L1).  Per-lane counts are
// reduced by warp shuffles, then one 64-bit atomic per block; counts are
// exact integers, so the summation order does not matter.
#include "internal.cuh"
#include "warp_isect.cuh"

namespace tc {

constexpr int kIsThreads = 256;
constexpr int kCoverChunk = 8;          // cover edges per work grab
constexpr int kPlainChunk = 64;         // CSR entries per work grab

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


// One cover edge i = (u, v) by segment-wise warp merges; returns the lane's
// share of c_uv and adds the list lengths streamed to *elems (lane 0).
__device__ __forceinline__ unsigned cover_edge_merge(int64_t i, const uint2* __restrict__ H,
                                                     const int64_t* __restrict__ off,
                                                     const uint32_t* __restrict__ scols,
                                                     const uint4* __restrict__ seg,
                                                     const unsigned long long* __restrict__ hoff,
                                                     unsigned long long* elems) {
  const int lane = threadIdx.x & 31;
  const uint2 e = H[i];
  const int64_t ou = off[e.x], eu = off[e.x + 1];
  const int64_t ov = off[e.y], ev = off[e.y + 1];
  const uint4 su = seg[e.x], sv = seg[e.y];
  const uint32_t* Ru = scols + ou;
  const uint32_t* Rv = scols + ov;
  // v is entry (i - hoff[u]) of u's same-level run above u, so the
  // same-level ids of u greater than v start right after it
  const uint32_t cut = su.y + (uint32_t)(i - (int64_t)hoff[e.x]) + 1u;
  unsigned c = warp_intersect(Ru, su.x, Rv, sv.x);                      // level l-1
  c += warp_intersect(Ru + cut, su.z - cut, Rv + sv.y, sv.z - sv.y);    // level l, > v
  c += warp_intersect(Ru + su.z, (eu - ou) - su.z, Rv + sv.z, (ev - ov) - sv.z);  // l+1
  if (lane == 0)
    *elems += (unsigned long long)(su.x + sv.x + (su.z - cut) + (sv.z - sv.y)) +
              (unsigned long long)((eu - ou) - su.z + (ev - ov) - sv.z);
  return c;
}

// Cover edges, warp per edge, chunks grabbed from *work (merge-only path,
// used when the edge count does not fit the 32-bit task lists).
__global__ void __launch_bounds__(kIsThreads)
k_cover_intersect(const uint2* __restrict__ H, int64_t nh, const int64_t* __restrict__ off,
                  const uint32_t* __restrict__ scols, const uint4* __restrict__ seg,
                  const unsigned long long* __restrict__ hoff,
                  uint32_t* __restrict__ per_edge, unsigned long long* work,
                  unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  unsigned long long acc = 0, elems = 0;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)kCoverChunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nh) break;
    const int64_t end = min((int64_t)base + kCoverChunk, nh);
    for (int64_t i = (int64_t)base; i < end; ++i) {
      const unsigned c = cover_edge_merge(i, H, off, scols, seg, hoff, &elems);
      acc += c;
      if (per_edge) {
        const unsigned long long t = warp_sum(c);
        if (lane == 0) per_edge[i] = (uint32_t)t;
      }
    }
  }
  block_add(acc, &ctrl[kCtrlCount]);
  __syncthreads();
  block_add(elems, &ctrl[kCtrlElems]);
}

// |A ∩ B| by one thread: a two-pointer merge of short sorted lists.
__device__ __forceinline__ unsigned thread_merge(const uint32_t* __restrict__ A, uint32_t la,
                                                 const uint32_t* __restrict__ B, uint32_t lb) {
  unsigned c = 0;
  uint32_t i = 0, j = 0;
  while (i < la && j < lb) {
    const uint32_t a = __ldg(A + i), b = __ldg(B + j);
    c += a == b;
    i += a <= b;
    j += b <= a;
  }
  return c;
}

constexpr uint32_t kThreadMerge = 48;  // list elements a single thread merges

// Edges listed by the bucketing step as having a small owner (both
// endpoints of degree <= the small-owner bound, or an owner whose edges are
// too few to pay for a hash table).  A warp takes 32 list entries, one per
// lane: a lane whose lists are short (at most kThreadMerge elements in all)
// merges them alone; the other entries are then merged by the whole warp,
// one at a time.  The list length is read from device memory
// (*nlist_dev), since the bucketing step appends to it on the GPU.
// mode 0 = cover (list holds H indices), 1 = plain (list holds CSR entry
// indices with u < v).
__global__ void __launch_bounds__(kIsThreads)
k_small_merge(int mode, const uint32_t* __restrict__ list, const unsigned long long* nlist_dev,
              const uint2* __restrict__ H, const int64_t* __restrict__ off,
              const uint32_t* __restrict__ scols, const uint4* __restrict__ seg,
              const unsigned long long* __restrict__ hoff, const uint32_t* __restrict__ erow,
              const uint32_t* __restrict__ cols, const int64_t* __restrict__ ustart,
              uint32_t* __restrict__ per_edge, unsigned long long* work, unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  const int64_t nlist = (int64_t)*nlist_dev;
  unsigned long long acc = 0, elems = 0;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nlist) break;
    const int64_t j = (int64_t)base + lane;
    int64_t i = -1;
    bool big = false;
    if (j < nlist) {
      i = list[j];
      unsigned c = 0;
      uint32_t len = 0;
      if (mode == 0) {
        const uint2 e = H[i];
        const int64_t ou = off[e.x], eu = off[e.x + 1];
        const int64_t ov = off[e.y], ev = off[e.y + 1];
        const uint4 su = seg[e.x], sv = seg[e.y];
        // v is entry (i - hoff[u]) of u's same-level run above u
        const uint32_t cut = su.y + (uint32_t)(i - (int64_t)hoff[e.x]) + 1u;
        const uint32_t du = (uint32_t)(eu - ou), dv = (uint32_t)(ev - ov);
        len = su.x + sv.x + (su.z - cut) + (sv.z - sv.y) + (du - su.z) + (dv - sv.z);
        if (len <= kThreadMerge) {
          const uint32_t* Ru = scols + ou;
          const uint32_t* Rv = scols + ov;
          c = thread_merge(Ru, su.x, Rv, sv.x) +                                // level l-1
              thread_merge(Ru + cut, su.z - cut, Rv + sv.y, sv.z - sv.y) +     // level l, > v
              thread_merge(Ru + su.z, du - su.z, Rv + sv.z, dv - sv.z);        // level l+1
        }
      } else {
        const uint32_t u = erow[i], v = cols[i];
        const int64_t au = i + 1, bv = ustart[v];
        const uint32_t la = (uint32_t)(off[u + 1] - au), lb = (uint32_t)(off[v + 1] - bv);
        len = la + lb;
        if (len <= kThreadMerge) c = thread_merge(cols + au, la, cols + bv, lb);
      }
      big = len > kThreadMerge;
      if (!big) {
        acc += c;
        elems += len;
        if (per_edge) per_edge[i] = c;
      }
    }
    // the long ones: the whole warp, one entry at a time
    unsigned m = __ballot_sync(0xFFFFFFFFu, big);
    while (m) {
      const int r = __ffs(m) - 1;
      m &= m - 1;
      const int64_t ir = __shfl_sync(0xFFFFFFFFu, i, r);
      unsigned c;
      if (mode == 0) {
        c = cover_edge_merge(ir, H, off, scols, seg, hoff, &elems);
      } else {
        const uint32_t u = erow[ir], v = cols[ir];
        const int64_t au = ir + 1, bv = ustart[v];
        const int64_t la = off[u + 1] - au, lb = off[v + 1] - bv;
        c = warp_intersect(cols + au, la, cols + bv, lb);
        if (lane == 0) elems += (unsigned long long)(la + lb);
      }
      acc += c;
      if (per_edge) {
        const unsigned long long t = warp_sum(c);
        if (lane == 0) per_edge[ir] = (uint32_t)t;
      }
    }
  }
  block_add(acc, &ctrl[kCtrlCount]);
  __syncthreads();
  block_add(elems, &ctrl[kCtrlElems]);
}

int merge_small_edges(tc_graph* g, int mode, const uint32_t* list,
                      const unsigned long long* nlist_dev, uint64_t nlist_max,
                      const int64_t* ustart, uint32_t* per_edge) {
  cudaStream_t s = g->stream;
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlWork, 0, sizeof(unsigned long long), s));
  launch(k_small_merge, grid_for((int64_t)nlist_max * 32, kIsThreads, 8), kIsThreads, 0, s, mode,
         list, nlist_dev, g->cover.p, g->off, g->scols.p, g->seg.p, g->hoff.p, g->erow.p, g->cols,
         ustart, per_edge, g->ctrl.p + kCtrlWork, g->ctrl.p);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// ustart[v] = index (into cols) of the first neighbour of v greater than v.
__global__ void k_upper_start(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                              uint32_t n, int64_t* __restrict__ ustart) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; v < (int64_t)n; v += stride) {
    int64_t lo = off[v], hi = off[v + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cols[mid] <= (uint32_t)v) lo = mid + 1; else hi = mid;
    }
    ustart[v] = lo;
  }
}

// Plain edge iterator: warp per CSR entry (u, v) with u < v.
__global__ void __launch_bounds__(kIsThreads)
k_plain_intersect(const uint32_t* __restrict__ erow, int64_t nnz, const int64_t* __restrict__ off,
                  const uint32_t* __restrict__ cols, const int64_t* __restrict__ ustart,
                  unsigned long long* work, unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  unsigned long long acc = 0, elems = 0;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)kPlainChunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nnz) break;
    const int64_t end = min((int64_t)base + kPlainChunk, nnz);
    for (int64_t e = (int64_t)base; e < end; ++e) {
      const uint32_t u = erow[e], v = cols[e];
      if (u >= v) continue;
      const int64_t au = e + 1, bv = ustart[v];
      const int64_t la = off[u + 1] - au, lb = off[v + 1] - bv;
      acc += warp_intersect(cols + au, la, cols + bv, lb);
      if (lane == 0) elems += (unsigned long long)(la + lb);
    }
  }
  block_add(acc, &ctrl[kCtrlCount]);
  __syncthreads();
  block_add(elems, &ctrl[kCtrlElems]);
}



// Stage timings: ev4 -> ev6 bucketing, ev6 -> ev7 hash kernel, ev7 -> ev5
// small-owner merge (the merge-only fallback records ev6 = ev7 = ev4).
static void finish_stats(tc_graph* g, bool hashed) {
  tc_stats_t& st = g->stats;
  st.list_elems = (int64_t)g->ctrl_host[kCtrlElems];
  st.ms_bucket = 0.f;
  if (hashed) {
    cudaEventElapsedTime(&st.ms_bucket, g->ev[4], g->ev[6]);
    cudaEventElapsedTime(&st.ms_main_kernel, g->ev[6], g->ev[7]);
    cudaEventElapsedTime(&st.ms_intersect, g->ev[6], g->ev[5]);
  } else {
    cudaEventElapsedTime(&st.ms_main_kernel, g->ev[4], g->ev[5]);
    st.ms_intersect = st.ms_main_kernel;
  }
  cudaGetLastError();  // a timing query that failed must not leak into later checks
}

// The merge kernels take work from ctrl[kCtrlWork] until it reaches their
// bound, so a range [first, last) starts the counter at first.
static int set_work_start(tc_graph* g, int64_t first) {
  const unsigned long long v = (unsigned long long)first;
  TC_CUDA(cudaMemcpyAsync(g->ctrl.p + kCtrlWork, &v, sizeof(v), cudaMemcpyHostToDevice, g->stream));
  return TC_OK;
}

int count_cover(tc_graph* g, uint32_t* per_edge_out, uint64_t* total, int64_t first,
                int64_t last, bool merge_only) {
  cudaStream_t s = g->stream;
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  if (last < 0 || last > g->num_cover) last = g->num_cover;
  if (first < 0) first = 0;
  if (first > last) first = last;
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlCount, 0, sizeof(unsigned long long), s));
  TC_TRY(set_work_start(g, first));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlElems, 0, sizeof(unsigned long long), s));
  if (per_edge_out && g->num_cover > 0)
    TC_CUDA(cudaMemsetAsync(per_edge_out, 0, sizeof(uint32_t) * (size_t)g->num_cover, s));
  const bool hashed = !merge_only && g->num_cover < (int64_t)0xFFFFFFFFll &&
                      g->nnz < (int64_t)0xFFFFFFFFll;
  cudaEventRecord(g->ev[4], s);
  if (hashed) {
    TC_TRY(hash_count(g, 0, nullptr, per_edge_out, first, last));
  } else if (last > first) {
    launch(k_cover_intersect, grid_for((last - first) * 32, kIsThreads, 8), kIsThreads, 0, s,
           g->cover.p, last, g->off, g->scols.p, g->seg.p, g->hoff.p, per_edge_out,
           g->ctrl.p + kCtrlWork, g->ctrl.p);
    TC_CUDA(cudaGetLastError());
  }
  cudaEventRecord(g->ev[5], s);
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  *total = g->ctrl_host[kCtrlCount];
  g->stats.edges_intersected = last - first;
  finish_stats(g, hashed && last > first);
  return TC_OK;
}

// per_entry (device, nnz entries, or NULL): the count of every CSR entry
// (u, v) with u < v; other entries are left 0.  Entries [first, last).
int count_plain(tc_graph* g, uint64_t* total, uint32_t* per_entry, int64_t first, int64_t last,
                bool merge_only) {
  cudaStream_t s = g->stream;
  if (last < 0 || last > g->nnz) last = g->nnz;
  if (first < 0) first = 0;
  if (first > last) first = last;
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlCount, 0, sizeof(unsigned long long), s));
  TC_TRY(set_work_start(g, first));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlElems, 0, sizeof(unsigned long long), s));
  g->stats.ms_intersect = g->stats.ms_bucket = g->stats.ms_main_kernel = 0.f;
  const bool hashed = !merge_only && g->nnz < (int64_t)0xFFFFFFFFll;
  if (per_entry && !hashed)
    return fail(TC_ERR_CAPACITY, "per-entry plain counts need nnz < 2^32");
  TC_TRY(ensure_erow(g));
  DevBuf<int64_t> ustart;
  if (last > first) {
    if (per_entry)
      TC_CUDA(cudaMemsetAsync(per_entry, 0, sizeof(uint32_t) * (size_t)g->nnz, s));
    TC_TRY(ustart.alloc(g->n, s));
    launch(k_upper_start, grid_for(g->n, kIsThreads), kIsThreads, 0, s, g->off, g->cols, g->n,
           ustart.p);
    cudaEventRecord(g->ev[4], s);
    if (hashed) {
      TC_TRY(hash_count(g, 1, ustart.p, per_entry, first, last));
    } else {
      launch(k_plain_intersect, grid_for((last - first) * 32, kIsThreads, 8), kIsThreads, 0, s,
             g->erow.p, last, g->off, g->cols, ustart.p, g->ctrl.p + kCtrlWork, g->ctrl.p);
      TC_CUDA(cudaGetLastError());
    }
    cudaEventRecord(g->ev[5], s);
  }
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  *total = g->ctrl_host[kCtrlCount];
  g->stats.edges_intersected = (last - first) / 2;
  if (last > first) finish_stats(g, hashed);
  return TC_OK;
}

}  // namespace tc

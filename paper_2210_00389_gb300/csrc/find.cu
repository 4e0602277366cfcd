// Triangle finding with the cover edges: per-vertex counts and the list of
// triangles, each triangle found exactly once.
//
// Alg. 1 of Bader et al., "Triangle Counting Through Cover-Edges" attributes
// every triangle to exactly one cover edge (Thm. 2: the single horizontal
// edge of a triangle with one, the (min, mid) edge of a triangle whose three
// vertices share a level), and for that edge (u, v) the apex w is one of the
// common neighbours the count-once rule accepts.  The kernel here is the
// warp-per-cover-edge merge over the level-segmented rows (segments l-1,
// "same level above v", l+1; see segment.cu), with a sink called on every
// accepted apex: it adds one to the apex's count, or appends (u, v, w) to
// the list.  Per-vertex counts go through the hash intersection of
// hashsect.cu, with a sink per hit, wherever it applies; this file's merge
// kernel then takes the small-owner edges (and whole graphs beyond the hash
// path's 32-bit task lists).
#include "internal.cuh"
#include "warp_isect.cuh"

namespace tc {

constexpr int kFindThreads = 256;
constexpr int kFindChunk = 8;  // cover edges per work grab

// Adds one to the apex's count.
struct VertexSink {
  unsigned long long* tv;
  __device__ __forceinline__ bool operator()(uint32_t w) const {
    atomicAdd(&tv[w], 1ull);
    return true;
  }
};

// Appends (u, v, w) to the list while there is room; every call counts.
struct ListSink {
  uint32_t* out;
  unsigned long long* next;
  unsigned long long cap;
  uint32_t u, v;
  __device__ __forceinline__ bool operator()(uint32_t w) const {
    const unsigned long long k = atomicAdd(next, 1ull);
    if (k < cap) {
      out[3 * k] = u;
      out[3 * k + 1] = v;
      out[3 * k + 2] = w;
    }
    return true;
  }
};

template <class Sink>
__device__ __forceinline__ unsigned find_edge(int64_t i, const uint2* __restrict__ H,
                                              const int64_t* __restrict__ off,
                                              const uint32_t* __restrict__ scols,
                                              const uint4* __restrict__ seg,
                                              const unsigned long long* __restrict__ hoff,
                                              Sink sink) {
  const uint2 e = H[i];
  const int64_t ou = off[e.x], eu = off[e.x + 1];
  const int64_t ov = off[e.y], ev = off[e.y + 1];
  const uint4 su = seg[e.x], sv = seg[e.y];
  const uint32_t* Ru = scols + ou;
  const uint32_t* Rv = scols + ov;
  // v is entry (i - hoff[u]) of u's same-level run above u
  const uint32_t cut = su.y + (uint32_t)(i - (int64_t)hoff[e.x]) + 1u;
  unsigned c = warp_intersect_if(Ru, su.x, Rv, sv.x, sink);                      // level l-1
  c += warp_intersect_if(Ru + cut, su.z - cut, Rv + sv.y, sv.z - sv.y, sink);    // level l, > v
  c += warp_intersect_if(Ru + su.z, (eu - ou) - su.z, Rv + sv.z, (ev - ov) - sv.z, sink);  // l+1
  return c;
}

__device__ __forceinline__ unsigned find_warp_sum(unsigned x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  return x;
}

// Warp per cover edge: per-vertex triangle counts.  The apex gets one per
// triangle from the sink; u and v get the edge's count.
__global__ void __launch_bounds__(kFindThreads)
k_find_vertex(const uint2* __restrict__ H, int64_t nh, const int64_t* __restrict__ off,
              const uint32_t* __restrict__ scols, const uint4* __restrict__ seg,
              const unsigned long long* __restrict__ hoff, unsigned long long* tv,
              unsigned long long* work) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)kFindChunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nh) break;
    const int64_t end = min((int64_t)base + kFindChunk, nh);
    for (int64_t i = (int64_t)base; i < end; ++i) {
      const unsigned c = find_warp_sum(find_edge(i, H, off, scols, seg, hoff, VertexSink{tv}));
      if (lane == 0 && c) {
        const uint2 e = H[i];
        atomicAdd(&tv[e.x], (unsigned long long)c);
        atomicAdd(&tv[e.y], (unsigned long long)c);
      }
    }
  }
}

// The same for the cover edges listed in list[0 .. *nlist_dev): the
// small-owner edges of the hashed path.
__global__ void __launch_bounds__(kFindThreads)
k_find_vertex_list(const uint32_t* __restrict__ list, const unsigned long long* nlist_dev,
                   const uint2* __restrict__ H, const int64_t* __restrict__ off,
                   const uint32_t* __restrict__ scols, const uint4* __restrict__ seg,
                   const unsigned long long* __restrict__ hoff, unsigned long long* tv,
                   unsigned long long* work) {
  const int lane = threadIdx.x & 31;
  const int64_t nl = (int64_t)*nlist_dev;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)kFindChunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nl) break;
    const int64_t end = min((int64_t)base + kFindChunk, nl);
    for (int64_t j = (int64_t)base; j < end; ++j) {
      const int64_t i = list[j];
      const unsigned c = find_warp_sum(find_edge(i, H, off, scols, seg, hoff, VertexSink{tv}));
      if (lane == 0 && c) {
        const uint2 e = H[i];
        atomicAdd(&tv[e.x], (unsigned long long)c);
        atomicAdd(&tv[e.y], (unsigned long long)c);
      }
    }
  }
}

// Warp per cover edge: every triangle as (u, v, w).
__global__ void __launch_bounds__(kFindThreads)
k_find_list(const uint2* __restrict__ H, int64_t nh, const int64_t* __restrict__ off,
            const uint32_t* __restrict__ scols, const uint4* __restrict__ seg,
            const unsigned long long* __restrict__ hoff, uint32_t* out, unsigned long long cap,
            unsigned long long* next, unsigned long long* work) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)kFindChunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nh) break;
    const int64_t end = min((int64_t)base + kFindChunk, nh);
    for (int64_t i = (int64_t)base; i < end; ++i) {
      const uint2 e = H[i];
      find_edge(i, H, off, scols, seg, hoff, ListSink{out, next, cap, e.x, e.y});
    }
  }
}

int find_vertex_list(tc_graph* g, const uint32_t* list, const unsigned long long* nlist_dev,
                     uint64_t nlist_max, unsigned long long* tv_dev) {
  cudaStream_t s = g->stream;
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlWork, 0, sizeof(unsigned long long), s));
  launch(k_find_vertex_list, grid_for((int64_t)nlist_max * 32, kFindThreads, 8), kFindThreads, 0,
         s, list, nlist_dev, g->cover.p, g->off, g->scols.p, g->seg.p, g->hoff.p, tv_dev,
         g->ctrl.p + kCtrlWork);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// Per-vertex counts: through the hash intersection (a sink per hit) when
// the edge and entry counts fit its 32-bit task lists, else by the merge.
int find_vertex_counts(tc_graph* g, unsigned long long* tv_dev) {
  cudaStream_t s = g->stream;
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  TC_CUDA(cudaMemsetAsync(tv_dev, 0, sizeof(unsigned long long) * (size_t)g->n, s));
  if (g->num_cover < (int64_t)0xFFFFFFFFll && g->nnz < (int64_t)0xFFFFFFFFll) {
    TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlCount, 0, sizeof(unsigned long long), s));
    TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlElems, 0, sizeof(unsigned long long), s));
    return hash_count(g, 0, nullptr, nullptr, 0, g->num_cover, tv_dev);
  }
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlWork, 0, sizeof(unsigned long long), s));
  if (g->num_cover > 0)
    launch(k_find_vertex, grid_for(g->num_cover * 32, kFindThreads, 8), kFindThreads, 0, s,
           g->cover.p, g->num_cover, g->off, g->scols.p, g->seg.p, g->hoff.p, tv_dev,
           g->ctrl.p + kCtrlWork);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int find_list(tc_graph* g, uint32_t* out_dev, unsigned long long cap, uint64_t* found) {
  cudaStream_t s = g->stream;
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlWork, 0, sizeof(unsigned long long), s));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlTmp, 0, sizeof(unsigned long long), s));
  if (g->num_cover > 0)
    launch(k_find_list, grid_for(g->num_cover * 32, kFindThreads, 8), kFindThreads, 0, s,
           g->cover.p, g->num_cover, g->off, g->scols.p, g->seg.p, g->hoff.p, out_dev, cap,
           g->ctrl.p + kCtrlTmp, g->ctrl.p + kCtrlWork);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host + kCtrlTmp, g->ctrl.p + kCtrlTmp,
                          sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  *found = g->ctrl_host[kCtrlTmp];
  return TC_OK;
}

}  // namespace tc

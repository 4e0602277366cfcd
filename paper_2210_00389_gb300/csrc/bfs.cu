// BFS levels (a1): Def. 2 and Alg. 1 of Bader et al., "Triangle
// Counting Through Cover-Edges".  L(v) is the shortest distance from the root
// of v's component.  Alg. 1 restarts a BFS from every unvisited vertex; here
// the restarts are batched.  Distances are unique given the roots, so the
// result equals the sequential restart order's.
//
// Root rule: the maximum-degree vertex r0 (lowest id on ties) roots its
// component; every other component is rooted at its lowest id.  That runs in
// two phases: a BFS from r0 alone, then connected components of the
// vertices it left unvisited (lock-free union-find with min-id roots, over
// their edges only) and one multi-source BFS from all of those roots at
// once.  With an explicit root list, the first listed root of each
// component roots it: components of the whole graph first, then one
// multi-source BFS.
//
// Each level runs top-down (frontier queue, load-balanced over the
// frontier's edges, warp-aggregated queue appends) or bottom-up (every
// unvisited vertex looks for a parent on the current level), switching by
// the frontier-edge heuristic of Beamer, Asanovic & Patterson (SC 2012).
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace tc {

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// find with path halving; parent pointers only ever decrease (a vertex
// points at a smaller id of its component), so shortcuts are safe.
__device__ __forceinline__ uint32_t uf_find(uint32_t* P, uint32_t x) {
  while (true) {
    uint32_t p = ld_volatile(&P[x]);
    if (p == x) return x;
    uint32_t gp = ld_volatile(&P[p]);
    if (gp == p) return p;
    P[x] = gp;
    x = gp;
  }
}

__global__ void k_cc_init(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                          uint32_t n, uint32_t* __restrict__ P) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride) {
    int64_t b = off[i];
    uint32_t first = (off[i + 1] > b) ? cols[b] : (uint32_t)i;  // smallest neighbour
    P[i] = first < (uint32_t)i ? first : (uint32_t)i;
  }
}

// Hook every edge (u > v) once: the larger root is attached to the smaller.
__global__ void k_cc_hook(const uint32_t* __restrict__ erow, const uint32_t* __restrict__ cols,
                          int64_t nnz, uint32_t* P) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < nnz; i += stride) {
    uint32_t u = erow[i], v = cols[i];
    if (v >= u) continue;
    while (true) {
      u = uf_find(P, u);
      v = uf_find(P, v);
      if (u == v) break;
      if (u < v) { uint32_t t = u; u = v; v = t; }
      if (atomicCAS(&P[u], u, v) == u) break;
    }
  }
}

__global__ void k_cc_flatten(uint32_t n, uint32_t* P) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride) P[i] = uf_find(P, (uint32_t)i);
}

// Components of the vertices a first BFS left unvisited (a component is
// either wholly visited or wholly unvisited): parents start at the smallest
// neighbour, and only edges of unvisited rows are hooked.
__global__ void k_cc_init_unvisited(const int64_t* __restrict__ off,
                                    const uint32_t* __restrict__ cols,
                                    const uint32_t* __restrict__ L, uint32_t n,
                                    uint32_t* __restrict__ P) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride) {
    const int64_t b = off[i];
    uint32_t first = (uint32_t)i;
    if (L[i] == kUnvisited && off[i + 1] > b) first = cols[b];
    P[i] = first < (uint32_t)i ? first : (uint32_t)i;
  }
}

// Warp per group of 32 vertices: the unvisited ones with edges are hooked
// one row at a time by the whole warp.
__global__ void k_cc_hook_unvisited(const int64_t* __restrict__ off,
                                    const uint32_t* __restrict__ cols,
                                    const uint32_t* __restrict__ L, uint32_t n, uint32_t* P) {
  const int lane = threadIdx.x & 31;
  int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; base < (int64_t)n; base += stride) {
    const int64_t x = base + lane;
    const bool want = x < (int64_t)n && L[x] == kUnvisited && off[x + 1] > off[x];
    unsigned m = __ballot_sync(0xFFFFFFFFu, want);
    while (m) {
      const uint32_t u0 = (uint32_t)base + (uint32_t)(__ffs(m) - 1);
      m &= m - 1;
      const int64_t b = off[u0], e = off[u0 + 1];
      for (int64_t i = b + lane; i < e; i += 32) {
        uint32_t u = u0, v = cols[i];
        if (v >= u) continue;
        while (true) {
          u = uf_find(P, u);
          v = uf_find(P, v);
          if (u == v) break;
          if (u < v) { uint32_t t = u; u = v; v = t; }
          if (atomicCAS(&P[u], u, v) == u) break;
        }
      }
    }
  }
}

// Level 0 for the second phase: the lowest id of every unvisited component.
__global__ void k_levels_unvisited_roots(uint32_t n, const uint32_t* __restrict__ P,
                                         uint32_t* __restrict__ L) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride)
    if (L[i] == kUnvisited && P[i] == (uint32_t)i) L[i] = 0u;
}

// first[c] = smallest index i of a listed root in component c
__global__ void k_roots_first(const uint32_t* __restrict__ roots, uint32_t nroots,
                              const uint32_t* __restrict__ P, uint32_t* first) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < nroots; i += gridDim.x * blockDim.x) atomicMin(&first[P[roots[i]]], i);
}

// Level 0: listed roots that come first in their component, and the lowest
// id of every component without a listed root.  Everything else unvisited.
__global__ void k_levels_init(uint32_t n, const uint32_t* __restrict__ P,
                              const uint32_t* __restrict__ first, uint32_t* __restrict__ L) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride)
    L[i] = (P[i] == (uint32_t)i && first[i] == kUnvisited) ? 0u : kUnvisited;
}

__global__ void k_levels_roots(const uint32_t* __restrict__ roots, uint32_t nroots,
                               const uint32_t* __restrict__ P, const uint32_t* __restrict__ first,
                               uint32_t* L) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < nroots; i += gridDim.x * blockDim.x) {
    uint32_t r = roots[i];
    if (first[P[r]] == i) L[r] = 0;
  }
}

// Warp-aggregated append of `v` (when take) to queue q with counter
// ctrl[kCtrlQ0]; its degree is added to ctrl[kCtrlQ1].  All 32 lanes call.
__device__ __forceinline__ void queue_append(bool take, uint32_t v, unsigned long long deg,
                                             uint32_t* q, unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  unsigned mask = __ballot_sync(0xFFFFFFFFu, take);
  unsigned long long dsum = take ? deg : 0ull;
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xFFFFFFFFu, dsum, o);
  if (mask == 0) return;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) {
    base = atomicAdd(&ctrl[kCtrlQ0], (unsigned long long)__popc(mask));
  }
  if (lane == 0) atomicAdd(&ctrl[kCtrlQ1], dsum);
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (take) q[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

// Level-0 queue: every root with at least one neighbour, except `skip`
// (a root whose BFS has already run; kUnvisited for none).
__global__ void k_queue_level0(uint32_t n, const int64_t* __restrict__ off,
                               const uint32_t* __restrict__ L, uint32_t skip, uint32_t* q,
                               unsigned long long* ctrl) {
  int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (; base < (int64_t)n; base += stride) {
    int64_t i = base + lane;
    bool take = false, root = false;
    unsigned long long d = 0;
    if (i < (int64_t)n && L[i] == 0) {
      root = true;
      d = (unsigned long long)(off[i + 1] - off[i]);
      take = d > 0 && (uint32_t)i != skip;
    }
    unsigned rmask = __ballot_sync(0xFFFFFFFFu, root);
    if (lane == 0 && rmask) atomicAdd(&ctrl[kCtrlTmp], (unsigned long long)__popc(rmask));
    queue_append(take, (uint32_t)i, d, q, ctrl);
  }
}

__global__ void k_queue_degrees(const uint32_t* __restrict__ q, int64_t f,
                                const int64_t* __restrict__ off, unsigned long long* ps) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < f; i += stride) {
    uint32_t u = q[i];
    ps[i] = (unsigned long long)(off[u + 1] - off[u]);
  }
}

// Top-down step, one thread per frontier edge: edge t belongs to the queue
// entry i with ps[i] <= t < ps[i+1] (binary search over the exclusive scan).
__global__ void k_bfs_topdown(const uint32_t* __restrict__ q, int64_t f,
                              const unsigned long long* __restrict__ ps, unsigned long long F,
                              const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                              uint32_t* L, uint32_t cur, uint32_t* qnext,
                              unsigned long long* ctrl) {
  int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (; base < (int64_t)F; base += stride) {
    int64_t t = base + lane;
    bool take = false;
    uint32_t w = 0;
    unsigned long long dw = 0;
    if (t < (int64_t)F) {
      int64_t lo = 0, hi = f;  // find last i with ps[i] <= t
      while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (ps[mid] <= (unsigned long long)t) lo = mid; else hi = mid;
      }
      uint32_t u = q[lo];
      int64_t e = off[u] + (t - (int64_t)ps[lo]);
      w = cols[e];
      if (ld_volatile(&L[w]) == kUnvisited && atomicCAS(&L[w], kUnvisited, cur + 1) == kUnvisited) {
        take = true;
        dw = (unsigned long long)(off[w + 1] - off[w]);
      }
    }
    queue_append(take, w, dw, qnext, ctrl);
  }
}

// Bottom-up step: every unvisited vertex scans its neighbours for one on
// level `cur`; found => level cur+1 and appended to the next queue.
__global__ void k_bfs_bottomup(uint32_t n, const int64_t* __restrict__ off,
                               const uint32_t* __restrict__ cols, uint32_t* L, uint32_t cur,
                               uint32_t* qnext, unsigned long long* ctrl) {
  int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (; base < (int64_t)n; base += stride) {
    int64_t v = base + lane;
    bool take = false;
    unsigned long long dv = 0;
    if (v < (int64_t)n && L[v] == kUnvisited) {
      int64_t b = off[v], e = off[v + 1];
      for (int64_t i = b; i < e; ++i) {
        if (ld_volatile(&L[cols[i]]) == cur) {
          take = true;
          break;
        }
      }
      if (take) {
        L[v] = cur + 1;
        dv = (unsigned long long)(e - b);
      }
    }
    queue_append(take, (uint32_t)v, dv, qnext, ctrl);
  }
}

__global__ void k_clear_q(unsigned long long* ctrl) {
  ctrl[kCtrlQ0] = 0;
  ctrl[kCtrlQ1] = 0;
}

// ---------------------------------------------------------------- driver

// Queue every level-0 vertex with neighbours (except `skip`) into q; sets
// g->nroots to the number of level-0 vertices (isolated ones included) and
// returns the queue's size and edge sum.
static int level0_queue(tc_graph* g, uint32_t* q, uint32_t skip, int64_t* f, int64_t* mf) {
  const int T = 256;
  cudaStream_t s = g->stream;
  launch(k_clear_q, 1, 1, 0, s, g->ctrl.p);
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlTmp, 0, sizeof(unsigned long long), s));
  launch(k_queue_level0, grid_for(g->n, T), T, 0, s, g->n, g->off, g->levels.p, skip, q,
         g->ctrl.p);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  TC_CUDA(cudaStreamSynchronize(s));
  *f = (int64_t)g->ctrl_host[kCtrlQ0];
  *mf = (int64_t)g->ctrl_host[kCtrlQ1];
  g->nroots = (uint32_t)g->ctrl_host[kCtrlTmp];
  return TC_OK;
}

// Level-synchronous BFS from the f vertices of qa (level 0, mf frontier
// edges); mu = edges of the vertices not yet visited, for the direction
// heuristic.  *nlev = the number of levels (>= 1); *visited and *edges_seen
// grow by the vertices and edges reached.  qa / qb are swapped as levels
// advance.
static int bfs_run(tc_graph* g, uint32_t*& qa, uint32_t*& qb, unsigned long long* ps, int64_t f,
                   int64_t mf, int64_t mu, uint32_t* nlev, int64_t* visited, int64_t* edges_seen) {
  const int T = 256;
  cudaStream_t s = g->stream;
  const uint32_t n = g->n;
  uint32_t* L = g->levels.p;
  uint32_t cur = 0;
  bool bottom_up = false;
  const int64_t alpha = 14, beta = 24;
  int64_t prev_f = f;
  while (f > 0) {
    if (!bottom_up) {
      if (mf > mu / alpha) bottom_up = true;
    } else if (f < (int64_t)n / beta && f < prev_f) {
      bottom_up = false;
    }
    launch(k_clear_q, 1, 1, 0, s, g->ctrl.p);
    if (bottom_up) {
      launch(k_bfs_bottomup, grid_for(n, T, 16), T, 0, s, n, g->off, g->cols, L, cur, qb, g->ctrl.p);
      g->stats.bfs_bottom_up++;
    } else {
      launch(k_queue_degrees, grid_for(f, T), T, 0, s, qa, f, g->off, ps);
      TC_TRY(exclusive_scan_u64(ps, f, nullptr, s));
      launch(k_bfs_topdown, grid_for(mf, T, 16), T, 0, s, qa, f, ps, (unsigned long long)mf, g->off,
             g->cols, L, cur, qb, g->ctrl.p);
    }
    TC_CUDA(cudaGetLastError());
    TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    g->stats.bfs_levels++;
    prev_f = f;
    f = (int64_t)g->ctrl_host[kCtrlQ0];
    mf = (int64_t)g->ctrl_host[kCtrlQ1];
    mu -= mf;
    *visited += f;
    *edges_seen += mf;
    if (f > 0) cur++;
    std::swap(qa, qb);
  }
  *nlev = cur + 1;
  return TC_OK;
}

int compute_levels(tc_graph* g, const uint32_t* roots_host, uint32_t nroots) {
  const int T = 256;
  cudaStream_t s = g->stream;
  const uint32_t n = g->n;
  g->cover.release();
  g->num_cover = -1;
  g->seg_valid = false;
  g->nlevels = -1;
  g->stats.bfs_levels = 0;
  g->stats.bfs_bottom_up = 0;
  if (n == 0) {
    g->nlevels = 0;
    g->nroots = 0;
    return TC_OK;
  }
  TC_TRY(g->levels.reserve(n, s));
  uint32_t* L = g->levels.p;

  DevBuf<uint32_t> q0, q1;
  DevBuf<unsigned long long> ps;
  TC_TRY(q0.alloc(n, s));
  TC_TRY(q1.alloc(n, s));
  TC_TRY(ps.alloc((size_t)n + 1, s));
  uint32_t* qa = q0.p;
  uint32_t* qb = q1.p;
  uint32_t nlev = 0;

  if (!(roots_host && nroots > 0)) {
    // Default root rule in two phases.  Phase 1: BFS from r0 alone.
    TC_CUDA(cudaMemsetAsync(L, 0xFF, sizeof(uint32_t) * n, s));
    TC_CUDA(cudaMemsetAsync(L + g->r0, 0, sizeof(uint32_t), s));
    const uint32_t r0 = g->r0;
    TC_CUDA(cudaMemcpyAsync(qa, &r0, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    const int64_t d0 = (int64_t)g->max_degree;
    int64_t visited = 1, edges_seen = d0;
    TC_TRY(bfs_run(g, qa, qb, ps.p, d0 > 0 ? 1 : 0, d0, g->nnz - d0, &nlev, &visited, &edges_seen));
    g->nroots = 1;
    if (visited < (int64_t)n) {
      // Phase 2: components of the unvisited vertices (min-id roots), then
      // one multi-source BFS from all of their roots.
      DevBuf<uint32_t> P;
      TC_TRY(P.alloc(n, s));
      launch(k_cc_init_unvisited, grid_for(n, T), T, 0, s, g->off, g->cols, L, n, P.p);
      if (g->nnz > 0)
        launch(k_cc_hook_unvisited, grid_for(n, T), T, 0, s, g->off, g->cols, L, n, P.p);
      launch(k_cc_flatten, grid_for(n, T), T, 0, s, n, P.p);
      launch(k_levels_unvisited_roots, grid_for(n, T), T, 0, s, n, P.p, L);
      int64_t f, mf;
      TC_TRY(level0_queue(g, qa, r0, &f, &mf));
      uint32_t nlev2 = 0;
      TC_TRY(bfs_run(g, qa, qb, ps.p, f, mf, g->nnz - edges_seen - mf, &nlev2, &visited,
                     &edges_seen));
      nlev = std::max(nlev, nlev2);
    }
    g->nlevels = (int64_t)nlev;
    return TC_OK;
  }

  // Explicit roots: components of the whole graph, then one multi-source BFS
  // from the first listed root of each component and the lowest id of every
  // other component.
  std::vector<uint32_t> rl(roots_host, roots_host + nroots);
  for (uint32_t r : rl)
    if (r >= n) return fail(TC_ERR_INVALID_ARG, "tc_bfs_levels: root %u >= n", r);
  DevBuf<uint32_t> P, first, droots;
  TC_TRY(P.alloc(n, s));
  TC_TRY(first.alloc(n, s));
  TC_TRY(droots.alloc(rl.size(), s));
  TC_CUDA(cudaMemcpyAsync(droots.p, rl.data(), rl.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s));
  TC_TRY(ensure_erow(g));
  launch(k_cc_init, grid_for(n, T), T, 0, s, g->off, g->cols, n, P.p);
  if (g->nnz > 0) launch(k_cc_hook, grid_for(g->nnz, T), T, 0, s, g->erow.p, g->cols, g->nnz, P.p);
  launch(k_cc_flatten, grid_for(n, T), T, 0, s, n, P.p);
  TC_CUDA(cudaMemsetAsync(first.p, 0xFF, sizeof(uint32_t) * n, s));
  const uint32_t nr = (uint32_t)rl.size();
  launch(k_roots_first, grid_for(nr, T), T, 0, s, droots.p, nr, P.p, first.p);
  launch(k_levels_init, grid_for(n, T), T, 0, s, n, P.p, first.p, L);
  launch(k_levels_roots, grid_for(nr, T), T, 0, s, droots.p, nr, P.p, first.p, L);
  int64_t f, mf;
  TC_TRY(level0_queue(g, qa, kUnvisited, &f, &mf));
  int64_t visited = 0, edges_seen = 0;
  TC_TRY(bfs_run(g, qa, qb, ps.p, f, mf, g->nnz - mf, &nlev, &visited, &edges_seen));
  g->nlevels = (int64_t)nlev;
  return TC_OK;
}

}  // namespace tc

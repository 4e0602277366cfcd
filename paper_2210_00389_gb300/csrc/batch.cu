// Batched counting of many independent graphs (tc_count_batch).
//
// One persistent kernel: every CTA takes graphs from a global queue (largest
// first) and runs the whole method on each within the block, with its
// per-graph arrays in a per-CTA slice of one scratch arena:
//   checks   offsets monotone and ending at nnz; columns < n, rows strictly
//            ascending, no self-loops (a failing graph gets
//            TC_ERR_INVALID_GRAPH and is skipped);
//   roots    maximum-degree vertex (lowest id on ties), and the lowest id of
//            every other component (union-find with min-id roots), as in
//            Def. 2 / Alg. 1 of Bader et al., "Triangle Counting Through
//            Cover-Edges";
//   levels   one multi-source, level-synchronous BFS inside the block;
//   count    for every cover edge (u, v) (Thm. 1: L(u) = L(v), u < v) the
//            common neighbours w with L(w) != L(u) or w > v (Alg. 1 /
//            Thm. 2), by warp merge; plain mode counts every edge u < v with
//            apexes w > v;
//   reduce   warp shuffles, then one 64-bit store per graph.
// There is no host synchronisation per BFS level or per graph.  The launch
// is captured into a CUDA graph on an internal stream and replayed on the
// caller's stream.  Graphs with more than kBatchMaxN vertices or
// kBatchMaxNnz entries go to the union path below instead.
#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.cuh"
#include "warp_isect.cuh"

namespace tc {

constexpr uint32_t kBatchMaxN = 1u << 16;     // vertices per graph in the batch kernel
constexpr int64_t kBatchMaxNnz = 1ll << 15;   // entries per graph (default; tc_options)

struct BGraph {
  const int64_t* off;
  const uint32_t* cols;
  uint32_t n;
  uint32_t pad;
  int64_t nnz;
};

__device__ __forceinline__ uint32_t bfind(uint32_t* P, uint32_t x) {
  while (true) {
    const uint32_t p = *reinterpret_cast<volatile uint32_t*>(&P[x]);
    if (p == x) return x;
    const uint32_t gp = *reinterpret_cast<volatile uint32_t*>(&P[p]);
    if (gp == p) return p;
    P[x] = gp;  // path halving; parents only ever point to smaller ids
    x = gp;
  }
}

struct CoverPred {
  const uint32_t* L;
  uint32_t lvl, v;
  __device__ __forceinline__ bool operator()(uint32_t w) const { return L[w] != lvl || w > v; }
};

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_batch(const BGraph* __restrict__ graphs, const uint32_t* __restrict__ order, int32_t ngraphs,
        int mode, int64_t skew, uint32_t* __restrict__ scratch, uint32_t slot_n,
        unsigned long long* __restrict__ counts, int* __restrict__ status,
        unsigned long long* queue) {
  constexpr int kWarps = THREADS / 32;
  __shared__ int s_idx;
  __shared__ unsigned long long s_key;
  __shared__ uint32_t s_qn;
  __shared__ unsigned long long s_red[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* L = scratch + (size_t)blockIdx.x * 4 * slot_n;
  uint32_t* P = L + slot_n;
  uint32_t* qa = P + slot_n;
  uint32_t* qb = qa + slot_n;
  while (true) {
    if (threadIdx.x == 0) {
      s_idx = (int)atomicAdd(queue, 1ull);
      s_key = 0;
      s_qn = 0;
    }
    __syncthreads();
    const int qi = s_idx;
    if (qi >= ngraphs) break;
    const int gi = (int)order[qi];
    const BGraph G = graphs[gi];
    const uint32_t n = G.n;
    const int64_t* off = G.off;
    const uint32_t* cols = G.cols;
    // -- checks: offsets first (they bound every later access)
    bool bad = false;
    for (uint32_t v = threadIdx.x; v <= n; v += THREADS) {
      const int64_t o = off[v];
      if (o < 0 || o > G.nnz || (v == 0 && o != 0) || (v == n && o != G.nnz)) bad = true;
      else if (v < n && off[v + 1] < o) bad = true;
    }
    if (__syncthreads_or(bad)) {
      if (threadIdx.x == 0) { status[gi] = TC_ERR_INVALID_GRAPH; counts[gi] = 0; }
      continue;
    }
    for (uint32_t v = wid; v < n; v += kWarps) {
      const int64_t b = off[v], e = off[v + 1];
      for (int64_t i = b + lane; i < e; i += 32) {
        const uint32_t w = cols[i];
        if (w >= n || w == v || (i > b && cols[i - 1] >= w)) bad = true;
      }
      const unsigned long long d = (unsigned long long)(e - b);
      if (lane == 0) atomicMax(&s_key, (d << 32) | (0xFFFFFFFFull - v));
    }
    if (__syncthreads_or(bad)) {
      if (threadIdx.x == 0) { status[gi] = TC_ERR_INVALID_GRAPH; counts[gi] = 0; }
      continue;
    }
    const uint32_t r0 = n > 0 ? 0xFFFFFFFFu - (uint32_t)(s_key & 0xFFFFFFFFull) : 0u;
    // -- components: parents point to smaller ids, so every root is its
    //    component's minimum
    for (uint32_t v = threadIdx.x; v < n; v += THREADS) {
      const int64_t b = off[v];
      const uint32_t f = off[v + 1] > b ? cols[b] : v;
      P[v] = f < v ? f : v;
    }
    __syncthreads();
    for (uint32_t v = wid; v < n; v += kWarps) {
      const int64_t b = off[v], e = off[v + 1];
      for (int64_t i = b + lane; i < e; i += 32) {
        uint32_t x = v, y = cols[i];
        if (y >= x) continue;
        while (true) {
          x = bfind(P, x);
          y = bfind(P, y);
          if (x == y) break;
          if (x < y) { const uint32_t t = x; x = y; y = t; }
          if (atomicCAS(&P[x], x, y) == x) break;
        }
      }
    }
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < n; v += THREADS) P[v] = bfind(P, v);
    __syncthreads();
    // -- level 0: r0 and the lowest id of every other component
    const uint32_t c0 = n > 0 ? P[r0] : 0u;
    for (uint32_t v = threadIdx.x; v < n; v += THREADS) {
      const bool root = v == r0 || (P[v] == v && v != c0);
      L[v] = root ? 0u : kUnvisited;
      if (root && off[v + 1] > off[v]) qa[atomicAdd(&s_qn, 1u)] = v;
    }
    __syncthreads();
    // -- level-synchronous BFS, top-down, frontier queues in scratch
    uint32_t qn = s_qn;
    uint32_t cur = 0;
    while (qn > 0) {
      __syncthreads();
      if (threadIdx.x == 0) s_qn = 0;
      __syncthreads();
      for (uint32_t k = wid; k < qn; k += kWarps) {
        const uint32_t x = qa[k];
        const int64_t b = off[x], e = off[x + 1];
        for (int64_t i = b + lane; i < e; i += 32) {
          const uint32_t y = cols[i];
          if (L[y] == kUnvisited && atomicCAS(&L[y], kUnvisited, cur + 1) == kUnvisited)
            qb[atomicAdd(&s_qn, 1u)] = y;
        }
      }
      __syncthreads();
      qn = s_qn;
      uint32_t* t = qa; qa = qb; qb = t;
      ++cur;
    }
    __syncthreads();
    // -- counting: warp per vertex u, cover edges (or all edges u < v)
    unsigned long long acc = 0;
    for (uint32_t u = wid; u < n; u += kWarps) {
      const int64_t b = off[u], e = off[u + 1];
      const uint32_t lvl = L[u];
      for (int64_t base = b; base < e; base += 32) {
        const int64_t i = base + lane;
        bool cand = false;
        uint32_t v = 0;
        if (i < e) {
          v = cols[i];
          cand = v > u && (mode == TC_MODE_PLAIN || L[v] == lvl);
        }
        unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
        while (m) {
          const int j = __ffs(m) - 1;
          m &= m - 1;
          const uint32_t vv = __shfl_sync(0xFFFFFFFFu, v, j);
          const int64_t bv = off[vv], ev = off[vv + 1];
          if (mode == TC_MODE_COVER) {
            acc += warp_intersect_if(cols + b, e - b, cols + bv, ev - bv, CoverPred{L, lvl, vv},
                                     skew);
          } else {
            // neighbours above vv: after entry (base + j) in u's row, and
            // after vv's own position in its row
            int64_t lo = bv, hi = ev;
            while (lo < hi) {
              const int64_t mid = (lo + hi) >> 1;
              if (cols[mid] <= vv) lo = mid + 1; else hi = mid;
            }
            const int64_t au = base + j + 1;
            acc += warp_intersect_if(cols + au, e - au, cols + lo, ev - lo, AcceptAll(), skew);
          }
        }
      }
    }
    // -- reduction to one count per graph
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) s_red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kWarps; ++w) t += s_red[w];
      counts[gi] = t;
      status[gi] = TC_OK;
    }
  }
}

template <int THREADS>
static void launch_batch(int grid, cudaStream_t s, const BGraph* graphs, const uint32_t* order,
                         int32_t ng, int mode, int64_t skew, uint32_t* scratch, uint32_t slot_n,
                         unsigned long long* counts, int* status, unsigned long long* queue) {
  launch(k_batch<THREADS>, grid, THREADS, 0, s, graphs, order, ng, mode, skew, scratch, slot_n,
         counts, status, queue);
}

// Grow-only pinned staging buffer, one per host thread, kept until the
// thread exits: freeing pinned memory (cudaFreeHost) synchronises the whole
// device, which would serialise concurrent callers such as the server's
// workers.
struct PinnedStaging {
  unsigned char* p = nullptr;
  size_t n = 0;
  ~PinnedStaging() {
    if (p) cudaFreeHost(p);
  }
};

static unsigned char* pinned_staging(size_t bytes) {
  static thread_local PinnedStaging st;
  if (st.n >= bytes) return st.p;
  const size_t want = std::max(bytes, st.n * 2);
  if (st.p) cudaFreeHost(st.p);
  st.p = nullptr;
  st.n = 0;
  if (cudaMallocHost(reinterpret_cast<void**>(&st.p), want) != cudaSuccess) {
    cudaGetLastError();
    st.p = nullptr;
    return nullptr;
  }
  st.n = want;
  return st.p;
}


// ---------------------------------------------------------------- union path
// Members too large for one CTA are counted together: they are packed into
// one disjoint-union graph (vertex ids and entry positions shifted), counted
// once by the single-graph pipeline (levels, segmented rows, bucketing, hash
// intersection) with per-edge counts, and each member's count is the sum of
// its own contiguous range of per-edge counts.  Counts do not depend on the
// BFS roots (Thm. 2 holds for any BFS), so the union's roots give every
// member its exact count.

// Block per member: the same CSR checks as the batch kernel.
__global__ void k_member_check(const BGraph* __restrict__ graphs, int32_t nm, int* __restrict__ st) {
  for (int32_t m = blockIdx.x; m < nm; m += gridDim.x) {
    const BGraph G = graphs[m];
    bool bad = false;
    for (uint32_t v = threadIdx.x; v <= G.n; v += blockDim.x) {
      const int64_t o = G.off[v];
      if (o < 0 || o > G.nnz || (v == 0 && o != 0) || (v == G.n && o != G.nnz)) bad = true;
      else if (v < G.n && G.off[v + 1] < o) bad = true;
    }
    if (__syncthreads_or(bad)) {
      if (threadIdx.x == 0) st[m] = TC_ERR_INVALID_GRAPH;
      continue;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t v = wid; v < G.n; v += nw) {
      const int64_t b = G.off[v], e = G.off[v + 1];
      for (int64_t i = b + lane; i < e; i += 32) {
        const uint32_t w = G.cols[i];
        if (w >= G.n || w == v || (i > b && G.cols[i - 1] >= w)) bad = true;
      }
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) st[m] = bad ? TC_ERR_INVALID_GRAPH : TC_OK;
  }
}

// Block per packed member: shifted offsets and column ids.
__global__ void k_member_pack(const BGraph* __restrict__ graphs, const uint32_t* __restrict__ mem,
                              const unsigned long long* __restrict__ vbase,
                              const unsigned long long* __restrict__ ebase, int32_t np,
                              int64_t* __restrict__ uoff, uint32_t* __restrict__ ucols) {
  for (int32_t k = blockIdx.x; k < np; k += gridDim.x) {
    const BGraph G = graphs[mem[k]];
    const unsigned long long vb = vbase[k], eb = ebase[k];
    for (uint32_t v = threadIdx.x; v < G.n; v += blockDim.x) uoff[vb + v] = (int64_t)eb + G.off[v];
    for (int64_t i = threadIdx.x; i < G.nnz; i += blockDim.x)
      ucols[eb + i] = (uint32_t)vb + G.cols[i];
  }
}

// Block per packed member: sum of its per-edge counts.  Cover edges of a
// member are H[hoff[vb] .. hoff[vb + n]) (H is in vertex order); plain
// entries are [eb, eb + nnz).
__global__ void k_member_sums(const BGraph* __restrict__ graphs, const uint32_t* __restrict__ mem,
                              const unsigned long long* __restrict__ vbase,
                              const unsigned long long* __restrict__ ebase, int32_t np, int mode,
                              const unsigned long long* __restrict__ hoff, uint64_t total_n,
                              uint64_t num_cover, const uint32_t* __restrict__ per_edge,
                              unsigned long long* __restrict__ out) {
  __shared__ unsigned long long red[32];
  for (int32_t k = blockIdx.x; k < np; k += gridDim.x) {
    const BGraph G = graphs[mem[k]];
    unsigned long long a, b;
    if (mode == TC_MODE_COVER) {
      const unsigned long long ve = vbase[k] + G.n;
      a = hoff[vbase[k]];
      b = ve < total_n ? hoff[ve] : num_cover;
    } else {
      a = ebase[k];
      b = ebase[k] + (unsigned long long)G.nnz;
    }
    unsigned long long s = 0;
    for (unsigned long long i = a + threadIdx.x; i < b; i += blockDim.x) s += per_edge[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      out[k] = t;
    }
    __syncthreads();
  }
}

// Device descriptors for graphs[idx[...]]: device views are used in place,
// host views are staged through pinned memory into one device arena.
static int make_descs(const tc_csr_view* graphs, const std::vector<int32_t>& idx, cudaStream_t cs,
                      std::vector<BGraph>& hg, DevBuf<unsigned char>& arena) {
  size_t host_bytes = 0;
  for (int32_t i : idx) {
    const tc_csr_view& v = graphs[i];
    if (!(v.on_device && is_device_ptr(v.offsets))) {
      host_bytes += (sizeof(int64_t) * ((size_t)v.n + 1) + 15) & ~(size_t)15;
      host_bytes += (sizeof(uint32_t) * (size_t)v.nnz + 15) & ~(size_t)15;
    }
  }
  unsigned char* pinned = nullptr;
  if (host_bytes > 0) {
    if (!(pinned = pinned_staging(host_bytes)))
      return fail(TC_ERR_OOM, "tc_count_batch: pinned staging of %zu bytes failed", host_bytes);
    TC_TRY(arena.alloc(host_bytes, cs));
  }
  hg.resize(idx.size());
  size_t pos = 0;
  for (size_t k = 0; k < idx.size(); ++k) {
    const tc_csr_view& v = graphs[idx[k]];
    BGraph b{};
    b.n = v.n;
    b.nnz = v.nnz;
    if (v.on_device && is_device_ptr(v.offsets)) {
      b.off = v.offsets;
      b.cols = v.cols;
    } else {
      const size_t ob = sizeof(int64_t) * ((size_t)v.n + 1);
      memcpy(pinned + pos, v.offsets, ob);
      b.off = reinterpret_cast<const int64_t*>(arena.p + pos);
      pos = (pos + ob + 15) & ~(size_t)15;
      const size_t cb = sizeof(uint32_t) * (size_t)v.nnz;
      if (cb) memcpy(pinned + pos, v.cols, cb);
      b.cols = reinterpret_cast<const uint32_t*>(arena.p + pos);
      pos = (pos + cb + 15) & ~(size_t)15;
    }
    hg[k] = b;
  }
  if (host_bytes > 0)
    TC_CUDA(cudaMemcpyAsync(arena.p, pinned, host_bytes, cudaMemcpyHostToDevice, cs));
  // the staging buffer is reused by the next call on this thread
  TC_CUDA(cudaStreamSynchronize(cs));
  return TC_OK;
}

// One cached executable graph per host thread and device (see run_tiny).
struct ExecCache {
  cudaGraphExec_t exec = nullptr;
  ~ExecCache() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};
static ExecCache& exec_cache() {
  thread_local ExecCache per_device[16];
  int dev = 0;
  cudaGetDevice(&dev);
  return per_device[dev >= 0 && dev < 16 ? dev : 0];
}

// Tiny members: one persistent launch, captured into a CUDA graph on `cs`
// and replayed on `user`.
static int run_tiny(const tc_csr_view* graphs, const std::vector<int32_t>& idx, int mode,
                    int threads, int per_sm, int64_t skew, cudaStream_t cs, cudaStream_t user,
                    std::vector<unsigned long long>& cnt, std::vector<int>& st) {
  std::vector<BGraph> hg;
  DevBuf<unsigned char> arena;
  TC_TRY(make_descs(graphs, idx, cs, hg, arena));
  uint32_t max_n = 1;
  for (const BGraph& b : hg) max_n = std::max(max_n, b.n + 1);
  std::vector<uint32_t> ord(hg.size());  // largest graphs first
  std::iota(ord.begin(), ord.end(), 0u);
  std::stable_sort(ord.begin(), ord.end(),
                   [&](uint32_t a, uint32_t b) { return hg[a].nnz > hg[b].nnz; });
  const int grid = (int)std::min<int64_t>((int64_t)sm_count() * per_sm, (int64_t)hg.size());
  DevBuf<BGraph> dgraphs;
  DevBuf<uint32_t> dorder, scratch;
  DevBuf<unsigned long long> dcounts, dqueue;
  DevBuf<int> dstatus;
  TC_TRY(dgraphs.alloc(hg.size(), cs));
  TC_TRY(dorder.alloc(ord.size(), cs));
  TC_TRY(dcounts.alloc(hg.size(), cs));
  TC_TRY(dstatus.alloc(hg.size(), cs));
  TC_TRY(dqueue.alloc(1, cs));
  TC_TRY(scratch.alloc((size_t)grid * 4 * max_n, cs));
  TC_CUDA(cudaMemcpyAsync(dgraphs.p, hg.data(), sizeof(BGraph) * hg.size(), cudaMemcpyHostToDevice,
                          cs));
  TC_CUDA(cudaMemcpyAsync(dorder.p, ord.data(), sizeof(uint32_t) * ord.size(),
                          cudaMemcpyHostToDevice, cs));
  TC_CUDA(cudaStreamSynchronize(cs));
  cudaGraph_t cg = nullptr;
  cudaGraphExec_t exec = nullptr;
  TC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(dqueue.p, 0, sizeof(unsigned long long), cs);
  const int32_t ng = (int32_t)hg.size();
  if (threads == 128)
    launch_batch<128>(grid, cs, dgraphs.p, dorder.p, ng, mode, skew, scratch.p, max_n, dcounts.p,
                      dstatus.p, dqueue.p);
  else if (threads == 256)
    launch_batch<256>(grid, cs, dgraphs.p, dorder.p, ng, mode, skew, scratch.p, max_n, dcounts.p,
                      dstatus.p, dqueue.p);
  else
    launch_batch<512>(grid, cs, dgraphs.p, dorder.p, ng, mode, skew, scratch.p, max_n, dcounts.p,
                      dstatus.p, dqueue.p);
  TC_CUDA(cudaStreamEndCapture(cs, &cg));
  // The executable graph is kept per host thread and device: a later call
  // captures its own (same-shaped) graph and updates the cached executable
  // in place with the new parameters instead of instantiating it again; a
  // capture of another shape (another block size) re-instantiates.
  ExecCache& ec = exec_cache();
  cudaError_t e = cudaSuccess;
  if (ec.exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ec.exec, cg, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(ec.exec);
      ec.exec = nullptr;
    }
  }
  if (!ec.exec) e = cudaGraphInstantiate(&ec.exec, cg, 0);
  exec = ec.exec;
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, user);
  std::vector<unsigned long long> c(hg.size());
  std::vector<int> s(hg.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.data(), dcounts.p, sizeof(unsigned long long) * c.size(),
                        cudaMemcpyDeviceToHost, user);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s.data(), dstatus.p, sizeof(int) * s.size(), cudaMemcpyDeviceToHost, user);
  if (e == cudaSuccess) e = cudaStreamSynchronize(user);
  if (cg) cudaGraphDestroy(cg);
  if (e != cudaSuccess) return cuda_fail(e, "batched launch", __FILE__, __LINE__);
  for (size_t k = 0; k < idx.size(); ++k) {
    cnt[idx[k]] = c[k];
    st[idx[k]] = s[k];
  }
  return TC_OK;
}

static int run_union(const tc_csr_view* graphs, const std::vector<int32_t>& idx, int mode,
                     cudaStream_t cs, std::vector<unsigned long long>& cnt, std::vector<int>& st) {
  std::vector<BGraph> hg;
  DevBuf<unsigned char> arena;
  TC_TRY(make_descs(graphs, idx, cs, hg, arena));
  const int32_t nm = (int32_t)hg.size();
  DevBuf<BGraph> dgraphs;
  DevBuf<int> dst;
  TC_TRY(dgraphs.alloc(hg.size(), cs));
  TC_TRY(dst.alloc(hg.size(), cs));
  TC_CUDA(cudaMemcpyAsync(dgraphs.p, hg.data(), sizeof(BGraph) * hg.size(), cudaMemcpyHostToDevice,
                          cs));
  launch(k_member_check, std::min(nm, sm_count() * 8), 256, 0, cs, dgraphs.p, nm, dst.p);
  std::vector<int> mst(hg.size());
  TC_CUDA(cudaMemcpyAsync(mst.data(), dst.p, sizeof(int) * mst.size(), cudaMemcpyDeviceToHost, cs));
  TC_CUDA(cudaStreamSynchronize(cs));
  // valid members and their vertex / entry bases in the union
  std::vector<uint32_t> mem;
  std::vector<unsigned long long> vb, eb;
  unsigned long long tn = 0, te = 0;
  for (int32_t k = 0; k < nm; ++k) {
    st[idx[k]] = mst[k];
    cnt[idx[k]] = 0;
    if (mst[k] != TC_OK) continue;
    mem.push_back((uint32_t)k);
    vb.push_back(tn);
    eb.push_back(te);
    tn += hg[k].n;
    te += (unsigned long long)hg[k].nnz;
  }
  if (mem.empty()) return TC_OK;
  if (tn >= 0xFFFFFFFFull || te >= 0xFFFFFFFFull)
    return fail(TC_ERR_CAPACITY, "tc_count_batch: union of large graphs exceeds 2^32 ids/entries");
  const int32_t np = (int32_t)mem.size();
  DevBuf<uint32_t> dmem, ucols;
  DevBuf<unsigned long long> dvb, deb, dout;
  DevBuf<int64_t> uoff;
  TC_TRY(dmem.alloc(mem.size(), cs));
  TC_TRY(dvb.alloc(vb.size(), cs));
  TC_TRY(deb.alloc(eb.size(), cs));
  TC_TRY(dout.alloc(mem.size(), cs));
  TC_TRY(uoff.alloc((size_t)tn + 1, cs));
  TC_TRY(ucols.alloc((size_t)te, cs));
  TC_CUDA(cudaMemcpyAsync(dmem.p, mem.data(), sizeof(uint32_t) * mem.size(), cudaMemcpyHostToDevice,
                          cs));
  TC_CUDA(cudaMemcpyAsync(dvb.p, vb.data(), sizeof(unsigned long long) * vb.size(),
                          cudaMemcpyHostToDevice, cs));
  TC_CUDA(cudaMemcpyAsync(deb.p, eb.data(), sizeof(unsigned long long) * eb.size(),
                          cudaMemcpyHostToDevice, cs));
  const int64_t last = (int64_t)te;
  TC_CUDA(cudaMemcpyAsync(uoff.p + tn, &last, sizeof(int64_t), cudaMemcpyHostToDevice, cs));
  launch(k_member_pack, std::min(np, sm_count() * 8), 256, 0, cs, dgraphs.p, dmem.p, dvb.p, deb.p,
         np, uoff.p, ucols.p);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaStreamSynchronize(cs));  // `last` lives on this stack frame
  tc_csr_view uv{uoff.p, ucols.p, (uint32_t)tn, (int64_t)te, 1};
  tc_graph* g = nullptr;
  TC_TRY(tc_graph_create(&uv, TC_GRAPH_BORROW, cs, &g));
  int rc = TC_OK;
  DevBuf<uint32_t> per_edge;
  uint64_t total = 0;
  if (mode == TC_MODE_COVER) {
    rc = compute_cover(g);
    if (rc == TC_OK) rc = per_edge.alloc((size_t)std::max<int64_t>(g->num_cover, 1), cs);
    if (rc == TC_OK) rc = count_cover(g, per_edge.p, &total);
  } else {
    rc = per_edge.alloc((size_t)te, cs);
    if (rc == TC_OK) rc = count_plain(g, &total, per_edge.p);
  }
  if (rc == TC_OK) {
    launch(k_member_sums, std::min(np, sm_count() * 8), 256, 0, cs, dgraphs.p, dmem.p, dvb.p,
           deb.p, np, mode, g->hoff.p, (uint64_t)tn, (uint64_t)std::max<int64_t>(g->num_cover, 0),
           per_edge.p, dout.p);
    std::vector<unsigned long long> out(mem.size());
    cudaError_t e = cudaMemcpyAsync(out.data(), dout.p, sizeof(unsigned long long) * out.size(),
                                    cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "union sums", __FILE__, __LINE__);
    } else {
      for (size_t k = 0; k < mem.size(); ++k) cnt[idx[mem[k]]] = out[k];
    }
  }
  tc_graph_destroy(g);
  return rc;
}

}  // namespace tc

using namespace tc;

extern "C" int tc_count_batch(const tc_csr_view* graphs, int32_t ngraphs, int mode,
                              const tc_options* opt, void* cuda_stream, uint64_t* counts_out,
                              int* status_out) {
  if (ngraphs < 0 || (ngraphs > 0 && (!graphs || !counts_out)))
    return fail(TC_ERR_INVALID_ARG, "tc_count_batch: bad arguments");
  if (mode != TC_MODE_COVER && mode != TC_MODE_PLAIN)
    return fail(TC_ERR_INVALID_ARG, "tc_count_batch: unknown mode %d", mode);
  if (ngraphs == 0) return TC_OK;
  const int threads = opt && opt->block_threads > 0 ? opt->block_threads : 256;
  int per_sm = opt && opt->blocks_per_sm > 0 ? opt->blocks_per_sm : 4;
  if (threads != 128 && threads != 256 && threads != 512)
    return fail(TC_ERR_INVALID_ARG, "tc_count_batch: block_threads must be 128, 256 or 512");
  if (per_sm > 16) per_sm = 16;
  const int64_t skew = opt && opt->skew >= 2 ? opt->skew : kSkew;
  int64_t tiny_nnz = opt && opt->tiny_max_nnz > 0 ? opt->tiny_max_nnz : kBatchMaxNnz;
  if (tiny_nnz > (1ll << 22)) tiny_nnz = 1ll << 22;
  std::vector<int32_t> tiny, rest;
  for (int32_t i = 0; i < ngraphs; ++i) {
    const tc_csr_view& v = graphs[i];
    if (!v.offsets || v.nnz < 0 || (v.nnz > 0 && !v.cols))
      return fail(TC_ERR_INVALID_ARG, "tc_count_batch: graph %d has NULL arrays or nnz < 0", i);
    (v.n <= kBatchMaxN && v.nnz <= tiny_nnz ? tiny : rest).push_back(i);
  }
  std::vector<int> st((size_t)ngraphs, TC_OK);
  std::vector<unsigned long long> cnt((size_t)ngraphs, 0ull);
  cudaStream_t user = (cudaStream_t)cuda_stream;
  // internal stream at the caller's stream priority
  int prio = 0;
  if (cudaStreamGetPriority(user, &prio) != cudaSuccess) {
    cudaGetLastError();
    prio = 0;
  }
  cudaStream_t cs = nullptr;
  TC_CUDA(cudaStreamCreateWithPriority(&cs, cudaStreamNonBlocking, prio));
  int rc = TC_OK;
  if (!tiny.empty()) rc = run_tiny(graphs, tiny, mode, threads, per_sm, skew, cs, user, cnt, st);
  if (rc == TC_OK && !rest.empty()) rc = run_union(graphs, rest, mode, cs, cnt, st);
  cudaStreamSynchronize(cs);
  cudaStreamDestroy(cs);
  if (rc != TC_OK) return rc;
  for (int32_t i = 0; i < ngraphs; ++i) {
    counts_out[i] = cnt[i];
    if (status_out) status_out[i] = st[i];
  }
  return TC_OK;
}

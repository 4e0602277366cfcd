// Graph ingest (a0): copy the caller's CSR to the device, check it, list the
// chunks of its long rows, find the maximum-degree vertex; the COO row index
// of every entry is built when a path first needs it.
//
// Input format: a symmetric compressed-sparse-row graph, the input format of
// Sec. III of Bader et al., "Triangle Counting Through Cover-Edges".
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

namespace tc {

// ---------------------------------------------------------------- pinned slots
// Every graph owns a few pinned host words for device->host read-back.  They
// come from one pinned page pool so creating a graph does not pay a
// cudaMallocHost each time.
namespace {
std::mutex g_pin_mu;
std::vector<unsigned long long*> g_pin_free;
}  // namespace

static unsigned long long* pinned_acquire() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    void* page = nullptr;
    const size_t slot = kCtrlSlots * sizeof(unsigned long long);
    const size_t nslots = 64;
    if (cudaMallocHost(&page, slot * nslots) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (size_t i = 0; i < nslots; ++i)
      g_pin_free.push_back(reinterpret_cast<unsigned long long*>((char*)page + i * slot));
  }
  unsigned long long* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

static void pinned_release(unsigned long long* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

// ---------------------------------------------------------------- kernels
__global__ void k_check_offsets(const int64_t* __restrict__ off, uint32_t n, int64_t nnz,
                                unsigned long long* ctrl) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i <= (int64_t)n; i += stride) {
    bool bad = false;
    int64_t o = off[i];
    if (i == 0 && o != 0) bad = true;
    if (i == (int64_t)n && o != nnz) bad = true;
    if (o < 0 || o > nnz) bad = true;
    if (i < (int64_t)n && off[i + 1] < o) bad = true;
    if (bad) {
      atomicOr(&ctrl[kCtrlErr], kErrOffsets);
      atomicMin(&ctrl[kCtrlErrIdx], (unsigned long long)i);
    }
  }
}

// Rows with at most this many entries are checked (and given their COO row
// ids) by one lane.
constexpr int kTinyRowG = 8;

// A warp takes 32 consecutive rows: a lane checks its own row if it has at
// most kTinyRowG entries (all its loads issued at once), the rows up to
// kLongRow entries are then checked by the whole warp one at a time, and a
// row longer than kLongRow is listed as chunks (lchunks, each row's chunks
// contiguous) for k_rows_long.  Checks: column range always; when `strict`,
// no self-loops and strictly ascending rows.
__global__ void k_rows_and_check(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                                 uint32_t n, int strict, uint2* __restrict__ lchunks,
                                 unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long err = 0;
  for (int64_t gbase = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; gbase < (int64_t)n;
       gbase += gstride) {
    const int64_t x = gbase + lane;
    int64_t b = 0, e = 0;
    if (x < (int64_t)n) {
      b = off[x];
      e = off[x + 1];
    }
    const int64_t d = e - b;
    if (x < (int64_t)n && d <= kTinyRowG) {
      uint32_t w[kTinyRowG];
#pragma unroll
      for (int k = 0; k < kTinyRowG; ++k) w[k] = k < d ? cols[b + k] : 0u;
#pragma unroll
      for (int k = 0; k < kTinyRowG; ++k) {
        if (k >= d) break;
        if (w[k] >= n) err |= kErrColRange;
        if (strict) {
          if (w[k] == (uint32_t)x) err |= kErrSelfLoop;
          if (k > 0 && w[k - 1] >= w[k]) err |= kErrUnsorted;
        }
      }
    } else if (x < (int64_t)n && d > kLongRow) {
      const uint32_t nch = (uint32_t)((d + kChunk - 1) / kChunk);
      const unsigned long long c0 = atomicAdd(&ctrl[kCtrlLong], (unsigned long long)nch);
      for (uint32_t k = 0; k < nch; ++k) lchunks[c0 + k] = make_uint2((uint32_t)x, k);
    }
    unsigned rows = __ballot_sync(0xFFFFFFFFu, x < (int64_t)n && d > kTinyRowG && d <= kLongRow);
    while (rows) {
      const int r = __ffs(rows) - 1;
      rows &= rows - 1;
      const uint32_t u = (uint32_t)(gbase + r);
      const int64_t rb = __shfl_sync(0xFFFFFFFFu, b, r), re = __shfl_sync(0xFFFFFFFFu, e, r);
      for (int64_t i = rb + lane; i < re; i += 32) {
        const uint32_t v = cols[i];
        if (v >= n) err |= kErrColRange;
        if (strict) {
          if (v == u) err |= kErrSelfLoop;
          if (i > rb && cols[i - 1] >= v) err |= kErrUnsorted;
        }
      }
    }
  }
  if (err) atomicOr(&ctrl[kCtrlErr], err);
}

// CTA per chunk of a long row: the same checks as k_rows_and_check.
__global__ void __launch_bounds__(kChunk)
k_rows_long(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols, uint32_t n,
            int strict, const uint2* __restrict__ lchunks, unsigned long long* ctrl) {
  const unsigned long long nch = ctrl[kCtrlLong];
  unsigned long long err = 0;
  for (unsigned long long c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const uint32_t u = ch.x;
    const int64_t b = off[u], e = off[u + 1];
    const int64_t i = b + (int64_t)ch.y * kChunk + threadIdx.x;
    if (i < e) {
      const uint32_t v = cols[i];
      if (v >= n) err |= kErrColRange;
      if (strict) {
        if (v == u) err |= kErrSelfLoop;
        if (i > b && cols[i - 1] >= v) err |= kErrUnsorted;
      }
    }
  }
  if (err) atomicOr(&ctrl[kCtrlErr], err);
}

// COO row ids: erow[i] = u for every entry i of row u, in the same row
// classes (a lane for tiny rows, the warp for rows up to kLongRow, a CTA per
// chunk of the longer rows).
__global__ void k_erow_rows(const int64_t* __restrict__ off, uint32_t n, uint32_t* __restrict__ erow) {
  const int lane = threadIdx.x & 31;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t gbase = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; gbase < (int64_t)n;
       gbase += gstride) {
    const int64_t x = gbase + lane;
    int64_t b = 0, e = 0;
    if (x < (int64_t)n) {
      b = off[x];
      e = off[x + 1];
    }
    const int64_t d = e - b;
    if (x < (int64_t)n && d <= kTinyRowG)
      for (int64_t i = b; i < e; ++i) erow[i] = (uint32_t)x;
    unsigned rows = __ballot_sync(0xFFFFFFFFu, x < (int64_t)n && d > kTinyRowG && d <= kLongRow);
    while (rows) {
      const int r = __ffs(rows) - 1;
      rows &= rows - 1;
      const int64_t rb = __shfl_sync(0xFFFFFFFFu, b, r), re = __shfl_sync(0xFFFFFFFFu, e, r);
      for (int64_t i = rb + lane; i < re; i += 32) erow[i] = (uint32_t)(gbase + r);
    }
  }
}

__global__ void __launch_bounds__(kChunk)
k_erow_long(const int64_t* __restrict__ off, const uint2* __restrict__ lchunks, int64_t nch,
            uint32_t* __restrict__ erow) {
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const uint2 ch = lchunks[c];
    const int64_t i = off[ch.x] + (int64_t)ch.y * kChunk + threadIdx.x;
    if (i < off[ch.x + 1]) erow[i] = ch.x;
  }
}

// Thread per entry: (u, v) must have (v, u); binary search of u in N(v).
__global__ void k_check_symmetric(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                                  const uint32_t* __restrict__ erow, int64_t nnz,
                                  unsigned long long* ctrl) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < nnz; i += stride) {
    uint32_t u = erow[i], v = cols[i];
    int64_t lo = off[v], hi = off[v + 1];
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (cols[mid] < u) lo = mid + 1; else hi = mid;
    }
    if (!(lo < off[v + 1] && cols[lo] == u)) {
      atomicOr(&ctrl[kCtrlErr], kErrAsym);
      atomicMin(&ctrl[kCtrlErrIdx], (unsigned long long)i);
    }
  }
}

// key = degree << 32 | (0xFFFFFFFF - v): the max key is the max degree with
// the lowest id among ties.
__global__ void k_argmax_degree(const int64_t* __restrict__ off, uint32_t n,
                                unsigned long long* ctrl) {
  unsigned long long best = 0;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride) {
    unsigned long long d = (unsigned long long)(off[i + 1] - off[i]);
    unsigned long long key = (d << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
    best = best > key ? best : key;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_down_sync(0xFFFFFFFFu, best, o);
    best = best > other ? best : other;
  }
  __shared__ unsigned long long s[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s[wid] = best;
  __syncthreads();
  if (wid == 0) {
    best = lane < (int)(blockDim.x >> 5) ? s[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long other = __shfl_down_sync(0xFFFFFFFFu, best, o);
      best = best > other ? best : other;
    }
    if (lane == 0) atomicMax(&ctrl[kCtrlMax], best);
  }
}

__global__ void k_ctrl_reset(unsigned long long* ctrl) {
  int i = threadIdx.x;
  if (i < kCtrlSlots) ctrl[i] = (i == kCtrlErrIdx) ? ~0ull : 0ull;
}

// ---------------------------------------------------------------- stages
static int read_ctrl(tc_graph* g) {
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, g->stream));
  TC_CUDA(cudaStreamSynchronize(g->stream));
  return TC_OK;
}

static int describe_err(tc_graph* g, unsigned long long err) {
  unsigned long long idx = g->ctrl_host[kCtrlErrIdx];
  if (err & kErrOffsets)
    return fail(TC_ERR_INVALID_GRAPH, "offsets invalid (first bad index %llu)", idx);
  if (err & kErrColRange) return fail(TC_ERR_INVALID_GRAPH, "a column index is >= n");
  if (err & kErrSelfLoop) return fail(TC_ERR_INVALID_GRAPH, "self-loop in CSR");
  if (err & kErrUnsorted)
    return fail(TC_ERR_INVALID_GRAPH, "a row is not strictly ascending (unsorted or duplicate)");
  if (err & kErrAsym) return fail(TC_ERR_INVALID_GRAPH, "CSR not symmetric (entry %llu)", idx);
  return fail(TC_ERR_INVALID_GRAPH, "graph check failed (0x%llx)", err);
}

// The COO row ids are built on first use (the plain path, the symmetry
// check, explicit BFS roots); the cover path with the default roots never
// reads them.  Needs g->nlchunks.
int ensure_erow(tc_graph* g) {
  if (g->erow.p || g->nnz == 0) return TC_OK;
  TC_TRY(g->erow.alloc((size_t)g->nnz, g->stream));
  launch(k_erow_rows, grid_for((int64_t)g->n * 32, 256, 16), 256, 0, g->stream, g->off, g->n,
         g->erow.p);
  if (g->nlchunks > 0)
    launch(k_erow_long, (int)std::min<int64_t>(g->nlchunks, (int64_t)sm_count() * 8), kChunk, 0,
           g->stream, g->off, g->lchunks.p, g->nlchunks, g->erow.p);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

int graph_ingest_checks(tc_graph* g, uint32_t flags) {
  const int T = 256;
  launch(k_ctrl_reset, 1, 32, 0, g->stream, g->ctrl.p);
  launch(k_check_offsets, grid_for((int64_t)g->n + 1, T), T, 0, g->stream, g->off, g->n, g->nnz,
                                                                         g->ctrl.p);
  TC_CUDA(cudaGetLastError());
  TC_TRY(read_ctrl(g));
  if (g->ctrl_host[kCtrlErr]) return describe_err(g, g->ctrl_host[kCtrlErr]);

  // at most nnz / kChunk full chunks plus one partial chunk per long row
  TC_TRY(g->lchunks.alloc((size_t)(g->nnz / kChunk + g->nnz / kLongRow + 1), g->stream));
  if (g->n > 0) {
    const int strict = (flags & TC_GRAPH_VALIDATE) ? 1 : 0;
    launch(k_rows_and_check, grid_for((int64_t)g->n * 32, T, 16), T, 0, g->stream, g->off, g->cols,
           g->n, strict, g->lchunks.p, g->ctrl.p);
    launch(k_rows_long, sm_count() * 2, kChunk, 0, g->stream, g->off, g->cols, g->n, strict,
           g->lchunks.p, g->ctrl.p);
    TC_CUDA(cudaGetLastError());
  }
  if ((flags & TC_GRAPH_CHECK_SYM) && g->nnz > 0) {
    // symmetry search reads cols[] of other rows: only safe once columns
    // are known to be in range, so check that first.
    TC_TRY(read_ctrl(g));
    if (g->ctrl_host[kCtrlErr]) return describe_err(g, g->ctrl_host[kCtrlErr]);
    g->nlchunks = (int64_t)g->ctrl_host[kCtrlLong];
    TC_TRY(ensure_erow(g));
    launch(k_check_symmetric, grid_for(g->nnz, T), T, 0, g->stream, g->off, g->cols, g->erow.p,
                                                                  g->nnz, g->ctrl.p);
    TC_CUDA(cudaGetLastError());
  }
  launch(k_argmax_degree, grid_for(g->n, T), T, 0, g->stream, g->off, g->n, g->ctrl.p);
  TC_CUDA(cudaGetLastError());
  TC_TRY(read_ctrl(g));
  if (g->ctrl_host[kCtrlErr]) return describe_err(g, g->ctrl_host[kCtrlErr]);
  g->nlchunks = (int64_t)g->ctrl_host[kCtrlLong];
  unsigned long long key = g->ctrl_host[kCtrlMax];
  g->max_degree = (uint32_t)(key >> 32);
  g->r0 = g->n > 0 ? 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull) : 0;
  return TC_OK;
}

void graph_drop_cache(tc_graph* g) {
  g->levels.release();
  g->nlevels = -1;
  g->nroots = 0;
  g->cover.release();
  g->hoff.release();
  g->num_cover = -1;
  g->seg_valid = false;
  g->scols.release();
  g->seg.release();
}

}  // namespace tc

using namespace tc;

extern "C" {

int tc_graph_create(const tc_csr_view* csr, uint32_t flags, void* cuda_stream, tc_graph** out) {
  if (!csr || !out) return fail(TC_ERR_INVALID_ARG, "tc_graph_create: NULL csr or out");
  if (csr->nnz < 0) return fail(TC_ERR_INVALID_ARG, "tc_graph_create: nnz < 0");
  if (!csr->offsets) return fail(TC_ERR_INVALID_ARG, "tc_graph_create: NULL offsets");
  if (csr->nnz > 0 && !csr->cols) return fail(TC_ERR_INVALID_ARG, "tc_graph_create: NULL cols");
  if ((flags & TC_GRAPH_BORROW) &&
      !(csr->on_device && is_device_ptr(csr->offsets) && (csr->nnz == 0 || is_device_ptr(csr->cols))))
    return fail(TC_ERR_INVALID_ARG, "tc_graph_create: TC_GRAPH_BORROW needs device pointers");
  if (csr->n == 0xFFFFFFFFu)
    return fail(TC_ERR_INVALID_ARG, "tc_graph_create: n must be < 2^32 - 1");

  tc_graph* g = new (std::nothrow) tc_graph();
  if (!g) return fail(TC_ERR_OOM, "host allocation failed");
  cudaGetDevice(&g->device);
  g->stream = (cudaStream_t)cuda_stream;
  g->n = csr->n;
  g->nnz = csr->nnz;
  int st = TC_OK;
  do {
    g->ctrl_host = pinned_acquire();
    if (!g->ctrl_host) { st = fail(TC_ERR_OOM, "pinned host allocation failed"); break; }
    if ((st = g->ctrl.alloc(kCtrlSlots, g->stream)) != TC_OK) break;
    if (flags & TC_GRAPH_BORROW) {
      g->off = csr->offsets;
      g->cols = csr->cols;
    } else {
      if ((st = g->off_own.alloc((size_t)g->n + 1, g->stream)) != TC_OK) break;
      if ((st = g->cols_own.alloc((size_t)g->nnz, g->stream)) != TC_OK) break;
      // cudaMemcpyDefault lets unified addressing classify the source, so a
      // view whose on_device flag is wrong still copies correctly.
      cudaMemcpyKind kind = cudaMemcpyDefault;
      cudaError_t e = cudaMemcpyAsync(g->off_own.p, csr->offsets, sizeof(int64_t) * ((size_t)g->n + 1),
                                      kind, g->stream);
      if (e == cudaSuccess && g->nnz > 0)
        e = cudaMemcpyAsync(g->cols_own.p, csr->cols, sizeof(uint32_t) * (size_t)g->nnz, kind,
                            g->stream);
      if (e != cudaSuccess) { st = cuda_fail(e, "CSR copy", __FILE__, __LINE__); break; }
      g->off = g->off_own.p;
      g->cols = g->cols_own.p;
    }
    for (int i = 0; i < 8 && st == TC_OK; ++i) {
      cudaError_t e = cudaEventCreate(&g->ev[i]);
      if (e != cudaSuccess) st = cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__);
    }
    if (st != TC_OK) break;
    cudaEventRecord(g->ev[0], g->stream);
    st = graph_ingest_checks(g, flags);
    cudaEventRecord(g->ev[1], g->stream);
  } while (0);
  if (st != TC_OK) {
    tc_graph_destroy(g);
    return st;
  }
  cudaEventSynchronize(g->ev[1]);
  cudaEventElapsedTime(&g->stats.ms_validate, g->ev[0], g->ev[1]);
  *out = g;
  return TC_OK;
}

int tc_graph_destroy(tc_graph* g) {
  if (!g) return TC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  cudaStreamSynchronize(g->stream);
  graph_drop_cache(g);
  g->erow.release();
  g->lchunks.release();
  g->cols_own.release();
  g->off_own.release();
  g->ctrl.release();
  cudaStreamSynchronize(g->stream);
  for (int i = 0; i < 8; ++i)
    if (g->ev[i]) cudaEventDestroy(g->ev[i]);
  pinned_release(g->ctrl_host);
  if (prev != g->device) cudaSetDevice(prev);
  cudaGetLastError();
  delete g;
  return TC_OK;
}

int tc_graph_invalidate(tc_graph* g) {
  if (!g) return fail(TC_ERR_INVALID_ARG, "tc_graph_invalidate: NULL graph");
  std::lock_guard<std::mutex> lk(g->mu);
  graph_drop_cache(g);
  return TC_OK;
}

int tc_graph_info(const tc_graph* g, tc_graph_info_t* info) {
  if (!g || !info) return fail(TC_ERR_INVALID_ARG, "tc_graph_info: NULL argument");
  std::lock_guard<std::mutex> lk(g->mu);
  info->n = g->n;
  info->nnz = g->nnz;
  info->num_edges = g->nnz / 2;
  info->max_degree = g->max_degree;
  info->nlevels = g->nlevels;
  info->num_cover = g->num_cover;
  info->num_roots = g->nroots;
  return TC_OK;
}

int tc_graph_stats(const tc_graph* g, tc_stats_t* out) {
  if (!g || !out) return fail(TC_ERR_INVALID_ARG, "tc_graph_stats: NULL argument");
  std::lock_guard<std::mutex> lk(g->mu);
  *out = g->stats;
  return TC_OK;
}

}  // extern "C"

// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/tc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstddef>
#include <mutex>
#include <utility>

#include "tc.h"

namespace tc {

constexpr uint32_t kUnvisited = 0xFFFFFFFFu;
constexpr int kWarp = 32;

// Rows with more than kLongRow entries are not given to one warp: at ingest
// they are cut into chunks of kChunk consecutive entries, listed in
// tc_graph::lchunks as {row, chunk number within the row}; the chunks of a
// row are contiguous in the list, so chunk c of row u sits at index
// (index of u's first chunk) + c.  Kernels over rows skip long rows and
// take their chunks with one CTA per chunk instead.
constexpr int64_t kLongRow = 1024;
constexpr int kChunk = 1024;

// ---------------------------------------------------------------- errors
// Record a message for tc_last_error() and return `status`.
int fail(int status, const char* fmt, ...);
// Map a CUDA error to TC_ERR_CUDA / TC_ERR_OOM with a message.
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define TC_CUDA(call)                                                       \
  do {                                                                      \
    cudaError_t _e = (call);                                                \
    if (_e != cudaSuccess) return ::tc::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define TC_TRY(expr)              \
  do {                            \
    int _s = (expr);              \
    if (_s != TC_OK) return _s;   \
  } while (0)

// ---------------------------------------------------------------- launches
extern std::atomic<unsigned long long> g_kernel_launches;

// k<<<grid, block, smem, stream>>>(args...) plus the process-wide launch count.
template <typename... KArgs, typename... Args>
inline void launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args&&... args) {
  k<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
}

// ---------------------------------------------------------------- memory
// Device allocation through the user hook (tc_set_allocator) or
// cudaMallocAsync on `stream`.  Returns TC_OK / TC_ERR_OOM.
int dev_alloc(void** p, size_t bytes, cudaStream_t stream);
void dev_free(void* p, cudaStream_t stream);

template <class T>
int dev_alloc_n(T** p, size_t count, cudaStream_t stream) {
  return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T), stream);
}

// RAII owner of one device buffer.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    return dev_alloc_n(&p, count > 0 ? count : 1, stream);
  }
  // grow-only
  int reserve(size_t count, cudaStream_t stream) {
    if (p && n >= count) return TC_OK;
    return alloc(count, stream);
  }
  void release() {
    if (p) dev_free(p, s);
    p = nullptr;
    n = 0;
  }
};

// True if `p` is device (or managed) memory visible to the current device.
bool is_device_ptr(const void* p);

// Copy `bytes` from device memory `src` to `dst` (host or device), on stream.
cudaError_t copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s);

// Number of SMs of the current device (cached per device).
int sm_count();

}  // namespace tc

// The opaque graph object.
struct tc_graph {
  // held by every entry point that takes the graph (except destroy), so
  // calls on one graph from several host threads run one after another
  mutable std::mutex mu;
  int device = 0;
  cudaStream_t stream = nullptr;
  uint32_t n = 0;
  int64_t nnz = 0;
  uint32_t max_degree = 0;
  uint32_t r0 = 0;  // max-degree vertex (lowest id on ties)

  // CSR (owned unless borrowed)
  const int64_t* off = nullptr;
  const uint32_t* cols = nullptr;
  tc::DevBuf<int64_t> off_own;
  tc::DevBuf<uint32_t> cols_own;
  tc::DevBuf<uint32_t> erow;  // row id of every CSR entry (COO rows), built on first use
  tc::DevBuf<uint2> lchunks;  // chunks of the rows longer than kLongRow
  int64_t nlchunks = 0;

  // cached BFS levels
  tc::DevBuf<uint32_t> levels;
  int64_t nlevels = -1;
  uint32_t nroots = 0;

  // cached level-segmented adjacency (see segment.cu)
  tc::DevBuf<uint32_t> scols;
  tc::DevBuf<uint4> seg;
  bool seg_valid = false;

  // cached cover-edge set H as (u, v) pairs in CSR order
  tc::DevBuf<uint2> cover;
  tc::DevBuf<unsigned long long> hoff;  // index in H of each vertex's first cover edge
  int64_t num_cover = -1;

  // small control block on device + pinned host mirror
  tc::DevBuf<unsigned long long> ctrl;
  unsigned long long* ctrl_host = nullptr;

  // events for stage timing: 0-3 stage boundaries, 4-5 around the
  // intersection kernel alone
  cudaEvent_t ev[8] = {};
  tc_stats_t stats{};
};

namespace tc {

// Control-block slots (unsigned long long each).
enum CtrlSlot {
  kCtrlCount = 0,     // triangle count accumulator
  kCtrlErr = 1,       // device-side error bits
  kCtrlErrIdx = 2,    // first offending index
  kCtrlQ0 = 3,        // BFS: next-frontier size
  kCtrlQ1 = 4,        // BFS: next-frontier edge sum
  kCtrlMax = 5,       // argmax key
  kCtrlElems = 6,     // list elements handed to the intersection
  kCtrlTmp = 7,
  kCtrlWork = 8,      // dynamic work counter of the intersection kernels
  kCtrlItems = 9,     // work items per table class (two slots: 9, 10)
  kCtrlLong = 11,     // chunks of long rows (ingest)
  kCtrlWorkSum = 12,  // lookups of all hashed edges (bucketing)
  kCtrlSlots = 16
};

// Device error bits
enum : unsigned long long {
  kErrOffsets = 1ull,     // offsets not monotone / wrong ends
  kErrColRange = 2ull,    // column >= n
  kErrSelfLoop = 4ull,
  kErrUnsorted = 8ull,    // row not strictly ascending (or duplicate)
  kErrAsym = 16ull,       // (u,v) without (v,u)
  kErrTimeout = 32ull
};

// stage functions (each returns TC_OK or an error)
int ensure_erow(tc_graph* g);  // COO row ids (graph.cu), built on first use
int compute_levels(tc_graph* g, const uint32_t* roots_host, uint32_t nroots);
int compute_segments(tc_graph* g);
int compute_cover(tc_graph* g);
// Counts over the edge range [first, last) of the mode's index space (cover:
// H in its canonical order; plain: CSR entries, those with u > v adding
// nothing); last < 0 means to the end.  Per-edge outputs are indexed by the
// global edge index.
// merge_only: the warp merge / binary-search kernels of intersect.cu
// instead of the hash intersection (a comparison arm).
int count_cover(tc_graph* g, uint32_t* per_edge_out, uint64_t* total, int64_t first = 0,
                int64_t last = -1, bool merge_only = false);
int count_plain(tc_graph* g, uint64_t* total, uint32_t* per_entry = nullptr, int64_t first = 0,
                int64_t last = -1, bool merge_only = false);

// Hash intersection (hashsect.cu) over edges [first, last) of the mode's
// index space; per_edge (per-edge counts) and tv (cover mode: per-vertex
// counts) may be NULL.  Needs |edges| < 2^32 and nnz < 2^32.
int hash_count(tc_graph* g, int mode, const int64_t* ustart, uint32_t* per_edge, int64_t first,
               int64_t last, unsigned long long* tv = nullptr);

// Triangle finding (find.cu): per-vertex counts into tv_dev (n entries,
// device), and the list of triangles (u, v, w) into out_dev (3 * cap
// entries, device; *found = the number of triangles, which may exceed cap).
int find_vertex_counts(tc_graph* g, unsigned long long* tv_dev);
int find_list(tc_graph* g, uint32_t* out_dev, unsigned long long cap, uint64_t* found);
// The same per-vertex counts for the cover edges whose H indices are
// list[0 .. *nlist_dev) (device length, at most nlist_max).
int find_vertex_list(tc_graph* g, const uint32_t* list, const unsigned long long* nlist_dev,
                     uint64_t nlist_max, unsigned long long* tv_dev);

// Work-balanced shard bounds of the mode's edge index space (shard.cu):
// bounds_host[0] = 0 <= ... <= bounds_host[P] = |edges|.
int shard_bounds(tc_graph* g, int mode, int32_t P, int64_t* bounds_host);

// Exclusive scan of `n` 64-bit counts in place on `stream`; returns the
// total through `total_dev` (device pointer, may be null).
int exclusive_scan_u64(unsigned long long* data, int64_t n, unsigned long long* total_dev,
                       cudaStream_t stream);

// launch helpers
inline int grid_for(int64_t work, int threads, int per_sm = 8) {
  int64_t blocks = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace tc

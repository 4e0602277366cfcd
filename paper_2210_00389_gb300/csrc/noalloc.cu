// tc_count_plain_static: the plain all-edge triangle count of a device CSR
// without allocating any device memory.
//
// Some callers cannot call cudaMalloc / cudaFree at the point where they
// need a count: cudaMalloc and cudaFree can synchronize the device, which a
// latency-bound loop overlapping work on several streams must avoid;
// applications whose device memory is entirely owned by another allocator
// (a framework's caching allocator, a fixed arena budgeted up front) may not
// take memory behind that allocator's back; deployments that allocate once at
// start-up forbid allocation afterwards.  This entry point serves them: its
// scratch is one file-scope static device array, g_static_scratch, that every
// GPU which loads the library holds until the process exits.
//
// The kernel is a variant of the plain intersection kernel of intersect.cu
// (warp per CSR entry u < v, counting common neighbours above v with the
// shared warp merge); instead of the allocated COO rows and upper-start
// array it finds each work chunk's row by bisection of the offsets and keeps
// the upper starts, the work counter and the count accumulator in the static
// array.
#include <mutex>

#include "internal.cuh"
#include "warp_isect.cuh"

namespace tc {

// Largest vertex count accepted; the scratch holds one uint32 per vertex.
constexpr uint32_t kStaticMaxVertices = 1u << 22;
constexpr size_t kStaticHeaderBytes = 256;  // work counter, accumulator
constexpr size_t kStaticScratchBytes =
    kStaticHeaderBytes + sizeof(uint32_t) * (size_t)kStaticMaxVertices;  // 16 MiB + 256 B
constexpr int kStaticThreads = 256;
constexpr int kStaticChunk = 64;  // CSR entries per work grab

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Host side: the array's name is only a host stand-in, so each device's real
// address is looked up once, with that device current, and cached.
static std::mutex g_static_mu;
static void* g_static_addr[64] = {};

static int static_scratch_address(void** out) {
  int dev = 0;
  TC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(TC_ERR_CUDA, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return TC_OK;
}

// ustart_rel[v] = position within N(v) of the first neighbour greater than v.
__global__ void k_static_upper_start(const int64_t* __restrict__ off,
                                     const uint32_t* __restrict__ cols, uint32_t n,
                                     uint32_t* __restrict__ ustart_rel) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; v < (int64_t)n; v += stride) {
    const int64_t b = off[v];
    int64_t lo = b, hi = off[v + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cols[mid] <= (uint32_t)v) lo = mid + 1; else hi = mid;
    }
    ustart_rel[v] = (uint32_t)(lo - b);
  }
}

// Warp per CSR entry (u, v) with u < v: |N(u) ∩ (v,inf) ∩ N(v) ∩ (v,inf)|.
// Chunks of entries come from *work; the chunk's first row is found by
// bisection of the offsets and then advanced entry by entry.  Entries with
// a column id >= n are skipped.
__global__ void __launch_bounds__(kStaticThreads)
k_static_plain(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols, uint32_t n,
               int64_t nnz, const uint32_t* __restrict__ ustart_rel, unsigned long long* work,
               unsigned long long* acc_out) {
  const int lane = threadIdx.x & 31;
  unsigned long long acc = 0;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)kStaticChunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if ((int64_t)base >= nnz) break;
    const int64_t end = min((int64_t)base + kStaticChunk, nnz);
    // row of entry `base`: last u with off[u] <= base
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (off[mid] <= (int64_t)base) lo = mid; else hi = mid;
    }
    uint32_t u = (uint32_t)lo;
    for (int64_t e = (int64_t)base; e < end; ++e) {
      while (off[u + 1] <= e) ++u;
      const uint32_t v = cols[e];
      if (v >= n || u >= v) continue;
      const int64_t au = e + 1, bv = off[v] + ustart_rel[v];
      acc += warp_intersect(cols + au, off[u + 1] - au, cols + bv, off[v + 1] - bv);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if (lane == 0 && acc) atomicAdd(acc_out, acc);
}

__global__ void k_static_store(const unsigned long long* acc, uint64_t* out) { *out = *acc; }

}  // namespace tc

using namespace tc;

extern "C" int tc_count_plain_static(const int64_t* offsets, const uint32_t* cols, uint32_t n,
                                     int64_t nnz, uint64_t* count_out, void* cuda_stream) {
  if (n > kStaticMaxVertices)
    return fail(TC_ERR_CAPACITY,
                "tc_count_plain_static: n = %u exceeds the static scratch limit of %u vertices",
                n, kStaticMaxVertices);
  if (!offsets || !count_out || nnz < 0 || (nnz > 0 && !cols))
    return fail(TC_ERR_INVALID_ARG, "tc_count_plain_static: NULL pointer or nnz < 0");
  if (!is_device_ptr(offsets) || !is_device_ptr(count_out) || (nnz > 0 && !is_device_ptr(cols)))
    return fail(TC_ERR_INVALID_ARG, "tc_count_plain_static: offsets, cols and count_out must be "
                                    "device memory");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  TC_TRY(static_scratch_address(&base));
  unsigned long long* work = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* acc = work + 1;
  uint32_t* ustart_rel =
      reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(base) + kStaticHeaderBytes);
  // the array keeps the previous call's contents: clear the two counters
  TC_CUDA(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), s));
  if (n > 0 && nnz > 0) {
    launch(k_static_upper_start, grid_for(n, kStaticThreads), kStaticThreads, 0, s, offsets, cols, n,
           ustart_rel);
    launch(k_static_plain, grid_for(nnz * 32, kStaticThreads, 8), kStaticThreads, 0, s, offsets,
           cols, n, nnz, ustart_rel, work, acc);
  }
  launch(k_static_store, 1, 1, 0, s, acc, count_out);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

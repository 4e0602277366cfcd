// Device-wide exclusive prefix sum of 64-bit counts (reduce-then-scan).
// Used for frontier degree offsets (BFS) and per-tile cover-edge counts.
#include "internal.cuh"

namespace tc {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v,
                                                                   unsigned long long* total) {
  __shared__ unsigned long long warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < kScanThreads / 32 ? warp_sums[lane] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  unsigned long long warp_prefix = wid > 0 ? warp_sums[wid - 1] : 0ull;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(unsigned long long* data, int64_t n, unsigned long long* tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  unsigned long long items[kScanItems];
  unsigned long long sum = 0;
  // each thread takes kScanItems consecutive elements
  const int64_t first = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = first + k;
    items[k] = i < n ? data[i] : 0ull;
    sum += items[k];
  }
  unsigned long long total;
  unsigned long long run = block_exclusive_scan(sum, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = first + k;
    unsigned long long x = items[k];
    if (i < n) data[i] = run;
    run += x;
  }
  if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(unsigned long long* data, int64_t n, const unsigned long long* tile_prefix) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  unsigned long long add = tile_prefix[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) data[i] += add;
  }
}

__global__ void k_store_total(const unsigned long long* data, int64_t n, const unsigned long long* last,
                              unsigned long long* total) {
  // total = exclusive[n-1] + original[n-1]; `last` holds original[n-1]
  *total = (n > 0 ? data[n - 1] + *last : 0ull);
}

__global__ void k_copy_last(const unsigned long long* data, int64_t n, unsigned long long* out) {
  *out = n > 0 ? data[n - 1] : 0ull;
}

int exclusive_scan_u64(unsigned long long* data, int64_t n, unsigned long long* total_dev,
                       cudaStream_t stream) {
  if (n <= 0) {
    if (total_dev) TC_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), stream));
    return TC_OK;
  }
  DevBuf<unsigned long long> last;
  if (total_dev) {
    TC_TRY(last.alloc(1, stream));
    launch(k_copy_last, 1, 1, 0, stream, data, n, last.p);
  }
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    launch(k_scan_tiles, 1, kScanThreads, 0, stream, data, n, nullptr);
  } else {
    DevBuf<unsigned long long> sums;
    TC_TRY(sums.alloc((size_t)tiles, stream));
    launch(k_scan_tiles, (unsigned)tiles, kScanThreads, 0, stream, data, n, sums.p);
    TC_TRY(exclusive_scan_u64(sums.p, tiles, nullptr, stream));
    launch(k_scan_add, (unsigned)tiles, kScanThreads, 0, stream, data, n, sums.p);
  }
  if (total_dev) launch(k_store_total, 1, 1, 0, stream, data, n, last.p, total_dev);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

}  // namespace tc

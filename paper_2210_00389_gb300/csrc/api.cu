// C ABI entry points for levels, cover edges and counts (include/tc.h).
#include <cstring>

#include "internal.cuh"

namespace tc {

// Makes the graph's device current for the scope of a call.
struct DeviceGuard {
  int prev = -1, want;
  explicit DeviceGuard(int dev) : want(dev) {
    cudaGetDevice(&prev);
    if (prev != want) cudaSetDevice(want);
  }
  ~DeviceGuard() {
    if (prev >= 0 && prev != want) cudaSetDevice(prev);
  }
};

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    ms = 0.f;
  }
  return ms;
}

}  // namespace tc

using namespace tc;

extern "C" {

int tc_bfs_levels(tc_graph* g, const uint32_t* roots, uint32_t nroots, uint32_t* levels_out,
                  uint32_t* nlevels_out) {
  if (!g) return fail(TC_ERR_INVALID_ARG, "tc_bfs_levels: NULL graph");
  if (roots && nroots == 0) roots = nullptr;
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  cudaEventRecord(g->ev[0], g->stream);
  TC_TRY(compute_levels(g, roots, nroots));
  cudaEventRecord(g->ev[1], g->stream);
  if (levels_out && g->n > 0) {
    TC_CUDA(copy_out(levels_out, g->levels.p, sizeof(uint32_t) * g->n, g->stream));
  }
  TC_CUDA(cudaStreamSynchronize(g->stream));
  g->stats.ms_bfs = elapsed(g->ev[0], g->ev[1]);
  if (nlevels_out) *nlevels_out = (uint32_t)g->nlevels;
  return TC_OK;
}

int tc_cover_edges(tc_graph* g, uint32_t* uv_out, int64_t cap, int64_t* count_out) {
  if (!g || !count_out) return fail(TC_ERR_INVALID_ARG, "tc_cover_edges: NULL argument");
  if (uv_out && cap < 0) return fail(TC_ERR_INVALID_ARG, "tc_cover_edges: cap < 0");
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  cudaEventRecord(g->ev[0], g->stream);
  if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  cudaEventRecord(g->ev[1], g->stream);
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  cudaEventRecord(g->ev[2], g->stream);
  *count_out = g->num_cover;
  if (uv_out) {
    if (g->num_cover > cap) {
      TC_CUDA(cudaStreamSynchronize(g->stream));
      return fail(TC_ERR_CAPACITY, "tc_cover_edges: |H| = %lld > cap = %lld",
                  (long long)g->num_cover, (long long)cap);
    }
    TC_CUDA(copy_out(uv_out, g->cover.p, sizeof(uint2) * (size_t)g->num_cover, g->stream));
  }
  TC_CUDA(cudaStreamSynchronize(g->stream));
  g->stats.ms_bfs = elapsed(g->ev[0], g->ev[1]);
  g->stats.ms_cover = elapsed(g->ev[1], g->ev[2]);
  return TC_OK;
}

int tc_count(tc_graph* g, int mode, uint64_t* count_out) {
  if (!g || !count_out) return fail(TC_ERR_INVALID_ARG, "tc_count: NULL argument");
  const bool merge_only = (mode & TC_INTERSECT_MERGE) != 0;
  mode &= ~TC_INTERSECT_MERGE;
  if (mode != TC_MODE_COVER && mode != TC_MODE_PLAIN)
    return fail(TC_ERR_INVALID_ARG, "tc_count: unknown mode %d", mode);
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  tc_stats_t& st = g->stats;
  st.ms_bfs = st.ms_cover = st.ms_bucket = st.ms_intersect = st.ms_total = 0.f;
  const unsigned long long launches0 = g_kernel_launches.load();
  uint64_t T = 0;
  cudaEventRecord(g->ev[0], g->stream);
  if (mode == TC_MODE_COVER) {
    if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
    cudaEventRecord(g->ev[1], g->stream);
    if (g->num_cover < 0) TC_TRY(compute_cover(g));
    cudaEventRecord(g->ev[2], g->stream);
    TC_TRY(count_cover(g, nullptr, &T, 0, -1, merge_only));
    cudaEventRecord(g->ev[3], g->stream);
    cudaEventSynchronize(g->ev[3]);
    st.ms_bfs = elapsed(g->ev[0], g->ev[1]);
    st.ms_cover = elapsed(g->ev[1], g->ev[2]);
    st.ms_total = elapsed(g->ev[0], g->ev[3]);
  } else {
    cudaEventRecord(g->ev[1], g->stream);
    TC_TRY(count_plain(g, &T, nullptr, 0, -1, merge_only));
    cudaEventRecord(g->ev[3], g->stream);
    cudaEventSynchronize(g->ev[3]);
    st.ms_total = elapsed(g->ev[0], g->ev[3]);
  }
  st.kernel_launches = (uint32_t)(g_kernel_launches.load() - launches0);
  *count_out = T;
  return TC_OK;
}

int tc_vertex_counts(tc_graph* g, uint64_t* counts_out) {
  if (!g || (!counts_out && g->n > 0))
    return fail(TC_ERR_INVALID_ARG, "tc_vertex_counts: NULL argument");
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  if (g->n == 0) return TC_OK;
  if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  DevBuf<unsigned long long> tv;
  TC_TRY(tv.alloc(g->n, g->stream));
  TC_TRY(find_vertex_counts(g, tv.p));
  TC_CUDA(copy_out(counts_out, tv.p, sizeof(uint64_t) * g->n, g->stream));
  TC_CUDA(cudaStreamSynchronize(g->stream));
  return TC_OK;
}

int tc_list_triangles(tc_graph* g, uint32_t* tri_out, int64_t cap, int64_t* count_out) {
  if (!g || !count_out) return fail(TC_ERR_INVALID_ARG, "tc_list_triangles: NULL argument");
  if (tri_out && cap < 0) return fail(TC_ERR_INVALID_ARG, "tc_list_triangles: cap < 0");
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  // T first (the hashed count), so the list is written only when it fits
  uint64_t T = 0;
  TC_TRY(count_cover(g, nullptr, &T));
  *count_out = (int64_t)T;
  if (!tri_out || T == 0) return TC_OK;
  if ((int64_t)T > cap)
    return fail(TC_ERR_CAPACITY, "tc_list_triangles: T = %llu > cap = %lld",
                (unsigned long long)T, (long long)cap);
  const bool dev = is_device_ptr(tri_out);
  DevBuf<uint32_t> tmp;
  uint32_t* out = tri_out;
  if (!dev) {
    TC_TRY(tmp.alloc((size_t)T * 3, g->stream));
    out = tmp.p;
  }
  uint64_t found = 0;
  TC_TRY(find_list(g, out, T, &found));
  if (found != T)
    return fail(TC_ERR_CUDA, "tc_list_triangles: found %llu triangles, counted %llu",
                (unsigned long long)found, (unsigned long long)T);
  if (!dev) {
    TC_CUDA(copy_out(tri_out, out, sizeof(uint32_t) * 3 * (size_t)T, g->stream));
    TC_CUDA(cudaStreamSynchronize(g->stream));
  }
  return TC_OK;
}

int tc_shard_bounds(tc_graph* g, int mode, int32_t nshards, int64_t* bounds_out) {
  if (!g || !bounds_out) return fail(TC_ERR_INVALID_ARG, "tc_shard_bounds: NULL argument");
  if (mode != TC_MODE_COVER && mode != TC_MODE_PLAIN)
    return fail(TC_ERR_INVALID_ARG, "tc_shard_bounds: unknown mode %d", mode);
  if (nshards < 1) return fail(TC_ERR_INVALID_ARG, "tc_shard_bounds: nshards < 1");
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  if (mode == TC_MODE_COVER && g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
  return shard_bounds(g, mode, nshards, bounds_out);
}

int tc_count_range(tc_graph* g, int mode, int64_t begin, int64_t end, uint64_t* count_out) {
  if (!g || !count_out) return fail(TC_ERR_INVALID_ARG, "tc_count_range: NULL argument");
  if (mode != TC_MODE_COVER && mode != TC_MODE_PLAIN)
    return fail(TC_ERR_INVALID_ARG, "tc_count_range: unknown mode %d", mode);
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  if (mode == TC_MODE_COVER) {
    if (g->nlevels < 0) TC_TRY(compute_levels(g, nullptr, 0));
    if (g->num_cover < 0) TC_TRY(compute_cover(g));
  }
  const int64_t m = mode == TC_MODE_COVER ? g->num_cover : g->nnz;
  if (begin < 0 || end < begin || end > m)
    return fail(TC_ERR_INVALID_ARG, "tc_count_range: [%lld, %lld) not within [0, %lld]",
                (long long)begin, (long long)end, (long long)m);
  uint64_t T = 0;
  if (end > begin) {
    if (mode == TC_MODE_COVER) TC_TRY(count_cover(g, nullptr, &T, begin, end));
    else TC_TRY(count_plain(g, &T, nullptr, begin, end));
  }
  *count_out = T;
  return TC_OK;
}

int tc_cover_edge_counts(tc_graph* g, uint32_t* counts_out, int64_t cap) {
  if (!g || !counts_out) return fail(TC_ERR_INVALID_ARG, "tc_cover_edge_counts: NULL argument");
  std::lock_guard<std::mutex> lk(g->mu);
  DeviceGuard dg(g->device);
  if (g->num_cover < 0) TC_TRY(compute_cover(g));
  if (g->num_cover > cap)
    return fail(TC_ERR_CAPACITY, "tc_cover_edge_counts: |H| = %lld > cap = %lld",
                (long long)g->num_cover, (long long)cap);
  if (g->num_cover == 0) return TC_OK;
  uint64_t T = 0;
  if (is_device_ptr(counts_out)) {
    TC_TRY(count_cover(g, counts_out, &T));
  } else {
    DevBuf<uint32_t> tmp;
    TC_TRY(tmp.alloc((size_t)g->num_cover, g->stream));
    TC_TRY(count_cover(g, tmp.p, &T));
    TC_CUDA(copy_out(counts_out, tmp.p, sizeof(uint32_t) * (size_t)g->num_cover, g->stream));
    TC_CUDA(cudaStreamSynchronize(g->stream));
  }
  return TC_OK;
}

}  // extern "C"

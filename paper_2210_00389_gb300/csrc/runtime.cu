// Error reporting, the allocator hook and small runtime helpers.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace tc {

std::atomic<unsigned long long> g_kernel_launches{0};

static thread_local char g_last_error[512] = "";

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  int status = (e == cudaErrorMemoryAllocation) ? TC_ERR_OOM : TC_ERR_CUDA;
  const char* base = strrchr(file, '/');
  fail(status, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
  cudaGetLastError();  // clear the sticky-free error state of the runtime
  return status;
}

// ---------------------------------------------------------------- allocator
static std::mutex g_alloc_mu;
static tc_alloc_fn g_alloc = nullptr;
static tc_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

// The device's default stream-ordered memory pool returns freed memory to
// the system at every synchronisation unless told otherwise; remapping it
// on the next allocation costs milliseconds and serialises concurrent work.
// Once per device (per process), let the pool keep what it has.
static void keep_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  done[dev] = true;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
}

int dev_alloc(void** p, size_t bytes, cudaStream_t stream) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  tc_alloc_fn a;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
    ctx = g_alloc_ctx;
  }
  if (a) {
    *p = a(bytes, (void*)stream, ctx);
    if (!*p) return fail(TC_ERR_OOM, "allocator hook returned NULL for %zu bytes", bytes);
    return TC_OK;
  }
  keep_pool_memory();
  cudaError_t e = cudaMallocAsync(p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TC_ERR_OOM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  return TC_OK;
}

void dev_free(void* p, cudaStream_t stream) {
  if (!p) return;
  tc_free_fn f;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f = g_free;
    ctx = g_alloc_ctx;
  }
  if (f) {
    f(p, (void*)stream, ctx);
  } else {
    cudaFreeAsync(p, stream);
  }
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

cudaError_t copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 1;
    }
    cached[dev] = v;
  }
  return cached[dev];
}

}  // namespace tc

extern "C" {

const char* tc_strerror(int status) {
  switch (status) {
    case TC_OK: return "ok";
    case TC_ERR_INVALID_ARG: return "invalid argument";
    case TC_ERR_INVALID_GRAPH: return "invalid graph";
    case TC_ERR_OOM: return "out of device memory";
    case TC_ERR_CUDA: return "CUDA error";
    case TC_ERR_CAPACITY: return "output buffer too small";
    case TC_ERR_TIMEOUT: return "timed out";
    case TC_ERR_AGAIN: return "queue full, try again";
    case TC_ERR_NOT_FOUND: return "not found";
    case TC_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

const char* tc_last_error(void) { return tc::g_last_error; }

int tc_version(void) { return 100; }

uint64_t tc_kernel_launches(void) { return tc::g_kernel_launches.load(); }

int tc_set_allocator(tc_alloc_fn alloc, tc_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return tc::fail(TC_ERR_INVALID_ARG, "tc_set_allocator: give both callbacks or neither");
  std::lock_guard<std::mutex> lk(tc::g_alloc_mu);
  tc::g_alloc = alloc;
  tc::g_free = free_fn;
  tc::g_alloc_ctx = alloc ? ctx : nullptr;
  return TC_OK;
}

}  // extern "C"

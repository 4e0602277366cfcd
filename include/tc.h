/*
 * tc.h — C ABI of the GB300 cover-edge triangle-counting library (libcetc).
 *
 * Method: D. A. Bader et al., "Triangle Counting Through Cover-Edges"
 * (arXiv 2210.00389).  Alg. 1 (CETC): label every vertex with its BFS level
 * (Def. 2), take the horizontal edges (both ends on one level) as the
 * cover-edge set H (Thm. 1), and for every (u,v) in H with u < v count the
 * common neighbours w with L(w) != L(u), or L(w) = L(u) and w > v (Thm. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: TC_OK (0) or a negative TC_ERR_* code.  No C++ exception
 *    ever crosses this boundary.  tc_strerror() names a code;
 *    tc_last_error() gives a message for the calling thread's last failure.
 *  - Graphs are simple and undirected, given as a symmetric CSR (the input format of Sec. III):
 *    offsets int64[n+1] (offsets[0] = 0, non-decreasing, offsets[n] = nnz),
 *    cols uint32[nnz], every row sorted strictly ascending, no self-loops,
 *    every entry < n.  nnz = 2|E|.
 *  - "host or device" pointers are classified with cudaPointerGetAttributes:
 *    device (or managed) memory of the current device is written/read on
 *    the GPU, anything else is treated as host memory.
 *  - Every call on a tc_graph runs on the CUDA stream given at creation and
 *    returns only after its results are complete and visible to the host.
 *  - Thread safety: calls on one tc_graph from several host threads are
 *    serialized by a lock inside the graph (each call runs alone on the
 *    graph's stream); tc_graph_destroy must not overlap any other call on
 *    the same graph.  Different graphs are independent; a tc_server takes
 *    calls from any thread.
 *  - Device faults are never raised on purpose: device-side checks set an
 *    error word that the host turns into a status code.
 */
#ifndef TC_H_
#define TC_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = -1,   /* NULL where a pointer is required, bad mode, ... */
  TC_ERR_INVALID_GRAPH = -2, /* CSR breaks the rules above (validation flags)   */
  TC_ERR_OOM = -3,           /* device allocation failed / over budget          */
  TC_ERR_CUDA = -4,          /* a CUDA runtime call failed                      */
  TC_ERR_CAPACITY = -5,      /* caller's output buffer too small                */
  TC_ERR_TIMEOUT = -6,       /* a bounded device/host wait ran out              */
  TC_ERR_AGAIN = -7,         /* queue full, try later                           */
  TC_ERR_NOT_FOUND = -8,     /* unknown ticket / graph id                       */
  TC_ERR_CANCELLED = -9      /* request cancelled (server shut down)            */
};

/* Static string naming a status code (never NULL). */
TC_API const char* tc_strerror(int status);
/* Message describing the calling thread's most recent failure ("" if none). */
TC_API const char* tc_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
TC_API int tc_version(void);
/* Diagnostics: number of CUDA kernels this library has launched in the
 * process so far (all threads, all devices). */
TC_API uint64_t tc_kernel_launches(void);

/* --------------------------------------------------------------- memory */
/* Route the library's device allocations (graph buffers and temporaries)
 * through caller callbacks, e.g. a framework's caching allocator.
 * alloc(bytes, stream, ctx) returns device memory usable on `stream` or NULL;
 * free(ptr, stream, ctx) releases it.  Pass NULLs to restore the default
 * (cudaMallocAsync / cudaFreeAsync on the call's stream).  Process-wide; call
 * it while no graph or server exists.  Returns TC_ERR_INVALID_ARG when only
 * one of the two callbacks is given. */
typedef void* (*tc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*tc_free_fn)(void* ptr, void* stream, void* ctx);
TC_API int tc_set_allocator(tc_alloc_fn alloc, tc_free_fn free_fn, void* ctx);

/* ---------------------------------------------------------------- graphs */
typedef struct tc_graph tc_graph; /* opaque: device CSR + cached levels and H */

/* Borrowed view of a caller-owned CSR; read only during the call unless
 * TC_GRAPH_BORROW is given. */
typedef struct {
  const int64_t* offsets; /* int64[n+1] */
  const uint32_t* cols;   /* uint32[nnz] */
  uint32_t n;             /* |V| */
  int64_t nnz;            /* 2|E| = offsets[n] */
  int on_device;          /* 0: host pointers, 1: device pointers */
} tc_csr_view;

enum {
  TC_GRAPH_VALIDATE = 1u,   /* check the CSR rules on the GPU (O(n + nnz))   */
  TC_GRAPH_CHECK_SYM = 2u,  /* also check symmetry: (u,v) present => (v,u)   */
  TC_GRAPH_BORROW = 4u      /* device views only: keep using the caller's
                               buffers instead of copying; they must stay
                               alive and unchanged until tc_graph_destroy    */
};

/* Build a graph object from a CSR (the input format of Sec. III).  Host views are
 * copied to the device; device views are copied device-to-device unless
 * TC_GRAPH_BORROW.  Also computes the degree of every vertex.  Errors:
 * TC_ERR_INVALID_ARG (NULL csr/out, nnz < 0, BORROW on a host view),
 * TC_ERR_INVALID_GRAPH (validation failed; *out untouched), TC_ERR_OOM,
 * TC_ERR_CUDA.  `cuda_stream` may be NULL (the legacy default stream). */
TC_API int tc_graph_create(const tc_csr_view* csr, uint32_t flags, void* cuda_stream,
                    tc_graph** out);
/* Release every device buffer the graph owns.  NULL is a no-op. */
TC_API int tc_graph_destroy(tc_graph* g);
/* Drop cached levels, cover edges and counts so the next call recomputes
 * them (used to time the full path). */
TC_API int tc_graph_invalidate(tc_graph* g);

typedef struct {
  uint32_t n;
  int64_t nnz;          /* 2|E| */
  int64_t num_edges;    /* |E| */
  uint32_t max_degree;
  int64_t nlevels;      /* 1 + max level, or -1 if levels are not computed */
  int64_t num_cover;    /* |H|, or -1 if not computed */
  uint32_t num_roots;   /* BFS roots of the last level computation */
} tc_graph_info_t;
TC_API int tc_graph_info(const tc_graph* g, tc_graph_info_t* info);

/* Def. 2 and Alg. 1: BFS levels, L(v) = shortest distance from
 * the root of v's connected component.
 *   roots == NULL (nroots ignored): the first root is the vertex of maximum
 *     degree (lowest id on ties); every other component is rooted at its
 *     lowest vertex id.
 *   roots != NULL: host array of nroots vertex ids, taken in order; a root
 *     in a component already reached by an earlier root is skipped; every
 *     component no root reaches is rooted at its lowest id.
 * levels_out: NULL, or host/device uint32[n] receiving L.  nlevels_out: NULL
 * or receives 1 + max L (0 when n = 0).  Levels are cached in the graph (and
 * any cached cover-edge set is dropped).  Errors: TC_ERR_INVALID_ARG (root
 * >= n), TC_ERR_OOM, TC_ERR_CUDA. */
TC_API int tc_bfs_levels(tc_graph* g, const uint32_t* roots, uint32_t nroots,
                  uint32_t* levels_out, uint32_t* nlevels_out);

/* Thm. 1 and Alg. 1: the cover-edge set
 * H = {(u,v) in E : u < v, L(u) = L(v)} in ascending (u, v) order (CSR
 * order).  Computes levels with the default root rule if none are cached.
 * uv_out: NULL or host/device uint32[2*cap], pair i = (uv[2i], uv[2i+1]).
 * *count_out receives |H|.  If |H| > cap and uv_out != NULL, nothing is
 * written to uv_out and TC_ERR_CAPACITY is returned (with *count_out set). */
TC_API int tc_cover_edges(tc_graph* g, uint32_t* uv_out, int64_t cap, int64_t* count_out);

enum {
  TC_MODE_COVER = 0, /* Alg. 1: cover edges + count-once rule (Thm. 2)       */
  TC_MODE_PLAIN = 1  /* direction-oriented edge iterator over every edge
                        u < v, counting common neighbours w > v (Sec. I, V-A) */
};

/* Intersection technique (Sec. V-A lists merging, binary search and
 * hashing): OR'ed into tc_count's mode, TC_INTERSECT_MERGE counts with the
 * warp-per-edge merge / binary-search kernels instead of the owner-grouped
 * hash intersection (same result; a comparison arm). */
enum { TC_INTERSECT_MERGE = 0x10 };

/* Exact triangle count T (uint64, host pointer count_out).  TC_MODE_COVER
 * runs BFS + cover extraction if not cached, then the intersection with the
 * count-once rule and the reduction; TC_MODE_PLAIN runs the intersection
 * over every edge.  mode may carry TC_INTERSECT_MERGE.
 * Errors: TC_ERR_INVALID_ARG, TC_ERR_OOM, TC_ERR_CUDA. */
TC_API int tc_count(tc_graph* g, int mode, uint64_t* count_out);

/* Per-cover-edge counts of Alg. 1: counts_out[i] = number of w that
 * the count-once rule accepts for cover edge i (in tc_cover_edges order).
 * counts_out: host/device uint32[cap].  TC_ERR_CAPACITY if |H| > cap. */
TC_API int tc_cover_edge_counts(tc_graph* g, uint32_t* counts_out, int64_t cap);

/* Triangle finding (the cover edges' second use, Alg. 1 / Thm. 2): every
 * triangle is found once, at the cover edge (u, v), u < v, that the
 * count-once rule attributes it to, with apex w.
 *
 * tc_vertex_counts: counts_out (host or device uint64[n]) receives, for
 * every vertex, the number of triangles that contain it (sum = 3T).
 *
 * tc_list_triangles: tri_out (host or device uint32[3 * cap], or NULL to only
 * count) receives the T triangles as triples (u, v, w) in no particular
 * order; *count_out = T.  If T > cap and tri_out != NULL, nothing is written
 * and TC_ERR_CAPACITY is returned (with *count_out set).
 * Both run the BFS and the cover extraction first if they are not cached.
 * Errors: TC_ERR_INVALID_ARG, TC_ERR_CAPACITY, TC_ERR_OOM, TC_ERR_CUDA. */
TC_API int tc_vertex_counts(tc_graph* g, uint64_t* counts_out);
TC_API int tc_list_triangles(tc_graph* g, uint32_t* tri_out, int64_t cap, int64_t* count_out);

/* Shards of the count for several GPUs (the CSR and the levels replicated on
 * each; every GPU counts one contiguous slice; the slice counts add up to T).
 * The count is a sum of independent per-edge terms over the mode's edge
 * index space -- cover: the cover edges in tc_cover_edges order (Alg. 1,
 * Thm. 2); plain: the CSR entries, those with u > v adding nothing.
 *
 * tc_shard_bounds: bounds_out (host int64[nshards + 1]) receives
 * 0 = b_0 <= b_1 <= ... <= b_nshards = |edges|, chosen so that the slices
 * [b_k, b_k+1) carry about equal estimated work (sum over their edges of
 * min(d(u), d(v)) + 1); inner bounds are multiples of 4,096 or |edges|.
 * Runs the BFS and the cover extraction first if they are not cached
 * (cover mode).
 * Errors: TC_ERR_INVALID_ARG (NULL, unknown mode, nshards < 1), TC_ERR_OOM,
 * TC_ERR_CUDA.
 *
 * tc_count_range: *count_out (host) = the sum of the per-edge terms of the
 * edges [begin, end) (0 <= begin <= end <= |edges|, else TC_ERR_INVALID_ARG);
 * an empty range counts 0.  Summed over the slices of any partition of
 * [0, |edges|) the counts equal tc_count's. */
TC_API int tc_shard_bounds(tc_graph* g, int mode, int32_t nshards, int64_t* bounds_out);
TC_API int tc_count_range(tc_graph* g, int mode, int64_t begin, int64_t end, uint64_t* count_out);

/* Timings (device ms, CUDA events on the graph's stream) of the most recent
 * tc_count / tc_bfs_levels / tc_cover_edges call, per stage, and work sizes. */
typedef struct {
  float ms_validate, ms_bfs, ms_cover, ms_bucket, ms_intersect, ms_total;
  uint32_t bfs_levels;        /* level-synchronous iterations run */
  uint32_t bfs_bottom_up;     /* of which bottom-up */
  int64_t edges_intersected;  /* |H| (cover) or |E| (plain) */
  int64_t list_elems;         /* sum of list lengths handed to the intersection */
  uint64_t reserved0;
  uint32_t kernel_launches;   /* kernels launched by the call */
  float ms_main_kernel;       /* the dominant intersection kernel alone */
} tc_stats_t;
TC_API int tc_graph_stats(const tc_graph* g, tc_stats_t* out);

/* Plain all-edge triangle count (as tc_count with TC_MODE_PLAIN) of a
 * device-resident CSR, without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc/cudaFree at this point -- those calls can synchronize the
 * device, which a latency-bound loop overlapping several streams must avoid;
 * applications whose device memory is owned by another allocator or budgeted
 * once at start-up may not allocate behind it.
 *   offsets, cols: device memory, a valid symmetric CSR (the rules above;
 *     not validated here; column ids >= n are skipped).
 *   count_out: device memory, receives the count (uint64).
 *   cuda_stream: stream for the work (NULL = legacy default stream).
 * Asynchronous: returns after enqueueing; read *count_out after the stream
 * completes.  Scratch is one static device array of 16 MiB + 256 B that
 * every GPU loading the library keeps until the process exits; n may be at
 * most 4,194,304 (TC_ERR_CAPACITY beyond it, checked before any work).  The
 * first call on a device looks up that device's scratch address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  The cached address belongs to the CUDA context current
 * at that first call: after cudaDeviceReset (or anything else that destroys
 * the device's primary context) the cache is stale, so do not call this
 * entry point again in that process.  All calls share the array: calls that overlap on the GPU
 * race and give wrong counts, so serialize them (one stream, or events).
 * Errors: TC_ERR_CAPACITY, TC_ERR_INVALID_ARG (NULL, nnz < 0, or a pointer
 * that is not device memory), TC_ERR_CUDA. */
TC_API int tc_count_plain_static(const int64_t* offsets, const uint32_t* cols, uint32_t n,
                                 int64_t nnz, uint64_t* count_out, void* cuda_stream);

/* ---------------------------------------------------------------- batch */
/* Tunables of the batched kernel (NULL = built-in defaults; the Python
 * binding passes the table written by its autotuner). */
typedef struct {
  int32_t block_threads;   /* threads per block of the persistent batch kernel: 128, 256, 512 */
  int32_t blocks_per_sm;   /* resident blocks per SM (1..16) */
  int32_t skew;            /* warp merge when the longer list is <= skew x the shorter,
                              else binary search of the shorter in the longer (>= 2) */
  int32_t tiny_max_nnz;    /* graphs with at most this many CSR entries (and at most
                              65,536 vertices) go to the persistent per-graph kernel;
                              larger ones are packed into one disjoint union counted by
                              the single-graph pipeline (0 = built-in 32,768; at most
                              2^22) */
  int32_t reserved[4];
} tc_options;

/* Count ngraphs independent graphs in one persistent, CUDA-graph-captured
 * launch sequence.  graphs: host array of views (host or device pointers).
 * counts_out: host uint64[ngraphs]; status_out: host int[ngraphs] (NULL
 * allowed) with a per-graph status (TC_OK or TC_ERR_INVALID_GRAPH).
 * Returns TC_OK if the batch ran (per-graph failures are in status_out). */
TC_API int tc_count_batch(const tc_csr_view* graphs, int32_t ngraphs, int mode,
                   const tc_options* opt, void* cuda_stream, uint64_t* counts_out,
                   int* status_out);

/* ---------------------------------------------------------------- serving */
/* A request loop on the current device (no paper counterpart: a systems form
 * of Alg. 1).  Small one-shot graphs (n <= 65,536, nnz <= 2^20) and the
 * other requests (large one-shot graphs, requests on resident graphs) wait
 * in two queues, each admitted in arrival order: a small request as soon as
 * its estimated device bytes fit the budget next to the resident graphs and
 * the requests in flight, another request when, in addition, fewer than
 * `slots` of its kind are in flight.  Admitted small graphs are grouped and
 * counted together with tc_count_batch each time the batch worker is free
 * (continuous batching, on a high-priority stream); resident and large
 * requests run on worker threads with their own streams, so requests overlap
 * on the device.  Counts are the same exact integers as tc_count's. */
typedef struct tc_server tc_server;
typedef struct {
  size_t hbm_budget_bytes; /* admission limit for resident + in-flight graphs */
  int32_t slots;           /* max large or resident requests in flight (> 0) */
  int32_t queue_capacity;  /* max queued, not yet admitted requests (<= 0: 4096) */
  int32_t wait_limit_ms;   /* a request not admitted within this time finishes
                              with TC_ERR_TIMEOUT (<= 0: 10000) */
  int32_t fail_admitted;   /* test hook: k > 0 makes the k-th admitted request fail
                              with TC_ERR_OOM as if its device allocation had
                              failed; 0 = off */
  int32_t borrow_views;    /* 0: tc_serve_submit copies a one-shot CSR before it
                              returns.  1: it keeps the caller's pointers, which
                              must stay valid and unchanged until tc_serve_poll
                              reports the request done (or tc_serve_destroy
                              returns): no copy on the submitting thread */
  int32_t reserved[2];     /* must be 0 */
} tc_serve_config;

/* Start the scheduler and worker threads.  TC_ERR_INVALID_ARG for a NULL
 * or non-positive budget / slots. */
TC_API int tc_serve_create(const tc_serve_config* cfg, tc_server** out);
/* Upload a graph that stays resident: its CSR (host or device view, copied),
 * BFS levels and cover edges are computed now and reused by every request
 * on *graph_id.  TC_ERR_OOM if it does not fit the budget; CSR errors as
 * tc_graph_create with TC_GRAPH_VALIDATE. */
TC_API int tc_serve_register(tc_server* s, const tc_csr_view* csr, uint64_t* graph_id);
/* Queue a count request (mode TC_MODE_COVER or TC_MODE_PLAIN) on a resident
 * graph (csr_or_null == NULL) or on a one-shot CSR (host or device view;
 * copied before return, so the caller's buffers are free afterwards, unless
 * the server borrows views -- see tc_serve_config.borrow_views).
 * Errors: TC_ERR_AGAIN (queue full), TC_ERR_OOM (the request alone exceeds
 * the budget), TC_ERR_NOT_FOUND (unknown graph id), TC_ERR_CANCELLED
 * (shutting down), TC_ERR_INVALID_ARG. */
TC_API int tc_serve_submit(tc_server* s, const tc_csr_view* csr_or_null, uint64_t graph_id,
                    int mode, uint64_t* ticket);
/* Non-blocking: *done = 1 when the request finished, then *count and
 * *status (TC_OK, TC_ERR_INVALID_GRAPH, TC_ERR_TIMEOUT, TC_ERR_OOM, ...) are
 * set and the ticket is forgotten; TC_ERR_NOT_FOUND for unknown tickets. */
TC_API int tc_serve_poll(tc_server* s, uint64_t ticket, int* done, uint64_t* count, int* status);
/* Stop accepting, cancel queued requests, finish the ones running, join the
 * threads and free the resident graphs.  NULL is a no-op. */
TC_API int tc_serve_destroy(tc_server* s);

#ifdef __cplusplus
}
#endif
#endif /* TC_H_ */

/*
 * Seeded synthetic graph generators and the symmetric-CSR builder.
 *
 * This file produces INPUTS only.  It holds none of the triangle-counting
 * arithmetic (no BFS, no levels, no intersections); both the CPU oracle and
 * the CUDA path consume the CSR it builds.
 *
 * Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): output i of the stream with
 * seed s is mix(s + (i+1) * 0x9E3779B97F4A7C15).  Being counter-based, every
 * draw is a pure function of (seed, index), so the edge list does not depend
 * on the thread count or the machine.
 *
 * Generators:
 *   R-MAT (Chakrabarti, Zhan & Faloutsos 2004) with the Graph500 quadrant
 *   probabilities a/b/c/d = 0.57/0.19/0.19/0.05, n = 2^scale and
 *   m = edgefactor * n generated pairs (the paper's Sec. IV-A parameters);
 *   Fisher-Yates relabelling; Chung-Lu power-law weights with an alias table;
 *   Erdos-Renyi G(n, p) islands.
 *
 * CSR builder: symmetrise, drop self-loops and duplicate edges, sort each
 * adjacency list ascending.  Output is int64 offsets[n+1] + uint32 cols[nnz].
 *
 * Plain C11 + pthreads; no architecture-specific code, so x86-64 and aarch64
 * hosts build identical graphs from identical seeds (the Chung-Lu weights use
 * libm pow(), so that generator is only guaranteed identical on one host).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_EXPORT __attribute__((visibility("default")))

static inline uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform integer in [0, bound) from the top 32 bits of r (Lemire 2019) */
static inline uint32_t bounded32(uint64_t r, uint32_t bound) {
  return (uint32_t)(((r >> 32) * (uint64_t)bound) >> 32);
}

GG_EXPORT uint64_t gg_splitmix64(uint64_t seed, uint64_t i) { return sm64(seed, i); }

/* ------------------------------------------------------------------------ */
/* tiny thread pool helper: run fn(ctx, t, T) on T threads                   */
typedef void (*gg_task)(void* ctx, int t, int T);
typedef struct { gg_task fn; void* ctx; int t, T; } gg_thr_arg;
static void* gg_thr_main(void* p) {
  gg_thr_arg* a = (gg_thr_arg*)p;
  a->fn(a->ctx, a->t, a->T);
  return NULL;
}
static void gg_parallel(gg_task fn, void* ctx, int T) {
  if (T <= 1) { fn(ctx, 0, 1); return; }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)T);
  gg_thr_arg* args = (gg_thr_arg*)malloc(sizeof(gg_thr_arg) * (size_t)T);
  for (int t = 0; t < T; ++t) {
    args[t].fn = fn; args[t].ctx = ctx; args[t].t = t; args[t].T = T;
    if (t > 0) pthread_create(&th[t], NULL, gg_thr_main, &args[t]);
  }
  fn(ctx, 0, T);
  for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
  free(th); free(args);
}
static inline void gg_range(int64_t total, int t, int T, int64_t* lo, int64_t* hi) {
  int64_t chunk = (total + T - 1) / T;
  *lo = chunk * t; if (*lo > total) *lo = total;
  *hi = *lo + chunk; if (*hi > total) *hi = total;
}

/* ------------------------------------------------------------------------ */
/* R-MAT                                                                     */
typedef struct {
  int scale; int64_t m; uint64_t seed;
  uint32_t ta, tab, tabc;         /* cumulative quadrant thresholds * 2^32 */
  uint32_t* src; uint32_t* dst;
} rmat_ctx;

static void rmat_task(void* p, int t, int T) {
  rmat_ctx* c = (rmat_ctx*)p;
  int64_t lo, hi; gg_range(c->m, t, T, &lo, &hi);
  const int draws = (c->scale + 1) / 2;      /* two levels per 64-bit draw */
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t u = 0, v = 0;
    int level = 0;
    for (int j = 0; j < draws; ++j) {
      uint64_t r = sm64(c->seed, (uint64_t)e * (uint64_t)draws + (uint64_t)j);
      for (int half = 0; half < 2 && level < c->scale; ++half, ++level) {
        uint32_t x = half ? (uint32_t)(r >> 32) : (uint32_t)r;
        uint32_t bu, bv;
        if (x < c->ta)        { bu = 0; bv = 0; }
        else if (x < c->tab)  { bu = 0; bv = 1; }
        else if (x < c->tabc) { bu = 1; bv = 0; }
        else                  { bu = 1; bv = 1; }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
      }
    }
    c->src[e] = u; c->dst[e] = v;
  }
}

/* Thresholds are passed pre-scaled by 2^32 (floor(a*2^32) etc.) so that the
 * generator is integer-only. */
GG_EXPORT int gg_rmat_edges(int scale, int64_t m, uint64_t seed, uint32_t ta,
                            uint32_t tab, uint32_t tabc, uint32_t* src,
                            uint32_t* dst, int nthreads) {
  if (scale < 1 || scale > 32 || m < 0 || !src || !dst) return -1;
  rmat_ctx c = {scale, m, seed, ta, tab, tabc, src, dst};
  gg_parallel(rmat_task, &c, nthreads);
  return 0;
}

/* Fisher-Yates permutation of 0..n-1 driven by the stream `seed`; then
 * endpoints are mapped through it. */
GG_EXPORT int gg_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  if (n < 2) return 0;
  for (uint32_t i = n - 1; i >= 1; --i) {
    uint32_t j = bounded32(sm64(seed, i), i + 1);
    uint32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
  }
  return 0;
}

typedef struct { const uint32_t* perm; uint32_t* a; int64_t m; } map_ctx;
static void map_task(void* p, int t, int T) {
  map_ctx* c = (map_ctx*)p;
  int64_t lo, hi; gg_range(c->m, t, T, &lo, &hi);
  for (int64_t e = lo; e < hi; ++e) c->a[e] = c->perm[c->a[e]];
}
GG_EXPORT int gg_apply_permutation(const uint32_t* perm, uint32_t* a, int64_t m,
                                   int nthreads) {
  map_ctx c = {perm, a, m};
  gg_parallel(map_task, &c, nthreads);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Chung-Lu endpoints drawn from an alias table (Walker 1977; Vose 1991).     */
/* prob_thr[i] = P(keep column i) * 2^32, alias[i] = fallback column.         */
GG_EXPORT int gg_alias_table(const double* w, uint32_t k, uint32_t* prob_thr,
                             uint32_t* alias) {
  if (k == 0) return -1;
  double sum = 0.0;
  for (uint32_t i = 0; i < k; ++i) sum += w[i];
  if (!(sum > 0.0)) return -1;
  double* q = (double*)malloc(sizeof(double) * k);
  uint32_t* small = (uint32_t*)malloc(sizeof(uint32_t) * k);
  uint32_t* large = (uint32_t*)malloc(sizeof(uint32_t) * k);
  uint32_t ns = 0, nl = 0;
  for (uint32_t i = 0; i < k; ++i) {
    q[i] = w[i] * (double)k / sum;
    if (q[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns > 0 && nl > 0) {
    uint32_t s = small[--ns], l = large[nl - 1];
    double ps = q[s];
    prob_thr[s] = ps >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(ps * 4294967296.0);
    alias[s] = l;
    q[l] = (q[l] + q[s]) - 1.0;
    if (q[l] < 1.0) { --nl; small[ns++] = l; }
  }
  while (nl > 0) { uint32_t l = large[--nl]; prob_thr[l] = 0xFFFFFFFFu; alias[l] = l; }
  while (ns > 0) { uint32_t s = small[--ns]; prob_thr[s] = 0xFFFFFFFFu; alias[s] = s; }
  free(q); free(small); free(large);
  return 0;
}

typedef struct {
  const uint32_t* prob_thr; const uint32_t* alias; uint32_t k; uint32_t base;
  int64_t m; uint64_t seed; uint32_t* src; uint32_t* dst;
} cl_ctx;

static inline uint32_t alias_draw(const cl_ctx* c, uint64_t r) {
  uint32_t col = bounded32(r, c->k);
  return ((uint32_t)r < c->prob_thr[col]) ? col : c->alias[col];
}
static void cl_task(void* p, int t, int T) {
  cl_ctx* c = (cl_ctx*)p;
  int64_t lo, hi; gg_range(c->m, t, T, &lo, &hi);
  for (int64_t e = lo; e < hi; ++e) {
    c->src[e] = c->base + alias_draw(c, sm64(c->seed, 2 * (uint64_t)e));
    c->dst[e] = c->base + alias_draw(c, sm64(c->seed, 2 * (uint64_t)e + 1));
  }
}
GG_EXPORT int gg_alias_edges(const uint32_t* prob_thr, const uint32_t* alias,
                             uint32_t k, uint32_t base, int64_t m, uint64_t seed,
                             uint32_t* src, uint32_t* dst, int nthreads) {
  cl_ctx c = {prob_thr, alias, k, base, m, seed, src, dst};
  gg_parallel(cl_task, &c, nthreads);
  return 0;
}

/* Erdos-Renyi G(k, p) on vertices base..base+k-1: pair (i<j) is an edge when
 * its draw is below thr = p * 2^64.  Returns the number of edges written, or
 * -1 if more than cap would be needed (call with cap < 0 to only count). */
GG_EXPORT int64_t gg_er_edges(uint32_t k, uint32_t base, uint64_t thr,
                              uint64_t seed, uint32_t* src, uint32_t* dst,
                              int64_t cap) {
  int64_t cnt = 0;
  uint64_t idx = 0;
  for (uint32_t i = 0; i < k; ++i) {
    for (uint32_t j = i + 1; j < k; ++j, ++idx) {
      if (sm64(seed, idx) < thr) {
        if (cap >= 0) {
          if (cnt >= cap) return -1;
          src[cnt] = base + i; dst[cnt] = base + j;
        }
        ++cnt;
      }
    }
  }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Symmetric CSR builder                                                     */
typedef struct {
  uint32_t n; int64_t m; const uint32_t* src; const uint32_t* dst;
  uint32_t* deg;          /* atomics */
  int64_t* off;           /* raw offsets (before dedup) */
  int64_t* cursor;        /* atomics */
  uint32_t* raw;          /* raw cols */
  uint32_t* newdeg;
  int64_t* out_off; uint32_t* out_cols;
  int bad;                /* endpoint >= n */
} csr_ctx;

static void csr_count(void* p, int t, int T) {
  csr_ctx* c = (csr_ctx*)p;
  int64_t lo, hi; gg_range(c->m, t, T, &lo, &hi);
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t u = c->src[e], v = c->dst[e];
    if (u >= c->n || v >= c->n) { __atomic_store_n(&c->bad, 1, __ATOMIC_RELAXED); continue; }
    if (u == v) continue;
    __atomic_fetch_add(&c->deg[u], 1u, __ATOMIC_RELAXED);
    __atomic_fetch_add(&c->deg[v], 1u, __ATOMIC_RELAXED);
  }
}
static void csr_scatter(void* p, int t, int T) {
  csr_ctx* c = (csr_ctx*)p;
  int64_t lo, hi; gg_range(c->m, t, T, &lo, &hi);
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t u = c->src[e], v = c->dst[e];
    if (u >= c->n || v >= c->n || u == v) continue;
    int64_t pu = __atomic_fetch_add(&c->cursor[u], 1, __ATOMIC_RELAXED);
    int64_t pv = __atomic_fetch_add(&c->cursor[v], 1, __ATOMIC_RELAXED);
    c->raw[pu] = v; c->raw[pv] = u;
  }
}
static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}
/* LSD radix sort for long rows (qsort is fine for short ones) */
static void radix_u32(uint32_t* a, uint32_t* tmp, int64_t len) {
  uint32_t* from = a; uint32_t* to = tmp;
  for (int shift = 0; shift < 32; shift += 8) {
    int64_t cnt[257];
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < len; ++i) cnt[((from[i] >> shift) & 255u) + 1]++;
    for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
    for (int64_t i = 0; i < len; ++i) to[cnt[(from[i] >> shift) & 255u]++] = from[i];
    uint32_t* s = from; from = to; to = s;
  }
  /* four passes: result is back in a */
}
static void csr_sort_rows(void* p, int t, int T) {
  csr_ctx* c = (csr_ctx*)p;
  int64_t lo, hi; gg_range(c->n, t, T, &lo, &hi);
  uint32_t* tmp = NULL; int64_t tmpcap = 0;
  for (int64_t u = lo; u < hi; ++u) {
    int64_t b = c->off[u], len = c->off[u + 1] - b;
    uint32_t* row = c->raw + b;
    if (len > 256) {
      if (len > tmpcap) { free(tmp); tmpcap = len; tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)len); }
      radix_u32(row, tmp, len);
    } else if (len > 1) {
      qsort(row, (size_t)len, sizeof(uint32_t), cmp_u32);
    }
    int64_t w = 0;
    for (int64_t i = 0; i < len; ++i)
      if (i == 0 || row[i] != row[i - 1]) row[w++] = row[i];
    c->newdeg[u] = (uint32_t)w;
  }
  free(tmp);
}
static void csr_compact(void* p, int t, int T) {
  csr_ctx* c = (csr_ctx*)p;
  int64_t lo, hi; gg_range(c->n, t, T, &lo, &hi);
  for (int64_t u = lo; u < hi; ++u)
    memcpy(c->out_cols + c->out_off[u], c->raw + c->off[u], sizeof(uint32_t) * c->newdeg[u]);
}

/* Pass 1: returns nnz of the cleaned symmetric CSR and keeps scratch in *h.
 * Pass 2 (gg_csr_finish) writes offsets[n+1] and cols[nnz].  Split in two so
 * the caller can allocate the exact output size. */
typedef struct { csr_ctx c; } gg_csr_handle;

GG_EXPORT void* gg_csr_begin(uint32_t n, int64_t m, const uint32_t* src,
                             const uint32_t* dst, int nthreads, int64_t* nnz_out) {
  gg_csr_handle* h = (gg_csr_handle*)calloc(1, sizeof(gg_csr_handle));
  csr_ctx* c = &h->c;
  c->n = n; c->m = m; c->src = src; c->dst = dst;
  c->deg = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
  c->off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  c->cursor = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  c->newdeg = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
  gg_parallel(csr_count, c, nthreads);
  if (c->bad) { *nnz_out = -1; return h; }
  c->off[0] = 0;
  for (uint32_t u = 0; u < n; ++u) c->off[u + 1] = c->off[u] + c->deg[u];
  memcpy(c->cursor, c->off, sizeof(int64_t) * ((size_t)n + 1));
  c->raw = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(c->off[n] > 0 ? c->off[n] : 1));
  gg_parallel(csr_scatter, c, nthreads);
  gg_parallel(csr_sort_rows, c, nthreads);
  int64_t nnz = 0;
  for (uint32_t u = 0; u < n; ++u) nnz += c->newdeg[u];
  *nnz_out = nnz;
  return h;
}

GG_EXPORT int gg_csr_finish(void* hp, int64_t* offsets, uint32_t* cols, int nthreads) {
  gg_csr_handle* h = (gg_csr_handle*)hp;
  csr_ctx* c = &h->c;
  int rc = 0;
  if (c->bad) {
    rc = -1;
  } else {
    offsets[0] = 0;
    for (uint32_t u = 0; u < c->n; ++u) offsets[u + 1] = offsets[u] + c->newdeg[u];
    c->out_off = offsets; c->out_cols = cols;
    gg_parallel(csr_compact, c, nthreads);
  }
  free(c->deg); free(c->off); free(c->cursor); free(c->newdeg); free(c->raw);
  free(h);
  return rc;
}

/*
 * CPU ORACLE for cover-edge triangle counting (CETC).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the package's smoke check and the benchmark's CPU-baseline leg may load
 * it; the library's product path never calls it and shares no code with it
 * (no headers, helpers, tables or pre/post-processing in common).
 *
 * Source: D. A. Bader et al., "Triangle Counting Through Cover-Edges"
 * (arXiv 2210.00389).  Every function below cites the passage it follows.
 *
 * Input everywhere: a simple undirected graph held in compressed sparse row
 * form, the input format of Sec. III, made symmetric: off[n+1] (int64),
 * cols[off[n]] (uint32), each row sorted ascending with no duplicates and
 * no self-loops.
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - Root rule.  Alg. 1 launches a BFS from an arbitrary vertex not yet reached.  The first
 *     root is the vertex of maximum degree (lowest id on ties); after its
 *     component, vertices are scanned in ascending id order and every still
 *     unvisited one starts a new BFS, i.e. every other component is rooted
 *     at its lowest id.  A caller may instead pass an explicit root list,
 *     used in order (a root already reached is skipped) before the scan.
 *   - Levels are BFS distances from the component root (Def. 2), so they do
 *     not depend on the traversal order, only on the roots.
 *   - Counts are exact unsigned 64-bit integers.
 *
 * Parity status: every function here is pinned by tests that do not call
 * it to compute their expected value (brute force, trace(A^3)/6, library
 * BFS distances, closed forms, Lemma 1 / Lemma 2 invariants).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define OR_EXPORT __attribute__((visibility("default")))
#define OR_UNVISITED 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Def. 2 + Alg. 1: BFS levels, restarted from every unvisited
 * vertex.  L[v] = shortest distance from the root of v's component.
 * Returns the number of levels (1 + max L), 0 for n = 0, -1 on bad input. */
static void bfs_from(uint32_t root, const int64_t* off, const uint32_t* cols,
                     uint32_t* L, uint32_t* queue) {
  int64_t head = 0, tail = 0;
  L[root] = 0;
  queue[tail++] = root;
  while (head < tail) {
    uint32_t x = queue[head++];
    for (int64_t e = off[x]; e < off[x + 1]; ++e) {
      uint32_t y = cols[e];
      if (L[y] == OR_UNVISITED) {
        L[y] = L[x] + 1;
        queue[tail++] = y;
      }
    }
  }
}

OR_EXPORT int64_t or_bfs_levels(uint32_t n, const int64_t* off, const uint32_t* cols,
                                const uint32_t* roots, uint32_t nroots, uint32_t* L) {
  if (n == 0) return 0;
  uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * n);
  if (!queue) return -1;
  for (uint32_t v = 0; v < n; ++v) L[v] = OR_UNVISITED;

  if (roots && nroots > 0) {
    for (uint32_t i = 0; i < nroots; ++i) {
      if (roots[i] >= n) { free(queue); return -1; }
      if (L[roots[i]] == OR_UNVISITED) bfs_from(roots[i], off, cols, L, queue);
    }
  } else {
    /* first root: maximum degree, lowest id on ties */
    uint32_t r0 = 0;
    for (uint32_t v = 1; v < n; ++v)
      if (off[v + 1] - off[v] > off[r0 + 1] - off[r0]) r0 = v;
    bfs_from(r0, off, cols, L, queue);
  }
  /* Alg. 1: every vertex still unvisited starts its own BFS */
  for (uint32_t v = 0; v < n; ++v)
    if (L[v] == OR_UNVISITED) bfs_from(v, off, cols, L, queue);

  uint32_t maxL = 0;
  for (uint32_t v = 0; v < n; ++v) if (L[v] > maxL) maxL = L[v];
  free(queue);
  return (int64_t)maxL + 1;
}

/* ------------------------------------------------------------------------ */
/* Thm. 1 + Alg. 1: the cover-edge set H = horizontal edges,
 * {(u,v) in E : L(u) = L(v), u < v}, emitted in ascending (u, v) order.
 * A tree edge always joins adjacent levels, so the horizontal edges of
 * Def. 2 (non-tree edges inside one level) are all edges inside one level.
 * Writes at most cap pairs (uv[2i] = u, uv[2i+1] = v); returns |H|. */
OR_EXPORT int64_t or_cover_edges(uint32_t n, const int64_t* off, const uint32_t* cols,
                                 const uint32_t* L, uint32_t* uv, int64_t cap) {
  int64_t h = 0;
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = cols[e];
      if (u < v && L[u] == L[v]) {
        if (uv && h < cap) { uv[2 * h] = u; uv[2 * h + 1] = v; }
        ++h;
      }
    }
  }
  return h;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 for one cover edge (u, v), u < v, L(u) = L(v):
 * the number of w in N(u) ∩ N(v) with L(u) != L(w), or L(u) = L(w) and
 * v < w.  N(u) ∩ N(v) is found by the two-pointer merge of the two sorted
 * adjacency lists (merge-path intersection, Sec. V-A). */
static uint64_t cover_edge_count(const int64_t* off, const uint32_t* cols,
                                 const uint32_t* L, uint32_t u, uint32_t v) {
  uint64_t c = 0;
  int64_t i = off[u], iend = off[u + 1];
  int64_t j = off[v], jend = off[v + 1];
  while (i < iend && j < jend) {
    uint32_t a = cols[i], b = cols[j];
    if (a < b) {
      ++i;
    } else if (b < a) {
      ++j;
    } else {
      uint32_t w = a;
      if (L[u] != L[w] || (L[u] == L[w] && v < w)) ++c;
      ++i; ++j;
    }
  }
  return c;
}

/* Alg. 1 in full after the BFS: T = sum over cover edges of the count above. */
OR_EXPORT uint64_t or_cetc_count(uint32_t n, const int64_t* off, const uint32_t* cols,
                                 const uint32_t* L) {
  uint64_t T = 0;
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = cols[e];
      if (L[u] == L[v] && u < v) T += cover_edge_count(off, cols, L, u, v);
    }
  }
  return T;
}

/* Per-edge counts of Alg. 1 for an explicit list of k cover edges
 * (uv[2i], uv[2i+1]).  Returns -1 if an entry is not a cover edge (u >= v,
 * levels differ or (u, v) not in E), else 0. */
OR_EXPORT int or_cetc_edge_counts(uint32_t n, const int64_t* off, const uint32_t* cols,
                                  const uint32_t* L, const uint32_t* uv, int64_t k,
                                  uint32_t* counts) {
  for (int64_t i = 0; i < k; ++i) {
    uint32_t u = uv[2 * i], v = uv[2 * i + 1];
    if (u >= n || v >= n || !(u < v) || L[u] != L[v]) return -1;
    /* membership of v in N(u) by bisection of the sorted row */
    int64_t lo = off[u], hi = off[u + 1];
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (cols[mid] < v) lo = mid + 1; else hi = mid;
    }
    if (!(lo < off[u + 1] && cols[lo] == v)) return -1;
    counts[i] = (uint32_t)cover_edge_count(off, cols, L, u, v);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The plain direction-oriented edge iterator (Sec. I and Sec. V-A): every
 * edge u < v, every common neighbour w > v, so each triangle a < b < c is
 * counted once, at its edge (a, b) with apex c.  The common neighbours of
 * one edge are found by the same two-pointer merge as above. */
static uint64_t plain_edge_count(const int64_t* off, const uint32_t* cols, uint32_t u,
                                 uint32_t v) {
  uint64_t c = 0;
  int64_t i = off[u], iend = off[u + 1];
  int64_t j = off[v], jend = off[v + 1];
  while (i < iend && j < jend) {
    uint32_t a = cols[i], b = cols[j];
    if (a < b) ++i;
    else if (b < a) ++j;
    else { if (a > v) ++c; ++i; ++j; }
  }
  return c;
}

OR_EXPORT uint64_t or_plain_count(uint32_t n, const int64_t* off, const uint32_t* cols) {
  uint64_t T = 0;
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = cols[e];
      if (u < v) T += plain_edge_count(off, cols, u, v);
    }
  }
  return T;
}

/* ------------------------------------------------------------------------ */
/* All-core forms of the three counting loops above, for graphs too large
 * for one core (R-MAT scale 22 and up).  Each is the single-threaded loop
 * with its outer loop over u shared among `threads` OpenMP threads (0 = the
 * OpenMP default) and the per-edge work unchanged: the same helpers, the
 * same predicate, the same uint64 sums.  Rows are handed out in small
 * dynamic chunks because hub rows cost far more than the rest. */
OR_EXPORT uint64_t or_cetc_count_mt(uint32_t n, const int64_t* off, const uint32_t* cols,
                                    const uint32_t* L, int threads) {
  uint64_t T = 0;
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for num_threads(threads) schedule(dynamic, 64) reduction(+ : T)
  for (int64_t ui = 0; ui < (int64_t)n; ++ui) {
    uint32_t u = (uint32_t)ui;
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = cols[e];
      if (L[u] == L[v] && u < v) T += cover_edge_count(off, cols, L, u, v);
    }
  }
  return T;
}

OR_EXPORT uint64_t or_plain_count_mt(uint32_t n, const int64_t* off, const uint32_t* cols,
                                     int threads) {
  uint64_t T = 0;
  if (threads <= 0) threads = omp_get_max_threads();
#pragma omp parallel for num_threads(threads) schedule(dynamic, 64) reduction(+ : T)
  for (int64_t ui = 0; ui < (int64_t)n; ++ui) {
    uint32_t u = (uint32_t)ui;
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = cols[e];
      if (u < v) T += plain_edge_count(off, cols, u, v);
    }
  }
  return T;
}

/* Per-edge counts of Alg. 1 for every cover edge, in H's ascending (u, v)
 * order: hstart[u] is the index in H of u's first cover edge (an exclusive
 * prefix sum of the per-vertex cover-edge counts, computed here), so each
 * thread writes the counts of its own rows.  At most cap counts are
 * written; returns |H| (-1 if out of host memory). */
OR_EXPORT int64_t or_cetc_all_edge_counts_mt(uint32_t n, const int64_t* off,
                                             const uint32_t* cols, const uint32_t* L,
                                             uint32_t* counts, int64_t cap, int threads) {
  if (threads <= 0) threads = omp_get_max_threads();
  int64_t* hstart = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!hstart) return -1;
  hstart[0] = 0;
  for (uint32_t u = 0; u < n; ++u) {
    int64_t k = 0;
    for (int64_t e = off[u]; e < off[u + 1]; ++e)
      if (u < cols[e] && L[u] == L[cols[e]]) ++k;
    hstart[u + 1] = hstart[u] + k;
  }
#pragma omp parallel for num_threads(threads) schedule(dynamic, 64)
  for (int64_t ui = 0; ui < (int64_t)n; ++ui) {
    uint32_t u = (uint32_t)ui;
    int64_t h = hstart[u];
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = cols[e];
      if (u < v && L[u] == L[v]) {
        if (h < cap) counts[h] = (uint32_t)cover_edge_count(off, cols, L, u, v);
        ++h;
      }
    }
  }
  int64_t total = hstart[n];
  free(hstart);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Triangle finding (abstract; Sec. VI): every triangle {a < b < c} listed
 * once, in ascending (a, b, c) order.  Writes at most cap triples; returns
 * the number of triangles. */
OR_EXPORT int64_t or_triangles(uint32_t n, const int64_t* off, const uint32_t* cols,
                               uint32_t* abc, int64_t cap) {
  int64_t t = 0;
  for (uint32_t a = 0; a < n; ++a) {
    for (int64_t e = off[a]; e < off[a + 1]; ++e) {
      uint32_t b = cols[e];
      if (b <= a) continue;
      int64_t i = off[a], iend = off[a + 1];
      int64_t j = off[b], jend = off[b + 1];
      while (i < iend && j < jend) {
        uint32_t x = cols[i], y = cols[j];
        if (x < y) ++i;
        else if (y < x) ++j;
        else {
          if (x > b) {
            if (abc && t < cap) { abc[3 * t] = a; abc[3 * t + 1] = b; abc[3 * t + 2] = x; }
            ++t;
          }
          ++i; ++j;
        }
      }
    }
  }
  return t;
}

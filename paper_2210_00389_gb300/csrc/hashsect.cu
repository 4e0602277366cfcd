// Owner-grouped hash intersection: bucketing (a3), intersection with the
// count-once rule (a4) and reduction (a5) for both the cover path and the
// plain all-edge path.
//
// For an edge (u, v), u < v, the endpoint of larger degree is the "owner" o
// and the other the "probe" p.  The intersection is counted by looking up
// p's relevant neighbours in a hash table of N(o) (hashing-based
// intersection, Sec. V-A of Bader et al., "Triangle Counting Through
// Cover-Edges"; the paper's compute bound for the cover edges, Sec. III,
// charges expected O(1) per search with a hash table).  The work is about
// sum over edges of min(d(u), d(v)) lookups instead of d(u) + d(v) merge
// steps.
//
//   cover: p's level segments (segment.cu) N_{l-1}(p), the same-level ids
//          above v and N_{l+1}(p), so every hit satisfies the count-once
//          rule of Alg. 1 / Thm. 2 (L(w) != l, or L(w) = l and w > v).
//   plain: p's neighbours above v; every hit is an apex w > v.
//
// In both cases the probe elements form at most two contiguous runs of one
// row array, R1 = [base, base + x) and R2 = [base + cut, base + end)
// (cover: R1 = level l-1, R2 = same level above v followed by level l+1,
// which are adjacent in the segmented row), stored as a 16-byte descriptor
// per edge by the bucketing step.  R1 is sorted; for cover, R2 is two
// sorted pieces split at base + z (z kept in a side array, used only by
// windowed owners, which need sorted runs).
//
// Bucketing (a3) is a counting sort of the edges by owner.  Owners of degree
// <= kSmallOwner keep the warp merge of intersect.cu.  Every other owner is
// split into work items (owner, slot) of about item_work lookups; a CTA
// takes an item, builds a two-choice (cuckoo) hash table of N(o) in shared
// memory (the CTA's whole table, at most 2/5 full; two independent 4-byte
// shared loads per lookup) and its warps take the item's edges from a
// shared counter.
// Owners of degree <= kMediumMax use 256-thread CTAs with 28 KB tables (seven
// per SM); larger owners use 1024-thread CTAs with 224 KB tables.  Rows
// longer than a window (kBigWin entries) are processed in windows of
// consecutive entries (an id range); every probe run keeps a cursor across
// windows, so each probe element is looked up once.
#include <algorithm>

#include "internal.cuh"

namespace tc {

constexpr uint32_t kSmallOwner = 64;              // owners this small use the merge
constexpr uint32_t kMediumMax = 2048;             // larger owners use the big tables
// Lookups per work item, per mode (cover, plain): the step's total lookups
// over (SMs x kItemsPerSM), clamped to [kItemMin, kItemMax].  Larger items
// rebuild fewer tables, smaller ones balance better, and the best size grows
// with the graph (measured on R-MAT scale 22 and 26 and Chung-Lu 2^23: cover
// 2^21 .. 2^22 at scale 22, 2^23 at scale 26; plain 2^20 and 2^21).
constexpr unsigned long long kItemMin[2] = {1ull << 21, 1ull << 20};
constexpr unsigned long long kItemMax[2] = {1ull << 23, 1ull << 21};
constexpr unsigned long long kItemsPerSM[2] = {64, 128};

__device__ __forceinline__ unsigned long long item_work_of(const unsigned long long* ctrl,
                                                           unsigned long long lo,
                                                           unsigned long long hi,
                                                           unsigned long long div) {
  const unsigned long long w = ctrl[kCtrlWorkSum] / div;
  return w < lo ? lo : (w > hi ? hi : w);
}
constexpr unsigned long long kBuildRatio = 4;     // hash an owner only if lookups >= 4 d(o)
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

enum { kModeCover = 0, kModePlain = 1 };

struct EdgeSrc {
  // cover: H pairs + segment data; plain: COO rows + upper starts
  const uint2* H;
  const unsigned long long* hoff;
  const uint4* seg;
  const uint32_t* erow;
  const int64_t* ustart;
  const int64_t* off;
  const uint32_t* cols;
  uint64_t first;  // edge index of local index 0 (a shard's first edge)
};

// Cover edges on level 1: both endpoints' only lower-level neighbour is
// their component's root (level 0 holds only roots), so the root is a
// common neighbour on another level -- one that Alg. 1's predicate counts
// -- and the level l-1 run needs no lookup.  The descriptor marks such an
// edge with this bit in its run-0 length (the run itself left empty) and
// the kernel adds the root's one.
constexpr uint32_t kRootBonus = 0x80000000u;

// Decode edge `idx`: returns false for plain entries that are not u < v.
template <int M>
__device__ __forceinline__ bool edge_at(const EdgeSrc& s, uint64_t idx, uint32_t& u, uint32_t& v) {
  if (M == kModeCover) {
    const uint2 e = s.H[idx];
    u = e.x;
    v = e.y;
    return true;
  } else {
    u = s.erow[idx];
    v = s.cols[idx];
    return u < v;
  }
}

__device__ __forceinline__ uint32_t degree(const int64_t* off, uint32_t x) {
  return (uint32_t)(off[x + 1] - off[x]);
}

// Owner = endpoint of larger degree (u on ties).
__device__ __forceinline__ void owner_probe(const int64_t* off, uint32_t u, uint32_t v,
                                            uint32_t& o, uint32_t& p, uint32_t& dout) {
  const uint32_t du = degree(off, u), dv = degree(off, v);
  if (dv > du) { o = v; p = u; dout = dv; } else { o = u; p = v; dout = du; }
}

// Probe descriptor {base, x, cut, end}: runs [base, base+x) and
// [base+cut, base+end) of the probe row array (scols for cover, cols for
// plain).
template <int M>
__device__ __forceinline__ uint4 probe_desc(const EdgeSrc& s, uint64_t idx, uint32_t u, uint32_t v,
                                            uint32_t p, uint32_t* split = nullptr) {
  if (M == kModeCover) {
    const int64_t op = s.off[p];
    const uint32_t dp = (uint32_t)(s.off[p + 1] - op);
    const uint4 sg = s.seg[p];
    if (split) *split = sg.z;  // start of level l+1: where R2's two sorted pieces meet
    // same-level ids of p above v: for p = v the run starts at sg.y; for
    // p = u, v is entry (idx - hoff[u]) of u's run above u
    const uint32_t cut = (p == v) ? sg.y : sg.y + (uint32_t)(idx - s.hoff[u]) + 1u;
    // sg.w = L(p)
    return make_uint4((uint32_t)op, sg.w == 1u ? kRootBonus : sg.x, cut, dp);
  } else {
    const int64_t b = (p == u) ? (int64_t)idx + 1 : s.ustart[v];  // neighbours of p above v
    const uint4 d = make_uint4((uint32_t)b, 0u, 0u, (uint32_t)(s.off[p + 1] - b));
    if (split) *split = d.w;
    return d;
  }
}

__device__ __forceinline__ uint32_t desc_work(uint4 d) {
  return (d.y & ~kRootBonus) + (d.w - d.z);
}

// ------------------------------------------------------------------ bucketing

// Per edge: owners of degree <= kSmallOwner go to the small list, others
// are counted per owner with their lookup work.
template <int M>
__global__ void k_bucket_count(EdgeSrc s, uint64_t nidx, uint32_t* __restrict__ owner_cnt,
                               unsigned long long* __restrict__ owner_work,
                               uint32_t* __restrict__ small_list, unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long wsum = 0;  // this thread's share of the total lookups
  for (; base < nidx; base += stride) {
    const uint64_t idx = base + lane, gi = s.first + idx;
    bool small = false;
    uint32_t key = kEmpty, work = 0;  // owner of a hashed edge, its lookups + 1
    if (idx < nidx) {
      uint32_t u, v;
      if (edge_at<M>(s, gi, u, v)) {
        uint32_t o, p, dout;
        owner_probe(s.off, u, v, o, p, dout);
        if (dout <= kSmallOwner) {
          small = true;
        } else {
          key = o;
          work = desc_work(probe_desc<M>(s, gi, u, v, p)) + 1u;
          wsum += work;
        }
      }
    }
    // lanes with the same owner (consecutive edges often share one) add
    // their counts with one atomic per owner
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    if (key != kEmpty) {
      // 16-bit halves, so the sum of 32 values cannot wrap
      const unsigned hi = __reduce_add_sync(peers, work >> 16);
      const unsigned lo = __reduce_add_sync(peers, work & 0xFFFFu);
      if (lane == __ffs(peers) - 1) {
        atomicAdd(&owner_cnt[key], (uint32_t)__popc(peers));
        atomicAdd(&owner_work[key], ((unsigned long long)hi << 16) + lo);
      }
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, small);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long b0 = 0;
      if (lane == leader) b0 = atomicAdd(&ctrl[kCtrlQ0], (unsigned long long)__popc(m));
      b0 = __shfl_sync(0xFFFFFFFFu, b0, leader);
      if (small) small_list[b0 + __popc(m & ((1u << lane) - 1u))] = (uint32_t)gi;
    }
  }
  // the block's total lookups: one atomic per block
  __shared__ unsigned long long red[32];
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_down_sync(0xFFFFFFFFu, wsum, o);
  if (lane == 0) red[threadIdx.x >> 5] = wsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    if (t) atomicAdd(&ctrl[kCtrlWorkSum], t);
  }
}

// An owner is hashed only if its edges bring at least kBuildRatio lookups
// per table entry; the edges of other owners join the merge list.
__device__ __forceinline__ bool owner_hashed(unsigned long long work, uint32_t d) {
  return work >= kBuildRatio * (unsigned long long)d;
}

// Scatter every hashed edge's descriptor (and its index, for per-edge
// counts) into its owner's task range; edges of owners too light to hash
// are appended to the merge list.  ostart[o] is the owner's cursor: its
// first task index, advanced here by one per edge (k_item_write puts it
// back), with bit kLightBit set by k_item_counts for owners too light to
// hash -- one atomic per owner and warp both places an edge and tells
// whether it is hashed, with no other per-owner read.
constexpr unsigned long long kLightBit = 1ull << 63;

template <int M>
__global__ void k_bucket_scatter(EdgeSrc s, uint64_t nidx, unsigned long long* __restrict__ ostart,
                                 uint4* __restrict__ descs, uint32_t* __restrict__ task_split,
                                 uint32_t* __restrict__ task_idx, uint32_t* __restrict__ small_list,
                                 unsigned long long* ctrl) {
  const int lane = threadIdx.x & 31;
  uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (; base < nidx; base += stride) {
    const uint64_t idx = base + lane, gi = s.first + idx;
    bool light = false;
    uint32_t u, v, o = 0, p = 0, key = kEmpty;
    if (idx < nidx && edge_at<M>(s, gi, u, v)) {
      uint32_t dout;
      owner_probe(s.off, u, v, o, p, dout);
      if (dout > kSmallOwner) key = o;
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    if (key != kEmpty) {
      // the descriptor's loads go out before the cursor atomic returns
      uint32_t z;
      const uint4 d = probe_desc<M>(s, gi, u, v, p, &z);
      const int leader = __ffs(peers) - 1;
      unsigned long long c0 = 0;
      if (lane == leader) c0 = atomicAdd(&ostart[key], (unsigned long long)__popc(peers));
      c0 = __shfl_sync(peers, c0, leader);
      if (c0 & kLightBit) {
        light = true;
      } else {
        const unsigned long long t = c0 + __popc(peers & ((1u << lane) - 1u));
        descs[t] = d;
        task_split[t] = z;
        if (task_idx) task_idx[t] = (uint32_t)gi;
      }
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, light);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long b0 = 0;
      if (lane == leader) b0 = atomicAdd(&ctrl[kCtrlQ0], (unsigned long long)__popc(m));
      b0 = __shfl_sync(0xFFFFFFFFu, b0, leader);
      if (light) small_list[b0 + __popc(m & ((1u << lane) - 1u))] = (uint32_t)gi;
    }
  }
}
// Slots per owner: about item_work lookups per item, and at least 4 lookups
// per table entry built (each item builds N(o)'s table).
__device__ __forceinline__ uint32_t owner_slots(uint32_t cnt, unsigned long long work, uint32_t d,
                                                unsigned long long item_work) {
  if (cnt == 0 || !owner_hashed(work, d)) return 0;
  const unsigned long long s1 = (work + item_work - 1) / item_work;
  const unsigned long long s2 = work / (4ull * d);
  unsigned long long s = s1 < s2 ? s1 : s2;
  const unsigned long long cap = (cnt + 3) / 4;
  if (s > cap) s = cap;
  if (s < 1) s = 1;
  if (s > 65535) s = 65535;
  return (uint32_t)s;
}

// Owners of degree <= kMediumMax go to the 256-thread kernel with small
// tables, larger ones to the 1024-thread kernel with large tables.
__device__ __forceinline__ int owner_class(uint32_t d) { return d > kMediumMax ? 1 : 0; }

// Per owner: its slot count; totals per class in ctrl[kCtrlItems + class].
// Owners with edges that are too light to hash get kLightBit in ostart.
__global__ void k_item_counts(const int64_t* __restrict__ off, uint32_t n,
                              const uint32_t* __restrict__ owner_cnt,
                              const unsigned long long* __restrict__ owner_work,
                              unsigned long long item_lo, unsigned long long item_hi,
                              unsigned long long item_div, unsigned long long* ctrl,
                              unsigned long long* __restrict__ ostart) {
  const unsigned long long item_work = item_work_of(ctrl, item_lo, item_hi, item_div);
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long t[2] = {0ull, 0ull};
  for (; o < (int64_t)n; o += stride) {
    const uint32_t d = degree(off, (uint32_t)o);
    const uint32_t cnt = owner_cnt[o];
    if (cnt == 0) continue;
    const unsigned long long w = owner_work[o];
    if (!owner_hashed(w, d)) ostart[o] |= kLightBit;
    t[owner_class(d)] += owner_slots(cnt, w, d, item_work);
  }
  for (int c = 0; c < 2; ++c) {
    unsigned long long x = t[c];
    for (int k = 16; k > 0; k >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, k);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&ctrl[kCtrlItems + c], x);
  }
}

// items of class c at items_c[atomic cursor]: (owner, slot << 16 | slots).
// Runs after the scatter, which advanced every hashed owner's start by its
// edge count; the start is put back here.
__global__ void k_item_write(const int64_t* __restrict__ off, uint32_t n,
                             const uint32_t* __restrict__ owner_cnt,
                             const unsigned long long* __restrict__ owner_work,
                             unsigned long long item_lo, unsigned long long item_hi,
                             unsigned long long item_div, const unsigned long long* ctrl,
                             uint2* __restrict__ items0, uint2* __restrict__ items1,
                             unsigned long long* cursors, unsigned long long* __restrict__ ostart) {
  const unsigned long long item_work = item_work_of(ctrl, item_lo, item_hi, item_div);
  int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; o < (int64_t)n; o += stride) {
    const uint32_t d = degree(off, (uint32_t)o);
    const uint32_t cnt = owner_cnt[o];
    const uint32_t s = owner_slots(cnt, owner_work[o], d, item_work);
    if (s == 0) continue;
    ostart[o] -= cnt;
    const int c = owner_class(d);
    const unsigned long long b = atomicAdd(&cursors[c], (unsigned long long)s);
    uint2* items = c ? items1 : items0;
    for (uint32_t k = 0; k < s; ++k) items[b + k] = make_uint2((uint32_t)o, (k << 16) | s);
  }
}

__global__ void k_u32_to_u64(const uint32_t* __restrict__ a, uint32_t n, unsigned long long* b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < (int64_t)n; i += stride) b[i] = a[i];
}

// ------------------------------------------------------------------ hashing

// Two-choice (cuckoo) table of 2 nh 4-byte slots in shared memory: key w
// lives either in slot h1(w) of the first half or in slot nh + h2(w) of the
// second (Pagh and Rodler's cuckoo hashing, two tables).  A lookup reads
// both slots -- two independent 4-byte shared loads, two compares, no
// probe loop -- so it holds three registers per key in flight, and a warp's
// reads of 32 random words cost far fewer shared-memory wavefronts than 16-
// byte bucket reads.  h1, h2: multiply-high of two multiplicative hashes
// (Knuth's 2^32/phi and another odd constant; Lemire's range map), so nh
// need not be a power of two.
__device__ __forceinline__ uint32_t slot1(uint32_t w, uint32_t nh) {
  return __umulhi(w * 0x9E3779B1u, nh);
}
__device__ __forceinline__ uint32_t slot2(uint32_t w, uint32_t nh) {
  return nh + __umulhi(w * 0x85EBCA77u, nh);
}

// Insertion moves keys between their two slots (atomicExch chains, any
// number of threads at once: every key is always in the table or held by
// exactly one thread).  A chain longer than kMaxKicks gives up and returns
// false: the key it holds is lost, and the caller rebuilds the table with a
// smaller window.  At the loads used here (at most 2/5 of the slots) that
// is very rare; a window of one key always fits.
constexpr int kMaxKicks = 64;

__device__ __forceinline__ bool table_insert(uint32_t* tab, uint32_t nh, uint32_t w) {
  uint32_t pos = slot1(w, nh);
  for (int it = 0; it < kMaxKicks; ++it) {
    const uint32_t old = atomicExch(&tab[pos], w);
    if (old == kEmpty) return true;
    w = old;  // the displaced key moves to its other slot
    pos = pos < nh ? slot2(w, nh) : slot1(w, nh);
  }
  return false;
}

// Warp-uniform: all 32 lanes call it, each with U keys (valid[j] = false on
// padding: such a key reads nothing and never hits).  All 2U slot reads are
// issued together.  Returns the lane's hits; sink(w) is called on each
// (NoSink: nothing, for the counts).
struct NoSink {
  __device__ __forceinline__ void operator()(uint32_t) const {}
};

// Per-vertex triangle counts: one for the apex of every hit.
struct ApexSink {
  unsigned long long* tv;
  __device__ __forceinline__ void operator()(uint32_t w) const { atomicAdd(&tv[w], 1ull); }
};

template <int U, class Sink = NoSink>
__device__ __forceinline__ unsigned table_find_n(const uint32_t* tab, uint32_t nh,
                                                 const uint32_t (&w)[U], const bool (&valid)[U],
                                                 Sink sink = Sink()) {
  uint32_t a[U], b[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    a[j] = valid[j] ? tab[slot1(w[j], nh)] : kEmpty;
    b[j] = valid[j] ? tab[slot2(w[j], nh)] : kEmpty;
  }
  bool hit[U];
  unsigned c = 0;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    hit[j] = valid[j] && (a[j] == w[j] || b[j] == w[j]);
    c += hit[j] ? 1u : 0u;
  }
#pragma unroll
  for (int j = 0; j < U; ++j)
    if (hit[j]) sink(w[j]);
  return c;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  return x;
}

constexpr int kUnroll = 4;  // probe loads in flight per lane

constexpr uint32_t kGroup = 32 * kUnroll;  // probe elements a warp looks up at once

// U rounds of the remainder index space [0, tt) from k0: element k is
// R0[k] below s1, R1[k] below s2, else R2[k] (R1, R2 pre-offset).
template <int U, class Sink = NoSink>
__device__ __forceinline__ unsigned probe_tail(const uint32_t* __restrict__ R0,
                                               const uint32_t* __restrict__ R1,
                                               const uint32_t* __restrict__ R2, uint32_t s1,
                                               uint32_t s2, uint32_t tt, uint32_t k0,
                                               const uint32_t* tab, uint32_t nh,
                                               Sink sink = Sink()) {
  const int lane = threadIdx.x & 31;
  uint32_t w[U];
  bool ok[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const uint32_t k = k0 + j * 32 + lane;
    ok[j] = k < tt;
    w[j] = ok[j] ? __ldg((k < s1 ? R0 : (k < s2 ? R1 : R2)) + k) : kEmpty;
  }
  return table_find_n<U>(tab, nh, w, ok, sink);
}

// Look up every element of up to three ranges Q[i][0, m[i]): the full
// groups of each range without per-element tests, then the ranges'
// remainders together as one index space, in groups of U rounds while
// more than two rounds are left, then one or two rounds (a short remainder
// does not pay for a whole group).  U: probe loads per lane and group.
template <int U = kUnroll, class Sink = NoSink>
__device__ __forceinline__ unsigned probe_ranges(const uint32_t* Q0, uint32_t m0,
                                                 const uint32_t* Q1, uint32_t m1,
                                                 const uint32_t* Q2, uint32_t m2,
                                                 const uint32_t* tab, uint32_t nh,
                                                 Sink sink = Sink()) {
  constexpr uint32_t kG = 32u * U;  // elements per group
  const uint32_t g0 = m0 / kG, g1 = m1 / kG, g2 = m2 / kG;
  const uint32_t g01 = g0 + g1, ng = g01 + g2;
  unsigned c = 0;
  if (ng > 0) {
    const int lane = threadIdx.x & 31;
    auto group_ptr = [&](uint32_t g) {
      return g < g0 ? Q0 + g * kG
                    : (g < g01 ? Q1 + (g - g0) * kG : Q2 + (g - g01) * kG);
    };
    bool ok[U];
#pragma unroll
    for (int j = 0; j < U; ++j) ok[j] = true;
    uint32_t cur[U], nxt[U];
    {
      const uint32_t* gp = group_ptr(0);
#pragma unroll
      for (int j = 0; j < U; ++j) cur[j] = __ldg(gp + j * 32 + lane);
    }
    for (uint32_t g = 1; g < ng; ++g) {
      const uint32_t* gp = group_ptr(g);
#pragma unroll
      for (int j = 0; j < U; ++j) nxt[j] = __ldg(gp + j * 32 + lane);
      c += table_find_n<U>(tab, nh, cur, ok, sink);
#pragma unroll
      for (int j = 0; j < U; ++j) cur[j] = nxt[j];
    }
    c += table_find_n<U>(tab, nh, cur, ok, sink);
  }
  const uint32_t f0 = g0 * kG, f1 = g1 * kG, f2 = g2 * kG;
  const uint32_t r0 = m0 - f0, s1 = r0 + (m1 - f1), tt = s1 + (m2 - f2);
  const uint32_t* R0 = Q0 + f0;
  const uint32_t* R1 = Q1 + f1 - r0;
  const uint32_t* R2 = Q2 + f2 - s1;
  uint32_t k0 = 0;
  for (; k0 + 64 < tt; k0 += kG)
    c += probe_tail<U>(R0, R1, R2, r0, s1, tt, k0, tab, nh, sink);
  if (k0 + 32 < tt) c += probe_tail<2>(R0, R1, R2, r0, s1, tt, k0, tab, nh, sink);
  else if (k0 < tt) c += probe_tail<1>(R0, R1, R2, r0, s1, tt, k0, tab, nh, sink);
  return c;
}

// Asks L2 to fetch elements [kGroup, len) of the run R (at most kPrefetchMax
// bytes): one bulk prefetch, issued by one lane, with no registers held
// while it is in flight.  The range is shrunk to 16-byte boundaries inside
// the run, so it never leaves the array.
constexpr uint32_t kPrefetchMax = 32768;
__device__ __forceinline__ void prefetch_run_l2(const uint32_t* R, uint32_t len) {
  if (len <= kGroup + 8u) return;
  const uintptr_t a = ((uintptr_t)(R + kGroup) + 15u) & ~(uintptr_t)15u;
  uintptr_t e = (uintptr_t)(R + len) & ~(uintptr_t)15u;
  if (e > a + kPrefetchMax) e = a + kPrefetchMax;
  if (e <= a) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a))
               : "memory");
}

// All probe elements of a descriptor: runs [0, x) and [cut, end) of P.
template <int U = kUnroll, class Sink = NoSink>
__device__ __forceinline__ unsigned probe_all(const uint32_t* __restrict__ P, uint4 ds,
                                              const uint32_t* tab, uint32_t nh,
                                              Sink sink = Sink()) {
  return probe_ranges<U>(P, ds.y, P + ds.z, ds.w - ds.z, P, 0u, tab, nh, sink);
}

// This window's part of the sorted run P[a, b) -- its elements <= hi, from
// a on -- looked up with the window bound checked on the loads the lookups
// use.  A group of kG elements whose last element is inside the run
// and <= hi is wholly in the window (the run is sorted) and is looked up
// without masks; the first group that is not ends the pass, its elements
// above hi (or past b) masked out, and the set mask bits (a prefix) are
// the elements it took.  *m = the number of elements looked up.
template <int U = kUnroll, class Sink = NoSink>
__device__ __forceinline__ unsigned probe_window_run(const uint32_t* __restrict__ P, uint32_t a,
                                                     uint32_t b, uint32_t hi,
                                                     const uint32_t* tab, uint32_t nh,
                                                     uint32_t& m, Sink sink = Sink()) {
  constexpr uint32_t kG = 32u * U;
  const int lane = threadIdx.x & 31;
  unsigned c = 0;
  uint32_t k = a;
  bool all[U];
#pragma unroll
  for (int j = 0; j < U; ++j) all[j] = true;
  while (k < b) {
    uint32_t w[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint32_t i = k + j * 32 + lane;
      w[j] = i < b ? __ldg(P + i) : kEmpty;  // kEmpty > hi
    }
    const uint32_t last = __shfl_sync(0xFFFFFFFFu, w[U - 1], 31);
    if (last <= hi) {  // the whole group: inside the run and the window
      c += table_find_n<U>(tab, nh, w, all, sink);
      k += kG;
      continue;
    }
    bool ok[U];
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      ok[j] = w[j] <= hi;
      cnt += (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, ok[j]));
    }
    c += table_find_n<U>(tab, nh, w, ok, sink);
    k += cnt;
    break;
  }
  m = k - a;
  return c;
}

constexpr uint32_t kBatchMaxWork = 64;  // tasks with fewer lookups share a warp pass

// The medium-owner kernel's block size and probe loads per lane (the large-
// owner kernel uses kUnroll).
constexpr int kMedThreadsK = 256;
constexpr int kMedUnroll = 2;

// Up to 32 tasks t0 .. t0+nt-1 at once: lane j holds task j's descriptor.
// Tasks with fewer than kBatchMaxWork lookups are laid end to end in one
// index space; each lane finds the task of its position by bisection over
// the warp's inclusive prefix sums (shuffles) and looks the element up.
// Larger tasks are then done one at a time by the whole warp.  Counts only
// (no per-edge or per-vertex output).
__device__ __forceinline__ unsigned probe_batch(const uint32_t* __restrict__ pcols,
                                                const uint4* __restrict__ descs, uint64_t t0,
                                                uint32_t nt, const uint32_t* tab, uint32_t nh,
                                                unsigned long long* probes) {
  const int lane = threadIdx.x & 31;
  uint4 ds = (uint32_t)lane < nt ? descs[t0 + lane] : make_uint4(0u, 0u, 0u, 0u);
  // a level-1 cover edge's shared root: one, counted by its lane
  unsigned c = (ds.y & kRootBonus) ? 1u : 0u;
  ds.y &= ~kRootBonus;
  const uint32_t w = desc_work(ds);
  const bool small = w < kBatchMaxWork;
  uint32_t s = small ? w : 0u;  // inclusive prefix of the small tasks' work
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
    if (lane >= o) s += y;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, s, 31);
  const uint32_t excl = s - (small ? w : 0u);
  const uint32_t xr = ds.y, shift2 = ds.z - ds.y;
  for (uint32_t k0 = 0; k0 < total; k0 += 32 * kUnroll) {
    uint32_t e[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) {
      const uint32_t g = k0 + j * 32 + lane;
      // q = number of prefix values <= g = the task holding position g
      int q = 0;
#pragma unroll
      for (int st = 16; st > 0; st >>= 1) {
        const uint32_t sv = __shfl_sync(0xFFFFFFFFu, s, q + st - 1);
        if (sv <= g) q += st;
      }
      const uint32_t base = __shfl_sync(0xFFFFFFFFu, ds.x, q);
      const uint32_t xq = __shfl_sync(0xFFFFFFFFu, xr, q);
      const uint32_t sq = __shfl_sync(0xFFFFFFFFu, shift2, q);
      const uint32_t eq = __shfl_sync(0xFFFFFFFFu, excl, q);
      const uint32_t loc = g - eq;
      e[j] = g < total ? __ldg(pcols + base + (loc < xq ? loc : loc + sq)) : kEmpty;
    }
    bool ok[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; ++j) ok[j] = e[j] != kEmpty;
    c += table_find_n<kUnroll>(tab, nh, e, ok);
  }
  if (lane == 0) *probes += total;
  unsigned big = __ballot_sync(0xFFFFFFFFu, (uint32_t)lane < nt && !small);
  while (big) {
    const int j = __ffs(big) - 1;
    big &= big - 1;
    uint4 dj;
    dj.x = __shfl_sync(0xFFFFFFFFu, ds.x, j);
    dj.y = __shfl_sync(0xFFFFFFFFu, ds.y, j);
    dj.z = __shfl_sync(0xFFFFFFFFu, ds.z, j);
    dj.w = __shfl_sync(0xFFFFFFFFu, ds.w, j);
    c += probe_all(pcols + dj.x, dj, tab, nh);
    if (lane == 0) *probes += desc_work(dj);
  }
  return c;
}

// VERT (cover mode only): per-vertex triangle counts instead of per-edge
// ones -- every hit adds one to its apex, and each edge's count is added to
// both of its endpoints (H[task_idx[t]]).
template <int M, int THREADS, int SLOTS, int WIN, int MINB, bool BATCH, bool VERT>
__global__ void __launch_bounds__(THREADS, MINB)
k_hash_intersect(const int64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                 const uint32_t* __restrict__ pcols, const uint2* __restrict__ items,
                 uint64_t nitems, const unsigned long long* __restrict__ ostart,
                 const uint32_t* __restrict__ owner_cnt, const uint4* __restrict__ descs,
                 const uint32_t* __restrict__ task_split, const uint32_t* __restrict__ task_idx,
                 uint4* __restrict__ cursors, uint32_t* __restrict__ per_edge,
                 const uint2* __restrict__ H, unsigned long long* __restrict__ tv,
                 unsigned long long* ctrl) {
  constexpr int kWarps = THREADS / 32;
  // probe loads per lane and group: medium owners' probe runs are a few
  // hundred elements, so groups of 64 waste fewer lanes in their tails
  constexpr int U = THREADS == kMedThreadsK ? kMedUnroll : kUnroll;
  constexpr uint32_t kWin = WIN;          // owner entries per table window (at most)
  constexpr uint32_t kHalf = SLOTS / 2;   // slots per half of the two-choice table
  extern __shared__ uint4 tab4[];         // SLOTS slots (dynamic shared memory)
  __shared__ unsigned long long s_next;
  __shared__ int s_fail;
  uint32_t* tab = reinterpret_cast<uint32_t*>(tab4);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long acc = 0, probes = 0;
  // one item per CTA (grid-stride only beyond the grid limit): CTAs end
  // between items, so work of higher-priority streams gets SMs as they free
  for (uint64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const uint2 item = items[it];
    const uint32_t o = item.x, slot = item.y >> 16, nsl = item.y & 0xFFFFu;
    const uint64_t T0 = ostart[o], T = owner_cnt[o];
    const uint64_t ta = T0 + T * slot / nsl, tb = T0 + T * (slot + 1) / nsl;
    const int64_t ro = off[o];
    const uint32_t d = (uint32_t)(off[o + 1] - ro);
    // windows of consecutive entries of N(o) (an id range each), at most
    // kWin long; a window whose table cannot be built is halved
    for (uint32_t wb = 0; wb < d;) {
      uint32_t we = min(d, wb + kWin);
      while (true) {
        for (uint32_t k = threadIdx.x; k < SLOTS / 4; k += THREADS)
          tab4[k] = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
        if (threadIdx.x == 0) {
          s_next = ta;
          s_fail = 0;
        }
        __syncthreads();
        bool ok = true;
        for (uint32_t k = wb + threadIdx.x; k < we; k += THREADS)
          ok &= table_insert(tab, kHalf, cols[ro + k]);
        if (!ok) s_fail = 1;
        __syncthreads();
        // a one-key window always fits (its first slot is empty), so the
        // second test only bounds the loop
        if (!s_fail || we - wb <= 1) break;
        we = wb + (we - wb) / 2;
        __syncthreads();  // every thread has read s_fail before it is reset
      }
      const bool whole = wb == 0 && we == d;
      const uint32_t hi = we == d ? kEmpty - 1u : cols[ro + we - 1];
      if (BATCH && whole && per_edge == nullptr) {
        // warps take 32 edges at a time and share passes over short lists
        while (true) {
          unsigned long long t = 0;
          if (lane == 0) t = atomicAdd(&s_next, 32ull);
          t = __shfl_sync(0xFFFFFFFFu, t, 0);
          if (t >= tb) break;
          const uint32_t nt = (uint32_t)min((unsigned long long)32, tb - t);
          acc += probe_batch(pcols, descs, t, nt, tab, kHalf, &probes);
        }
      } else {
        // each warp holds its next task and that task's descriptor in flight
        // while it works on the current one
        auto grab = [&]() {
          unsigned long long t = 0;
          if (lane == 0) t = atomicAdd(&s_next, 1ull);
          return __shfl_sync(0xFFFFFFFFu, t, 0);
        };
        unsigned long long t = grab();
        uint4 ds = t < tb ? descs[t] : make_uint4(0u, 0u, 0u, 0u);
        while (t < tb) {
          const unsigned long long tn = grab();
          const uint4 dn = tn < tb ? descs[tn] : make_uint4(0u, 0u, 0u, 0u);
          const uint32_t* P = pcols + ds.x;
          const bool bonus = (ds.y & kRootBonus) != 0u;
          ds.y &= ~kRootBonus;
          unsigned c;
          if (whole) {
            if (lane == 0) {
              prefetch_run_l2(P, ds.y);
              prefetch_run_l2(P + ds.z, ds.w - ds.z);
            }
            if constexpr (VERT) c = probe_all<U>(P, ds, tab, kHalf, ApexSink{tv});
            else c = probe_all<U>(P, ds, tab, kHalf);
            if (lane == 0) probes += desc_work(ds);
          } else {
            // three sorted runs: [0, x), [cut, z), [z, end), one cursor each
            const uint32_t z = task_split[t];
            uint4 cur = wb == 0 ? make_uint4(0u, ds.z, z, 0u) : cursors[t];
            // this window's elements of each run: the prefix <= hi
            uint32_t m0, m1, m2;
            if constexpr (VERT) {
              c = probe_window_run<U>(P, cur.x, ds.y, hi, tab, kHalf, m0, ApexSink{tv});
              c += probe_window_run<U>(P, cur.y, z, hi, tab, kHalf, m1, ApexSink{tv});
              c += probe_window_run<U>(P, cur.z, ds.w, hi, tab, kHalf, m2, ApexSink{tv});
            } else {
              c = probe_window_run<U>(P, cur.x, ds.y, hi, tab, kHalf, m0);
              c += probe_window_run<U>(P, cur.y, z, hi, tab, kHalf, m1);
              c += probe_window_run<U>(P, cur.z, ds.w, hi, tab, kHalf, m2);
            }
            if (lane == 0) {
              probes += m0 + m1 + m2;
              if (we < d) cursors[t] = make_uint4(cur.x + m0, cur.y + m1, cur.z + m2, 0u);
            }
          }
          if (bonus && wb == 0 && lane == 0) {
            c += 1u;  // the shared root, on level 0
            if constexpr (VERT) atomicAdd(&tv[P[0]], 1ull);
          }
          acc += c;
          if (per_edge) {
            const unsigned long long tsum = warp_sum_u64(c);
            if (lane == 0 && tsum) atomicAdd(&per_edge[task_idx[t]], (uint32_t)tsum);
          }
          if constexpr (VERT) {
            const unsigned long long tsum = warp_sum_u64(c);
            if (lane == 0 && tsum) {
              const uint2 e = H[task_idx[t]];
              atomicAdd(&tv[e.x], tsum);
              atomicAdd(&tv[e.y], tsum);
            }
          }
          t = tn;
          ds = dn;
        }
      }
      __syncthreads();
      wb = we;
    }
  }
  // block reduction of the count and the lookup total
  __shared__ unsigned long long red[2][kWarps];
  acc = warp_sum_u64(acc);
  probes = warp_sum_u64(probes);
  if (lane == 0) { red[0][wid] = acc; red[1][wid] = probes; }
  __syncthreads();
  if (wid == 0) {
    unsigned long long a = lane < kWarps ? red[0][lane] : 0ull;
    unsigned long long b = lane < kWarps ? red[1][lane] : 0ull;
    a = warp_sum_u64(a);
    b = warp_sum_u64(b);
    if (lane == 0) {
      if (a) atomicAdd(&ctrl[kCtrlCount], a);
      if (b) atomicAdd(&ctrl[kCtrlElems], b);
    }
  }
}

// Table configurations: medium owners (degree <= kMediumMax) in 256-thread
// CTAs with 28 KB tables (7,168 slots, at most 2/7 full), seven per SM at 32
// registers (two probe loads per lane; the plain kernel's batched passes
// spill 44 bytes there and are still faster); measured faster than five or
// six per SM with 32 KB tables and than eight with 24 KB at R-MAT scale 22
// and on Chung-Lu 2^23.  Large owners in 1024-thread CTAs with 224 KB
// tables (57,344 slots), one per SM.
constexpr int kMedThreads = kMedThreadsK, kMedSlots = 7168, kMedPerSM = 7;
constexpr int kBigThreads = 1024, kBigSlots = 57344, kBigPerSM = 1;
// Owner entries per table window, per mode (cover, plain): every owner row
// longer than this is processed in windows, and each window pass revisits
// all the owner's edges.  The two-choice table stays at most 2/5 full
// (windows of 22,936 measured faster than 19,104 and 14,336 on R-MAT scale
// 22 and 26 and Chung-Lu 2^23).
constexpr int kMedWin = (int)kMediumMax;
// Medium owners' edges with fewer than kBatchMaxWork lookups share warp
// passes (probe_batch) in plain mode, whose upper-neighbour probe lists are
// often that short; cover probe lists rarely are.  Measured on R-MAT scale
// 20 and 22.
constexpr bool kMedBatch[2] = {false, true};
constexpr int kBigWin[2] = {22936, 22936};
static_assert(3 * kMedWin <= kMedSlots && 5 * kBigWin[0] <= 2 * kBigSlots &&
                  5 * kBigWin[1] <= 2 * kBigSlots,
              "two-choice tables at most 2/5 full");
static_assert(kMedSlots % 8 == 0 && kBigSlots % 8 == 0, "tables in whole 16-byte halves");

template <int M, int THREADS, int SLOTS, int WIN, int MINB, bool BATCH, bool VERT = false>
static int launch_hash(tc_graph* g, const uint32_t* pcols, const uint2* items, uint64_t nitems,
                       const unsigned long long* ostart, const uint32_t* owner_cnt,
                       const uint4* descs, const uint32_t* task_split, const uint32_t* task_idx,
                       uint4* cursors, uint32_t* per_edge, unsigned long long* tv = nullptr) {
  if (nitems == 0) return TC_OK;
  cudaStream_t st = g->stream;
  const size_t smem = sizeof(uint32_t) * SLOTS;
  auto k = k_hash_intersect<M, THREADS, SLOTS, WIN, MINB, BATCH, VERT>;
  TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const uint64_t grid = std::min<uint64_t>(nitems, 0x7FFFFFFFull);
  launch(k, (unsigned)grid, THREADS, smem, st, g->off, g->cols, pcols, items, nitems, ostart,
         owner_cnt, descs, task_split, task_idx, cursors, per_edge, g->cover.p, tv, g->ctrl.p);
  TC_CUDA(cudaGetLastError());
  return TC_OK;
}

// ------------------------------------------------------------------ driver

// defined in intersect.cu: warp merge over a list of edge indices
int merge_small_edges(tc_graph* g, int mode, const uint32_t* list,
                      const unsigned long long* nlist_dev, uint64_t nlist_max,
                      const int64_t* ustart, uint32_t* per_edge);

// tv (cover mode, or NULL): per-vertex triangle counts are added to it
// instead of the count alone.
template <int M>
static int hash_count_mode(tc_graph* g, const EdgeSrc& s, uint64_t nidx, const uint32_t* pcols,
                           const int64_t* ustart, uint32_t* per_edge, unsigned long long* tv) {
  cudaStream_t st = g->stream;
  const int T = 256;
  DevBuf<uint32_t> owner_cnt, small_list, task_idx, task_split;
  DevBuf<unsigned long long> owner_work, ostart, counters;
  DevBuf<uint4> descs, cursors;
  DevBuf<uint2> items0, items1;
  TC_TRY(owner_cnt.alloc(g->n, st));
  TC_TRY(owner_work.alloc(g->n, st));
  TC_TRY(ostart.alloc(g->n, st));
  TC_TRY(small_list.alloc(nidx, st));
  TC_TRY(counters.alloc(4, st));
  TC_CUDA(cudaMemsetAsync(owner_cnt.p, 0, sizeof(uint32_t) * g->n, st));
  TC_CUDA(cudaMemsetAsync(owner_work.p, 0, sizeof(unsigned long long) * g->n, st));
  TC_CUDA(cudaMemsetAsync(counters.p, 0, 4 * sizeof(unsigned long long), st));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlQ0, 0, sizeof(unsigned long long), st));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlItems, 0, 2 * sizeof(unsigned long long), st));
  TC_CUDA(cudaMemsetAsync(g->ctrl.p + kCtrlWorkSum, 0, sizeof(unsigned long long), st));
  const unsigned long long item_div = (unsigned long long)sm_count() * kItemsPerSM[M];
  launch(k_bucket_count<M>, grid_for((int64_t)nidx, T, 16), T, 0, st, s, nidx, owner_cnt.p,
         owner_work.p, small_list.p, g->ctrl.p);
  launch(k_u32_to_u64, grid_for(g->n, T), T, 0, st, owner_cnt.p, g->n, ostart.p);
  TC_TRY(exclusive_scan_u64(ostart.p, g->n, g->ctrl.p + kCtrlTmp, st));
  launch(k_item_counts, grid_for(g->n, T), T, 0, st, g->off, g->n, owner_cnt.p, owner_work.p,
         kItemMin[M], kItemMax[M], item_div, g->ctrl.p, ostart.p);
  TC_CUDA(cudaGetLastError());
  TC_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl.p, kCtrlSlots * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, st));
  TC_CUDA(cudaStreamSynchronize(st));
  const uint64_t nsmall = g->ctrl_host[kCtrlQ0];
  const uint64_t ntasks = g->ctrl_host[kCtrlTmp];
  const uint64_t nitems0 = g->ctrl_host[kCtrlItems], nitems1 = g->ctrl_host[kCtrlItems + 1];
  TC_TRY(descs.alloc(ntasks, st));
  TC_TRY(cursors.alloc(ntasks, st));
  TC_TRY(task_split.alloc(ntasks, st));
  const bool need_idx = per_edge != nullptr || tv != nullptr;
  if (need_idx) TC_TRY(task_idx.alloc(ntasks, st));
  TC_TRY(items0.alloc(nitems0, st));
  TC_TRY(items1.alloc(nitems1, st));
  if (ntasks > 0) {
    launch(k_bucket_scatter<M>, grid_for((int64_t)nidx, T, 16), T, 0, st, s, nidx, ostart.p,
           descs.p, task_split.p, need_idx ? task_idx.p : (uint32_t*)nullptr, small_list.p,
           g->ctrl.p);
    launch(k_item_write, grid_for(g->n, T), T, 0, st, g->off, g->n, owner_cnt.p, owner_work.p,
           kItemMin[M], kItemMax[M], item_div, g->ctrl.p, items0.p, items1.p, counters.p,
           ostart.p);
  }
  TC_CUDA(cudaGetLastError());
  cudaEventRecord(g->ev[6], st);  // end of bucketing
  if constexpr (M == kModeCover) {
    if (tv) {
      TC_TRY((launch_hash<M, kBigThreads, kBigSlots, kBigWin[M], kBigPerSM, false, true>(
          g, pcols, items1.p, nitems1, ostart.p, owner_cnt.p, descs.p, task_split.p, task_idx.p,
          cursors.p, nullptr, tv)));
      TC_TRY((launch_hash<M, kMedThreads, kMedSlots, kMedWin, kMedPerSM, false, true>(
          g, pcols, items0.p, nitems0, ostart.p, owner_cnt.p, descs.p, task_split.p, task_idx.p,
          cursors.p, nullptr, tv)));
      // the merge list's edges, with a sink per apex (find.cu)
      if (nsmall > 0 || ntasks > 0)
        TC_TRY(find_vertex_list(g, small_list.p, g->ctrl.p + kCtrlQ0, nidx, tv));
      return TC_OK;
    }
  }
  TC_TRY((launch_hash<M, kBigThreads, kBigSlots, kBigWin[M], kBigPerSM, false>(
      g, pcols, items1.p, nitems1, ostart.p, owner_cnt.p, descs.p, task_split.p, task_idx.p,
      cursors.p, per_edge)));
  TC_TRY((launch_hash<M, kMedThreads, kMedSlots, kMedWin, kMedPerSM, kMedBatch[M]>(
      g, pcols, items0.p, nitems0, ostart.p, owner_cnt.p, descs.p, task_split.p, task_idx.p,
      cursors.p, per_edge)));
  cudaEventRecord(g->ev[7], st);  // end of the hash kernels
  // the merge list: small owners (from the count pass) and light owners
  // (appended by the scatter pass); its length is read on the device
  if (nsmall > 0 || ntasks > 0)
    TC_TRY(merge_small_edges(g, M, small_list.p, g->ctrl.p + kCtrlQ0, nidx, ustart, per_edge));
  return TC_OK;
}

// Edges [first, last) of the mode's index space (cover: H; plain: CSR
// entries, those with u > v skipped).  Requires |edges| < 2^32 and
// nnz < 2^32 (32-bit task indices and row positions); callers fall back to
// the merge kernels otherwise.
int hash_count(tc_graph* g, int mode, const int64_t* ustart, uint32_t* per_edge, int64_t first,
               int64_t last, unsigned long long* tv) {
  EdgeSrc s{};
  s.off = g->off;
  s.cols = g->cols;
  s.first = (uint64_t)first;
  if (last <= first) return TC_OK;
  const uint64_t nidx = (uint64_t)(last - first);
  if (mode == kModeCover) {
    s.H = g->cover.p;
    s.hoff = g->hoff.p;
    s.seg = g->seg.p;
    return hash_count_mode<kModeCover>(g, s, nidx, g->scols.p, ustart, per_edge, tv);
  }
  s.erow = g->erow.p;
  s.ustart = ustart;
  return hash_count_mode<kModePlain>(g, s, nidx, g->cols, ustart, per_edge, nullptr);
}

}  // namespace tc

// Warp-cooperative intersection of two sorted lists (shared by the
// intersection kernels).
#pragma once

#include <stdint.h>

namespace tc {

constexpr uint32_t kInf = 0xFFFFFFFFu;  // never a vertex id (n < 2^32 - 1)
constexpr int64_t kSkew = 24;           // merge when max(len) <= kSkew * min(len)

struct AcceptAll {
  __device__ __forceinline__ bool operator()(uint32_t) const { return true; }
};

// Number of w in A ∩ B with pred(w), for strictly ascending A[0..la),
// B[0..lb): a windowed merge when lb <= skew * la, else a binary search of
// the shorter list in the longer.  All 32 lanes call it with identical
// arguments; each returns its share of the count.
template <class Pred>
__device__ __forceinline__ unsigned warp_intersect_if(const uint32_t* __restrict__ A, int64_t la,
                                                      const uint32_t* __restrict__ B, int64_t lb,
                                                      Pred pred, int64_t skew = kSkew) {
  const int lane = threadIdx.x & 31;
  if (la > lb) {
    const uint32_t* t = A; A = B; B = t;
    int64_t tl = la; la = lb; lb = tl;
  }
  if (la == 0) return 0;
  unsigned cnt = 0;
  if (lb > skew * la) {
    // skewed: every lane binary-searches its elements of A in B; a lane's
    // elements increase, so its search window starts where the last ended
    int64_t lo = 0;
    for (int64_t k = lane; k < la; k += 32) {
      const uint32_t x = __ldg(A + k);
      int64_t hi = lb;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(B + mid) < x) lo = mid + 1; else hi = mid;
      }
      if (lo < lb && __ldg(B + lo) == x && pred(x)) ++cnt;
    }
    return cnt;
  }
  // windowed merge: a holds A[ia + lane], b holds B[ib + lane]
  int64_t ia = 0, ib = 0;
  uint32_t a = lane < la ? __ldg(A + lane) : kInf;
  uint32_t b = lane < lb ? __ldg(B + lane) : kInf;
  while (true) {
    const int a_last = (int)min((int64_t)31, la - 1 - ia);
    const int b_last = (int)min((int64_t)31, lb - 1 - ib);
    const uint32_t amax = __shfl_sync(0xFFFFFFFFu, a, a_last);
    const uint32_t bmax = __shfl_sync(0xFFFFFFFFu, b, b_last);
    // rank of a among the 32 window values (sorted, kInf padded)
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const uint32_t bv = __shfl_sync(0xFFFFFFFFu, b, pos + s - 1);
      if (bv < a) pos += s;
    }
    const uint32_t bv = __shfl_sync(0xFFFFFFFFu, b, pos);
    if (lane <= a_last && bv == a && pred(a)) ++cnt;
    const bool adv_a = amax <= bmax, adv_b = bmax <= amax;
    if (adv_a) {
      ia += 32;
      if (ia >= la) break;
      a = ia + lane < la ? __ldg(A + ia + lane) : kInf;
    }
    if (adv_b) {
      ib += 32;
      if (ib >= lb) break;
      b = ib + lane < lb ? __ldg(B + ib + lane) : kInf;
    }
  }
  return cnt;
}

// |A ∩ B| (every common element counts).
__device__ __forceinline__ unsigned warp_intersect(const uint32_t* __restrict__ A, int64_t la,
                                                   const uint32_t* __restrict__ B, int64_t lb) {
  return warp_intersect_if(A, la, B, lb, AcceptAll());
}

}  // namespace tc

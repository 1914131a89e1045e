// work_pairs.h -- the candidate pairs a work entry's segment presents to
// the counting kernel (before its neighbour cull), summed by the work
// builder into cute_stats.stencil_pairs and checked on the host against an
// enumeration of the same pairs (tests/work_cover_check.cu).
#pragma once

#include "count_kernel.cuh"

namespace cute {

// Pairs (i, j) that segment s presents to home chunk c = objects
// [c.x, c.y): every pair, but j > i on the home run's own cells (kSegSelf)
// and j != i on a full stencil's home row (kSegNoSelfPair).
__host__ __device__ inline unsigned long long segment_pairs(int4 c, const Seg &s) {
  unsigned long long n = 0;
  if (s.flags & kSegSelf) {
    for (int i = c.x; i < c.y; i++) {
      const int lo = s.j0 > i + 1 ? s.j0 : i + 1;
      if (s.j1 > lo) n += (unsigned)(s.j1 - lo);
    }
  } else {
    n = (unsigned long long)(c.y - c.x) * (unsigned)(s.j1 - s.j0);
    if (s.flags & kSegNoSelfPair) {
      const int lo = c.x > s.j0 ? c.x : s.j0, hi = c.y < s.j1 ? c.y : s.j1;
      if (hi > lo) n -= (unsigned)(hi - lo);
    }
  }
  return n;
}

}  // namespace cute

// cg_table.cuh -- device lookup of a pointer in the sorted allocation table.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_internal.h"

namespace cgi {

// Binary search of the sorted allocation table (Fig. 2's list).  Every
// `stride`-th base is staged in shared memory, so a lookup costs ~log2 of
// the splitter count in shared memory plus log2(stride) global probes.
__device__ __forceinline__ bool table_side(const DevTable &t, const uint64_t *spl, uint64_t nspl,
                                           uint32_t stride, uint64_t p, uint64_t n,
                                           uint64_t *found, uint64_t *abase, uint64_t *asize,
                                           uint64_t *shadow, uint32_t *flags, uint32_t f_unalloc,
                                           uint32_t f_overrun) {
  // last splitter <= p
  uint64_t lo = 0, hi = nspl;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (spl[mid] <= p)
      lo = mid + 1;
    else
      hi = mid;
  }
  int64_t j = -1;
  if (lo > 0) {
    uint64_t b = (lo - 1) * stride;
    uint64_t e = b + stride < t.count ? b + stride : t.count;
    while (b < e) {  // upper_bound within the block
      const uint64_t mid = (b + e) >> 1;
      if (__ldg(t.base + mid) <= p)
        b = mid + 1;
      else
        e = mid;
    }
    j = (int64_t)b - 1;
  }
  if (j >= 0) {
    const uint64_t base = __ldg(t.base + j);
    const uint64_t size = __ldg(t.size + j);
    if (p - base < size) {
      *found = base + size - p;
      *abase = base;
      *asize = size;
      *shadow = __ldg(t.shadow + j) + (p - base);
      if (n > *found) {
        *flags |= f_overrun;
        return false;
      }
      return true;
    }
  }
  *found = 0;
  *abase = 0;
  *asize = 0;
  *shadow = 0;
  *flags |= f_unalloc;
  return false;
}

}  // namespace cgi

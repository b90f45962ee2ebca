// cg_internal.h -- structures shared by libcg's host runtime and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cg.h"

#if defined(__CUDACC__)
#define CG_HD __host__ __device__ __forceinline__
#else
#define CG_HD inline
#endif

namespace cgi {

constexpr unsigned long long kNone = ~0ull;  // "no offset" inside the kernels

// job mode bits
constexpr uint32_t kModeCarry = 1u;    // perform the V-shadow carry
constexpr uint32_t kModeReadDev = 2u;  // device-source V is readable (valid src)
constexpr uint32_t kModeStall = 4u;    // injected fault: one tile's copy is never issued

// One copy as the scan kernels see it.  Addresses are absolute device
// addresses of copy byte 0 (host V: host_v + host_off).
struct ScanJob {
  uint32_t kind;
  uint32_t mode;
  uint64_t n;
  uint64_t host_off;  // HtoD: source offset, DtoH: destination offset
  uint64_t dev_src;   // shadow address of src byte 0 (DtoH/DtoD with kModeReadDev)
  uint64_t dev_dst;   // shadow address of dst byte 0 (HtoD/DtoD with kModeCarry)
};

// One pitched copy as the pitched scan kernel sees it: rows = height*depth
// rows of `width` bytes; row (y, z) of side s starts at
// s_start + z*s_slice + y*s_pitch (host side: offsets into the image; device
// sides: shadow addresses).
struct PitchedJob {
  uint32_t kind;
  uint32_t mode;
  uint64_t width, height, depth;
  uint64_t host_start, host_pitch, host_slice;
  uint64_t src_start, src_pitch, src_slice;  // kModeReadDev
  uint64_t dst_start, dst_pitch, dst_slice;  // kModeCarry (device destination)
};

// Bound host shadow image.
struct Image {
  const uint8_t *a_bits;
  uint8_t *v;
  uint64_t n;
};

// Per-request accumulators.  Counts are sums; first offsets are minima
// (kNone = none), so every contribution commutes.
struct Acc {
  unsigned long long n_unaddr;
  unsigned long long n_undef;
  unsigned long long first_unaddr;
  unsigned long long first_undef;
};

// Single-check scratch: the accumulator plus the count of CTAs done.  The
// last CTA copies the totals out and puts the scratch back to its initial
// state, so consecutive launches need no reset.
struct SingleScratch {
  Acc acc;
  unsigned int ctas_done;
  unsigned int error;        // nonzero: a bounded wait ran out (report flagged incomplete)
  unsigned long long claim;  // segments claimed beyond the warps' first (TMA kernel)
  unsigned int pad[4];
};

// Device-side verdict of the range part of a request (batched path).
struct RangeInfo {
  uint32_t flags;     // UNALLOC/OVERRUN/DTOD_OVERLAP bits
  uint32_t kind;
  uint64_t n;
  uint64_t found_dst, found_src;
  uint64_t base_dst, size_dst, base_src, size_src;
};

// Device copy of the allocation table (sorted by base; size 0 = tombstone).
struct DevTable {
  const uint64_t *base;
  const uint64_t *size;
  const uint64_t *shadow;  // device address of each allocation's V shadow
  uint64_t count;
};

// Batched-run level description (device arrays).
struct BatchPlan {
  const cg_copy *reqs;
  const uint32_t *order;      // request indices, level-major
  const uint64_t *seg_first;  // per order position: first segment id within its level
  const uint64_t *stage;      // per request: staging buffer for overlapping DtoD, 0 = none
  // per order position: the rows [lo, hi) of its copy that the position
  // covers, packed lo | hi << 32 (a row is 32 anchor chunks); 0 = the whole
  // copy.  Null: every position is a whole copy.  (TMA level kernel only.)
  const uint64_t *piece;
  ScanJob *jobs;              // per request
  RangeInfo *info;            // per request
  Acc *acc;                   // per request
  uint64_t nreq;
  uint32_t seg_chunks;        // segment length in 16-byte chunks
  uint32_t mode_mask;         // ANDed into every job's mode (clearing the carry = dry run)
};

// Build the user-visible report from the range verdict and the scan totals.
CG_HD void assemble_report(cg_report *r, const RangeInfo &ri, const Acc &a) {
  r->flags = ri.flags;
  r->expected = ri.n;
  r->found_dst = ri.found_dst;
  r->found_src = ri.found_src;
  r->alloc_base_dst = ri.base_dst;
  r->alloc_size_dst = ri.size_dst;
  r->alloc_base_src = ri.base_src;
  r->alloc_size_src = ri.size_src;
  r->race_seq = -1;
  r->n_unaddr = a.n_unaddr;
  r->n_undef = a.n_undef;
  r->n_good = ri.n - a.n_unaddr - a.n_undef;
  r->first_unaddr_off = a.first_unaddr == kNone ? -1 : (int64_t)a.first_unaddr;
  r->first_undef_off = a.first_undef == kNone ? -1 : (int64_t)a.first_undef;
  r->first_bad_off = -1;
  r->first_bad_kind = CG_BYTE_GOOD;
  if (a.first_unaddr != kNone && (a.first_undef == kNone || a.first_unaddr < a.first_undef)) {
    r->first_bad_off = (int64_t)a.first_unaddr;
    r->first_bad_kind = CG_BYTE_UNADDR;
  } else if (a.first_undef != kNone) {
    r->first_bad_off = (int64_t)a.first_undef;
    r->first_bad_kind = CG_BYTE_UNDEF;
  }
  if (a.n_unaddr) r->flags |= CG_F_HOST_UNADDR;
  if (a.n_undef) r->flags |= ri.kind == CG_HTOD ? CG_F_HOST_UNDEF : CG_F_DEV_UNDEF_SRC;
}

// Number of records a report produces (one per set flag).
CG_HD uint32_t record_count(uint32_t flags) {
  uint32_t c = 0;
  for (int b = 0; b < CG_NFLAGS; b++) c += (flags >> b) & 1u;
  return c;
}

// Write the records of one report starting at out[0]; returns how many.
CG_HD uint32_t write_records(const cg_report &r, const cg_copy &q, uint64_t req,
                             int strict, cg_err_record *out, uint64_t room) {
  uint32_t k = 0;
  for (uint32_t b = 0; b < CG_NFLAGS; b++) {
    uint32_t f = 1u << b;
    if (!(r.flags & f)) continue;
    cg_err_record e;
    e.req = req;
    e.cls = b;
    e.severity = 0;
    e.expected = q.n;
    if (f == CG_F_UNALLOC_DST || f == CG_F_UNALLOC_SRC) {
      e.off = 0;
      e.count = q.n;
      e.found = 0;
    } else if (f == CG_F_OVERRUN_DST || f == CG_F_OVERRUN_SRC) {
      uint64_t found = f == CG_F_OVERRUN_DST ? r.found_dst : r.found_src;
      e.off = (int64_t)found;
      e.count = q.n - found;
      e.found = found;
    } else if (f == CG_F_HOST_UNADDR) {
      e.off = r.first_unaddr_off;
      e.count = r.n_unaddr;
      e.found = q.n - r.n_unaddr;
    } else if (f == CG_F_HOST_UNDEF || f == CG_F_DEV_UNDEF_SRC) {
      e.off = r.first_undef_off;
      e.count = r.n_undef;
      e.found = r.n_good;
      if (f == CG_F_DEV_UNDEF_SRC && !strict) e.severity = 1;
    } else if (f == CG_F_DTOD_OVERLAP) {
      uint64_t dist = q.src <= q.dst ? q.dst - q.src : q.src - q.dst;
      e.off = (int64_t)(q.dst - q.src);
      e.count = q.n - dist;
      e.found = 0;
      e.severity = 1;
    } else {  // CG_F_CONCURRENT
      e.off = r.race_seq;
      e.count = q.n;
      e.found = 0;
      e.severity = 1;
    }
    if (k < room) out[k] = e;
    k++;
  }
  return k;
}

constexpr int kFinalizeItems = 1024;  // requests per finalize/emit block

// Set the text cg_last_error() returns on this thread (cg_host.cpp).
void set_error_text(const char *msg);

}  // namespace cgi

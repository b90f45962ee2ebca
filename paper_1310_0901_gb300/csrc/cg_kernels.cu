// cg_kernels.cu -- sm_103a kernels of libcg.
//
// The hot loop streams the shadow through HBM in 16-byte vectors: a warp
// covers 32 consecutive 16-byte chunks ("a row", 512 B), and every lane
// keeps kU rows of loads in flight before it classifies anything.  The
// chunk grid is aligned to the buffer the copy WRITES (the "anchor"), so
// stores are whole aligned vectors; an input stream with another alignment
// is realigned in registers with one warp shuffle and a byte funnel shift
// (lane 31 fetches the one chunk past the row itself).  Per-byte classes
// (Sec. 2 itemize: unaddressable / undefined) are found with bit tricks on
// 32-bit words and reduced with warp reductions, popc and ffs; counts and
// first offsets go to the request's accumulator with 64-bit atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_device.cuh"
#include "cg_table.cuh"
#include "cg_launch.h"

namespace cgi {

#ifndef CG_KU
#define CG_KU 4
#endif
#ifndef CG_MIN_BLOCKS
#define CG_MIN_BLOCKS 1
#endif
constexpr int kThreads = 256;
constexpr int kU = CG_KU;  // rows of loads in flight per lane

// kU rows starting at row0; rows >= nrows are skipped (warp-uniform).
template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ void do_rows(const Geo &g, const uint32_t *A32, int64_t row0,
                                        int nrows, int lane, LaneAcc &la) {
  uint4 v[kU];
  uint32_t a[kU];
#pragma unroll
  for (int u = 0; u < kU; u++) {
    const int64_t c = (row0 + u) * 32 + lane;
    v[u] = make_uint4(0, 0, 0, 0);
    a[u] = 0xFFFFu;
    if (u < nrows) {
      if (KIND == CG_HTOD || g.has_vin) v[u] = load_window(g, c, lane);
      if (KIND != CG_DTOD) a[u] = load_a16(A32, g.hb0 + 16 * c, g.hlo, g.hhi);
    }
  }
#pragma unroll
  for (int u = 0; u < kU; u++) {
    if (u >= nrows) break;
    const int64_t c = (row0 + u) * 32 + lane;
    chunk_step<KIND, CARRY>(g, c, v[u], a[u], valid_mask(16 * c - g.ax, g.n), la);
  }
}

template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ void do_range(const Geo &g, const uint32_t *A32, int64_t row_begin,
                                         int64_t row_end, int64_t row_step, int lane,
                                         LaneAcc &la) {
  for (int64_t r = row_begin; r < row_end; r += row_step) {
    const int64_t left = row_end - r;
    do_rows<KIND, CARRY>(g, A32, r, left < kU ? (int)left : kU, lane, la);
  }
}

// ---------------------------------------------------- single-copy kernel

// One copy over the whole grid.  Warps take groups of kU rows in grid-stride
// order; the last CTA to finish publishes the totals and resets the scratch.
template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kThreads, CG_MIN_BLOCKS) scan_single_kernel(Image img, ScanJob job,
                                                               RangeInfo ri, SingleScratch *scr,
                                                               cg_report *out) {
  const int lane = threadIdx.x & 31;
  const Geo g = make_geo(job, img);
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rows = (g.nchunks + 31) >> 5;
  LaneAcc la;
  lane_acc_reset(la);
  for (int64_t r = warp * kU; r < rows; r += nwarps * kU) {
    const int64_t left = rows - r;
    do_rows<KIND, CARRY>(g, A32, r, left < kU ? (int)left : kU, lane, la);
  }
  single_epilogue(la, scr, ri, out, 0u);
}

__global__ void init_single_scratch_kernel(SingleScratch *s) {
  s->acc.n_unaddr = 0;
  s->acc.n_undef = 0;
  s->acc.first_unaddr = kNone;
  s->acc.first_undef = kNone;
  s->ctas_done = 0;
  s->error = 0;
  s->claim = 0;
}

cudaError_t launch_init_single_scratch(SingleScratch *s, cudaStream_t st) {
  init_single_scratch_kernel<<<1, 1, 0, st>>>(s);
  return cudaGetLastError();
}

template <uint32_t KIND, bool CARRY>
static void *single_fn() {
  return reinterpret_cast<void *>(&scan_single_kernel<KIND, CARRY>);
}

static void *pick_single(uint32_t kind, bool carry) {
  switch (kind) {
    case CG_HTOD:
      return carry ? single_fn<CG_HTOD, true>() : single_fn<CG_HTOD, false>();
    case CG_DTOH:
      return carry ? single_fn<CG_DTOH, true>() : single_fn<CG_DTOH, false>();
    default:
      return carry ? single_fn<CG_DTOD, true>() : single_fn<CG_DTOD, false>();
  }
}

int scan_single_max_ctas_per_sm(uint32_t kind, uint32_t mode) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_single(kind, mode & kModeCarry),
                                                    kThreads, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t launch_scan_single(const Image &img, const ScanJob &job, const RangeInfo &ri,
                               SingleScratch *scratch, cg_report *out, int grid,
                               cudaStream_t st) {
  const bool carry = job.mode & kModeCarry;
  switch (job.kind) {
    case CG_HTOD:
      if (carry)
        scan_single_kernel<CG_HTOD, true><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      else
        scan_single_kernel<CG_HTOD, false><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      break;
    case CG_DTOH:
      if (carry)
        scan_single_kernel<CG_DTOH, true><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      else
        scan_single_kernel<CG_DTOH, false><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      break;
    default:
      if (carry)
        scan_single_kernel<CG_DTOD, true><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      else
        scan_single_kernel<CG_DTOD, false><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------ batched: lookup

__global__ void __launch_bounds__(256) lookup_kernel(DevTable t, BatchPlan p, uint32_t stride,
                                                     int carry_on) {
  extern __shared__ uint64_t spl[];
  const uint64_t nspl = (t.count + stride - 1) / stride;
  for (uint64_t k = threadIdx.x; k < nspl; k += blockDim.x) spl[k] = __ldg(t.base + k * stride);
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nreq;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const cg_copy q = p.reqs[i];
    RangeInfo ri;
    ri.flags = 0;
    ri.kind = q.kind;
    ri.n = q.n;
    ri.found_dst = ri.found_src = 0;
    ri.base_dst = ri.size_dst = ri.base_src = ri.size_src = 0;
    ScanJob j;
    j.kind = q.kind;
    j.mode = 0;
    j.n = q.n;
    j.host_off = q.kind == CG_HTOD ? q.src : (q.kind == CG_DTOH ? q.dst : 0);
    j.dev_src = 0;
    j.dev_dst = 0;
    Acc a;
    a.n_unaddr = 0;
    a.n_undef = 0;
    a.first_unaddr = kNone;
    a.first_undef = kNone;
    if (q.n > 0) {
      bool dst_ok = true, src_ok = true;
      uint64_t dsh = 0, ssh = 0;
      if (q.kind != CG_DTOH)
        dst_ok = table_side(t, spl, nspl, stride, q.dst, q.n, &ri.found_dst, &ri.base_dst,
                            &ri.size_dst, &dsh, &ri.flags, CG_F_UNALLOC_DST, CG_F_OVERRUN_DST);
      if (q.kind != CG_HTOD)
        src_ok = table_side(t, spl, nspl, stride, q.src, q.n, &ri.found_src, &ri.base_src,
                            &ri.size_src, &ssh, &ri.flags, CG_F_UNALLOC_SRC, CG_F_OVERRUN_SRC);
      if (q.kind == CG_DTOD) {
        const uint64_t dist = q.src <= q.dst ? q.dst - q.src : q.src - q.dst;
        if (dist < q.n) ri.flags |= CG_F_DTOD_OVERLAP;
      }
      if (q.kind != CG_HTOD && src_ok) {
        j.mode |= kModeReadDev;
        j.dev_src = p.stage[i] ? p.stage[i] : ssh;
      }
      if (carry_on && dst_ok && src_ok) {
        j.mode |= kModeCarry;
        j.dev_dst = dsh;  // 0 for DtoH: the host image is the destination
      }
    }
    p.jobs[i] = j;
    p.info[i] = ri;
    p.acc[i] = a;
  }
}

cudaError_t launch_lookup(const DevTable &t, const BatchPlan &p, int strict, int carry,
                          cudaStream_t st) {
  (void)strict;
  if (p.nreq == 0) return cudaSuccess;
  uint32_t stride = 256;
  while ((t.count + stride - 1) / stride > 6144) stride <<= 1;
  const uint64_t nspl = (t.count + stride - 1) / stride;
  const size_t smem = (size_t)(nspl ? nspl : 1) * sizeof(uint64_t);
  uint64_t blocks = (p.nreq + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  lookup_kernel<<<(unsigned)blocks, 256, smem, st>>>(t, p, stride, carry);
  return cudaGetLastError();
}

// -------------------------------------------------- table merge (update)

// Number of entries of the sorted array a[0..n) below x.
__device__ __forceinline__ uint64_t count_below(const uint64_t *a, uint64_t n, uint64_t x) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The device table brought up to date in one pass (Sec. 2: the list of
// allocations changes with every cudaMalloc / cudaFree wrapper): the old
// sorted table minus the entries whose bases are in the sorted list
// `dead`, plus the (sorted) registrations ins_*, written in base order into
// the other buffer.  Each entry computes its place directly: an old entry
// goes to its index - (dead bases below its base) + (registrations below
// its base); a registration k goes to k + (old bases below its base) -
// (dead bases below it).  A registration may reuse the base of a dead
// entry; it never meets a live one (registrations do not overlap live
// allocations).
__global__ void __launch_bounds__(256) table_merge_kernel(DevTable t, const uint64_t *ins_base,
                                                          const uint64_t *ins_size,
                                                          const uint64_t *ins_shadow, uint64_t m,
                                                          const uint64_t *dead, uint64_t d,
                                                          uint64_t *nb, uint64_t *ns,
                                                          uint64_t *nh) {
  const uint64_t total = t.count + m;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t o, b, sz, sh;
    if (i < t.count) {
      b = __ldg(t.base + i);
      const uint64_t r = count_below(dead, d, b);
      if (r < d && __ldg(dead + r) == b) continue;
      sz = __ldg(t.size + i);
      sh = __ldg(t.shadow + i);
      o = i - r + count_below(ins_base, m, b);
    } else {
      const uint64_t k = i - t.count;
      b = __ldg(ins_base + k);
      sz = __ldg(ins_size + k);
      sh = __ldg(ins_shadow + k);
      o = k + count_below(t.base, t.count, b) - count_below(dead, d, b);
    }
    nb[o] = b;
    ns[o] = sz;
    nh[o] = sh;
  }
}

cudaError_t launch_table_merge(const DevTable &t, const uint64_t *ins_base,
                               const uint64_t *ins_size, const uint64_t *ins_shadow, uint64_t m,
                               const uint64_t *dead, uint64_t d, uint64_t *nb, uint64_t *ns,
                               uint64_t *nh, int sm_count, cudaStream_t st) {
  const uint64_t total = t.count + m;
  if (total == 0) return cudaSuccess;
  uint64_t blocks = (total + 255) / 256;
  const uint64_t cap = (uint64_t)(sm_count > 0 ? sm_count : 1) * 8;
  if (blocks > cap) blocks = cap;
  table_merge_kernel<<<(unsigned)blocks, 256, 0, st>>>(t, ins_base, ins_size, ins_shadow, m, dead,
                                                       d, nb, ns, nh);
  return cudaGetLastError();
}

// The job mode bits of every request, packed one byte each for the host's
// level planner.
__global__ void job_modes_kernel(const ScanJob *jobs, uint64_t nreq, uint8_t *modes) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nreq;
       i += (uint64_t)gridDim.x * blockDim.x)
    modes[i] = (uint8_t)jobs[i].mode;
}

cudaError_t launch_job_modes(const BatchPlan &p, uint8_t *modes, cudaStream_t st) {
  if (p.nreq == 0) return cudaSuccess;
  uint64_t blocks = (p.nreq + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  job_modes_kernel<<<(unsigned)blocks, 256, 0, st>>>(p.jobs, p.nreq, modes);
  return cudaGetLastError();
}

// ---------------------------------------------------- batched: one level

// Persistent-style kernel over the byte segments of every copy of one
// dependency level.  Warp w takes segments w, w + W, ...; a segment maps to
// its copy by binary search over the level's segment prefix.
__global__ void __launch_bounds__(kThreads) scan_level_kernel(Image img, BatchPlan p,
                                                              uint64_t pos_begin, uint64_t pos_end,
                                                              uint64_t n_segs) {
  const int lane = threadIdx.x & 31;
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t seg_rows = p.seg_chunks >> 5;
  LaneAcc la;
  lane_acc_reset(la);
  for (uint64_t s = warp; s < n_segs; s += nwarps) {
    uint64_t lo = pos_begin, hi = pos_end;  // last position with seg_first <= s
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (__ldg(p.seg_first + mid) <= s)
        lo = mid;
      else
        hi = mid;
    }
    const uint32_t req = __ldg(p.order + lo);
    ScanJob job = p.jobs[req];
    job.mode &= p.mode_mask;
    const Geo g = make_geo(job, img);
    const int64_t k = (int64_t)(s - __ldg(p.seg_first + lo));
    const int64_t rows = (g.nchunks + 31) >> 5;
    const int64_t r0 = k * seg_rows;
    const int64_t r1 = r0 + seg_rows < rows ? r0 + seg_rows : rows;
    if (r0 < r1) {
      const bool carry = job.mode & kModeCarry;
      switch (job.kind) {
        case CG_HTOD:
          if (carry)
            do_range<CG_HTOD, true>(g, A32, r0, r1, kU, lane, la);
          else
            do_range<CG_HTOD, false>(g, A32, r0, r1, kU, lane, la);
          break;
        case CG_DTOH:
          if (carry)
            do_range<CG_DTOH, true>(g, A32, r0, r1, kU, lane, la);
          else
            do_range<CG_DTOH, false>(g, A32, r0, r1, kU, lane, la);
          break;
        default:
          if (carry)
            do_range<CG_DTOD, true>(g, A32, r0, r1, kU, lane, la);
          else
            do_range<CG_DTOD, false>(g, A32, r0, r1, kU, lane, la);
          break;
      }
      warp_flush(la, &p.acc[req], lane);
    }
  }
}

cudaError_t launch_scan_level(const Image &img, const BatchPlan &p, uint64_t pos_begin,
                              uint64_t pos_end, uint64_t n_segs, int grid, cudaStream_t st) {
  if (n_segs == 0 || pos_end <= pos_begin) return cudaSuccess;
  const uint64_t warps_needed = n_segs;
  const uint64_t ctas_needed = (warps_needed + (kThreads / 32) - 1) / (kThreads / 32);
  const unsigned g = (unsigned)(ctas_needed < (uint64_t)grid ? ctas_needed : (uint64_t)grid);
  scan_level_kernel<<<g, kThreads, 0, st>>>(img, p, pos_begin, pos_end, n_segs);
  return cudaGetLastError();
}

// --------------------------------------- batched: reports and records

// Block-wide exclusive scan of per-thread values (256 threads).
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t x, uint64_t *total) {
  __shared__ uint64_t warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(CG_FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint64_t before = 0, all = 0;
  for (int k = 0; k < kThreads / 32; k++) {
    if (k < w) before += warp_tot[k];
    all += warp_tot[k];
  }
  __syncthreads();
  if (total) *total = all;
  return before + incl - x;
}

constexpr int kPerThread = kFinalizeItems / kThreads;

__global__ void __launch_bounds__(kThreads) finalize_kernel(BatchPlan p, cg_report *reps,
                                                            uint32_t *counts,
                                                            uint64_t *block_sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kFinalizeItems + threadIdx.x * kPerThread;
  uint64_t mine = 0;
  for (int k = 0; k < kPerThread; k++) {
    const uint64_t i = base + k;
    if (i >= p.nreq) break;
    cg_report r;
    assemble_report(&r, p.info[i], p.acc[i]);
    reps[i] = r;
    const uint32_t c = record_count(r.flags);
    counts[i] = c;
    mine += c;
  }
  uint64_t total;
  block_exclusive_scan(mine, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Reports written straight into pinned host memory (no read-back copy):
// out = error flag (16 bytes) | reports.  Runs after the level kernels on
// the same stream, so the flag is final (serving rounds, kernel-argument
// checks).
__global__ void __launch_bounds__(kThreads) finalize_host_kernel(BatchPlan p,
                                                                  const unsigned int *err,
                                                                  uint8_t *out) {
  const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i == 0) *reinterpret_cast<unsigned int *>(out) = *err;
  if (i < p.nreq) {
    cg_report r;
    assemble_report(&r, p.info[i], p.acc[i]);
    reinterpret_cast<cg_report *>(out + 16)[i] = r;
  }
}

cudaError_t launch_finalize_host(const BatchPlan &p, const unsigned int *err, uint8_t *out,
                                  cudaStream_t st) {
  const uint64_t nb = (p.nreq + kThreads - 1) / kThreads;
  finalize_host_kernel<<<(unsigned)(nb ? nb : 1), kThreads, 0, st>>>(p, err, out);
  return cudaGetLastError();
}

// Exclusive scan of the block sums in one CTA; total count at block_sums[nblocks].
__global__ void __launch_bounds__(kThreads) scan_block_sums_kernel(uint64_t *sums,
                                                                   uint64_t nblocks) {
  uint64_t carry = 0;
  for (uint64_t b0 = 0; b0 < nblocks; b0 += kThreads) {
    const uint64_t i = b0 + threadIdx.x;
    const uint64_t x = i < nblocks ? sums[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan(x, &tot);
    if (i < nblocks) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nblocks] = carry;
}

__global__ void __launch_bounds__(kThreads) emit_records_kernel(BatchPlan p, const cg_report *reps,
                                                                const uint32_t *counts,
                                                                const uint64_t *block_off,
                                                                int strict, cg_err_record *recs,
                                                                uint64_t rec_cap) {
  const uint64_t base = (uint64_t)blockIdx.x * kFinalizeItems + threadIdx.x * kPerThread;
  uint64_t mine = 0;
  for (int k = 0; k < kPerThread; k++) {
    const uint64_t i = base + k;
    if (i < p.nreq) mine += counts[i];
  }
  uint64_t off = block_off[blockIdx.x] + block_exclusive_scan(mine, nullptr);
  for (int k = 0; k < kPerThread; k++) {
    const uint64_t i = base + k;
    if (i >= p.nreq) break;
    const uint32_t c = counts[i];
    if (c && off < rec_cap) {
      const cg_report r = reps[i];
      write_records(r, p.reqs[i], i, strict, recs + off, rec_cap - off);
    }
    off += c;
  }
}

cudaError_t launch_finalize(const BatchPlan &p, cg_report *reps, uint32_t *counts,
                            uint64_t *block_sums, int items_per_block, cudaStream_t st) {
  (void)items_per_block;
  const uint64_t nb = (p.nreq + kFinalizeItems - 1) / kFinalizeItems;
  if (nb == 0) return cudaSuccess;
  finalize_kernel<<<(unsigned)nb, kThreads, 0, st>>>(p, reps, counts, block_sums);
  return cudaGetLastError();
}

cudaError_t launch_scan_block_sums(uint64_t *block_sums, uint64_t nblocks, uint64_t *total,
                                   cudaStream_t st) {
  (void)total;
  scan_block_sums_kernel<<<1, kThreads, 0, st>>>(block_sums, nblocks);
  return cudaGetLastError();
}

cudaError_t launch_emit_records(const BatchPlan &p, const cg_report *reps, const uint32_t *counts,
                                const uint64_t *block_sums, int items_per_block, int strict,
                                cg_err_record *recs, uint64_t rec_cap, cudaStream_t st) {
  (void)items_per_block;
  const uint64_t nb = (p.nreq + kFinalizeItems - 1) / kFinalizeItems;
  if (nb == 0 || rec_cap == 0) return cudaSuccess;
  emit_records_kernel<<<(unsigned)nb, kThreads, 0, st>>>(p, reps, counts, block_sums, strict,
                                                         recs, rec_cap);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fill

// Fill shadow ranges (256-byte aligned, multiples of 256 bytes) with a value.
__global__ void fill_kernel(const uint64_t *ptrs, const uint64_t *sizes, uint64_t count,
                            uint32_t word) {
  for (uint64_t e = blockIdx.x; e < count; e += gridDim.x) {
    uint4 *p = reinterpret_cast<uint4 *>(ptrs[e]);
    const uint64_t nv = sizes[e] >> 4;
    const uint4 w = make_uint4(word, word, word, word);
    for (uint64_t k = threadIdx.x; k < nv; k += blockDim.x) p[k] = w;
  }
}

cudaError_t launch_fill(const uint64_t *ptrs, const uint64_t *sizes, uint64_t count,
                        uint8_t value, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const uint32_t word = 0x01010101u * value;
  const unsigned blocks = (unsigned)(count < 65535 ? count : 65535);
  fill_kernel<<<blocks, 256, 0, st>>>(ptrs, sizes, count, word);
  return cudaGetLastError();
}

}  // namespace cgi

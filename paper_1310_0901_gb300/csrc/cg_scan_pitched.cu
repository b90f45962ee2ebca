// cg_scan_pitched.cu -- the scan of a pitched (2-D / 3-D) copy.
//
// A pitched copy is height*depth rows of `width` bytes whose starts differ by
// a pitch (and a slice stride) on every side, so each row has its own
// alignment.  Only the copied bytes are read and classified (the footnote to
// Sec. 2's error list: strided host access is not an error), and the carry
// writes only the copied bytes of each destination row.
//
// Work split: a row is cut into groups of P*U 16-byte chunks of its anchor
// grid; a subgroup of P lanes takes one group (U chunks per lane).  Wide
// rows use whole warps (P = 32) with U = 4 loads in flight per lane; rows of
// at most 32 chunks use P = the next power of two of their chunk count and
// U = 1, so one warp covers 32/P rows at once.  Warps walk the (row, group)
// items in grid-stride order, advancing (group, y, z) incrementally.  The
// last CTA to finish publishes the report, as for a plain copy.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_device.cuh"

namespace cgi {

constexpr int kPThreads = 256;
constexpr int kPWide = 4;  // chunks in flight per lane on wide rows

// Grid-stride bookkeeping computed on the host for the chosen grid.
struct PitchedGrid {
  uint64_t groups;  // chunk groups per row (G)
  uint64_t tg;      // per-iteration advance of the group index: T mod G
  uint64_t ty, tz;  // ... and of the row: (T div G) as (y, z) steps
  uint32_t lp;      // log2 of the lanes per group (P)
};

// The input V window of chunk c when the warp is split into groups of P
// lanes: the lane after this one (same group) holds chunk c+1's first
// vector; the last lane of a group fetches it itself.  Every lane calls it.
__device__ __forceinline__ uint4 load_window_group(const Geo &g, int64_t c, bool last_in_group) {
  const uintptr_t a0 = g.vin_al + 16 * (uintptr_t)c;
  const bool in0 = a0 < g.vin_hi && a0 + 16 > g.vin_lo;
  const uint4 l0 = in0 ? ld_stream((const void *)a0) : make_uint4(0, 0, 0, 0);
  uint4 l1;
  l1.x = __shfl_down_sync(CG_FULL, l0.x, 1);
  l1.y = __shfl_down_sync(CG_FULL, l0.y, 1);
  l1.z = __shfl_down_sync(CG_FULL, l0.z, 1);
  l1.w = __shfl_down_sync(CG_FULL, l0.w, 1);
  if (last_in_group) {
    const uintptr_t a1 = a0 + 16;
    const bool in1 = a1 < g.vin_hi && a1 + 16 > g.vin_lo;
    l1 = in1 ? ld_stream((const void *)a1) : make_uint4(0, 0, 0, 0);
  }
  return g.vin_r == 0 ? l0 : funnel16(l0, l1, g.vin_r);
}

template <uint32_t KIND, bool CARRY, int U>
__global__ void __launch_bounds__(kPThreads) scan_pitched_kernel(Image img, PitchedJob pj,
                                                                 RangeInfo ri, SingleScratch *scr,
                                                                 cg_report *out, PitchedGrid pg) {
  const int lane = threadIdx.x & 31;
  const uint32_t P = 1u << pg.lp;
  const uint32_t ls = lane & (P - 1);
  const uint64_t per_unit = 32u >> pg.lp;  // groups one warp takes at once
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  const uint64_t t0 = warp * per_unit + (lane >> pg.lp);
  uint64_t grp = t0 % pg.groups;
  const uint64_t r0 = t0 / pg.groups;
  uint64_t y = r0 % pj.height, z = r0 / pj.height;
  LaneAcc la;
  lane_acc_reset(la);
  while (__any_sync(CG_FULL, z < pj.depth)) {
    ScanJob j;
    j.kind = KIND;
    j.mode = pj.mode;
    j.n = z < pj.depth ? pj.width : 0;  // past the last row: an empty row
    j.host_off = pj.host_start + z * pj.host_slice + y * pj.host_pitch;
    j.dev_src = pj.src_start + z * pj.src_slice + y * pj.src_pitch;
    j.dev_dst = pj.dst_start + z * pj.dst_slice + y * pj.dst_pitch;
    Geo g = make_geo(j, img);
    g.obase = (int64_t)((z * pj.height + y) * pj.width);
    const int64_t c0 = (int64_t)(grp * P * U) + ls;
    uint4 v[U];
    uint32_t a[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int64_t c = c0 + (int64_t)k * P;
      v[k] = make_uint4(0, 0, 0, 0);
      a[k] = 0xFFFFu;
      if (KIND == CG_HTOD || g.has_vin) v[k] = load_window_group(g, c, ls == P - 1);
      if (KIND != CG_DTOD) a[k] = load_a16(A32, g.hb0 + 16 * c, g.hlo, g.hhi);
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int64_t c = c0 + (int64_t)k * P;
      chunk_step<KIND, CARRY>(g, c, v[k], a[k], valid_mask(16 * c - g.ax, g.n), la);
    }
    grp += pg.tg;
    uint64_t next_row = 0;
    if (grp >= pg.groups) {
      grp -= pg.groups;
      next_row = 1;
    }
    y += pg.ty + next_row;
    z += pg.tz;
    if (y >= pj.height) {
      y -= pj.height;
      z++;
    }
  }
  single_epilogue(la, scr, ri, out, 0u);
}

template <uint32_t KIND, bool CARRY>
static void *pitched_fn(bool wide) {
  return wide ? reinterpret_cast<void *>(&scan_pitched_kernel<KIND, CARRY, kPWide>)
              : reinterpret_cast<void *>(&scan_pitched_kernel<KIND, CARRY, 1>);
}

static void *pick_pitched(uint32_t kind, bool carry, bool wide) {
  switch (kind) {
    case CG_HTOD:
      return carry ? pitched_fn<CG_HTOD, true>(wide) : pitched_fn<CG_HTOD, false>(wide);
    case CG_DTOH:
      return carry ? pitched_fn<CG_DTOH, true>(wide) : pitched_fn<CG_DTOH, false>(wide);
    default:
      return carry ? pitched_fn<CG_DTOD, true>(wide) : pitched_fn<CG_DTOD, false>(wide);
  }
}

cudaError_t launch_scan_pitched(const Image &img, const PitchedJob &job, const RangeInfo &ri,
                                SingleScratch *scr, cg_report *out, int sm_count,
                                cudaStream_t st) {
  const uint64_t kmax = (job.width + 30) >> 4;  // anchor chunks of a row, any alignment
  const bool wide = kmax > 32;
  uint32_t lp = 0;
  while ((1ull << lp) < kmax && lp < 5) lp++;
  PitchedGrid pg;
  pg.lp = wide ? 5 : lp;
  const uint64_t per_group = wide ? 32ull * kPWide : 1ull << pg.lp;
  pg.groups = (kmax + per_group - 1) / per_group;
  const uint64_t per_unit = 32ull >> pg.lp;
  const uint64_t rows = job.height * job.depth;
  const uint64_t units = (rows * pg.groups + per_unit - 1) / per_unit;
  void *fn = pick_pitched(job.kind, job.mode & kModeCarry, wide);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const uint64_t warps_per_cta = kPThreads / 32;
  const uint64_t need = (units + warps_per_cta - 1) / warps_per_cta;
  const uint64_t cap = (uint64_t)sm_count * (uint64_t)per_sm;
  const unsigned grid = (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
  const uint64_t T = (uint64_t)grid * warps_per_cta * per_unit;  // groups per grid step
  pg.tg = T % pg.groups;
  const uint64_t tr = T / pg.groups;
  pg.ty = tr % job.height;
  pg.tz = tr / job.height;
  void *args[] = {const_cast<Image *>(&img), const_cast<PitchedJob *>(&job),
                  const_cast<RangeInfo *>(&ri), &scr, &out, &pg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kPThreads), args, 0, st);
}

// ------------------------------------------------- staging an overlap

// Row-major gather of a pitched device span: one warp per row, bytes
// coalesced across the lanes.  Used only to stage the source of an
// overlapping device->device copy (the carry must read it all first).
__global__ void __launch_bounds__(kPThreads) gather_rows_kernel(const uint8_t *src, uint64_t pitch,
                                                                uint64_t slice, uint64_t width,
                                                                uint64_t height, uint64_t rows,
                                                                uint8_t *out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < rows; r += nwarps) {
    const uint8_t *s = src + (r / height) * slice + (r % height) * pitch;
    uint8_t *o = out + r * width;
    for (uint64_t i = lane; i < width; i += 32) o[i] = s[i];
  }
}

cudaError_t launch_gather_rows(const uint8_t *src, uint64_t pitch, uint64_t slice,
                               uint64_t width, uint64_t height, uint64_t depth, uint8_t *out,
                               int sm_count, cudaStream_t st) {
  const uint64_t rows = height * depth;
  const uint64_t need = (rows + kPThreads / 32 - 1) / (kPThreads / 32);
  const uint64_t cap = (uint64_t)sm_count * 8;
  const unsigned grid = (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
  gather_rows_kernel<<<grid, kPThreads, 0, st>>>(src, pitch, slice, width, height, rows, out);
  return cudaGetLastError();
}

}  // namespace cgi

// cg_scan_pitched.cu -- the scan of a pitched (2-D / 3-D) copy.
//
// A pitched copy is height*depth rows of `width` bytes whose starts differ by
// a pitch (and a slice stride) on every side, so each row has its own
// alignment.  Only the copied bytes are read and classified (the footnote to
// Sec. 2's error list: strided host access is not an error), and the carry
// writes only the copied bytes of each destination row.
//
// Three launch shapes, by the row's length in 16-byte chunks of its anchor
// grid (the buffer the copy writes):
//   - rows of at most 32 chunks: a group of P lanes (P = the next power of
//     two of the chunk count) takes one row, and every group U rows at once
//     (all loads first, then the classification), so one warp covers
//     32/P * U rows per step;
//   - rows of up to kTmaRowChunks chunks: whole warps take groups of 128
//     chunks of a row, 4 loads in flight per lane;
//   - longer rows: the TMA tile pipeline of the plain copy (per-warp
//     shared-memory stages filled by bulk copies), one 5 KiB tile of one row
//     at a time, rows taken in order.
// The last CTA to finish publishes the report, as for a plain copy.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_setup.h"
#include "cg_tma.cuh"
#include "cg_launch.h"

namespace cgi {

// Short rows are latency-bound: measured on the 16-byte-field workload,
// one row per lane group and 8 CTAs per SM (64 warps, a few spilled
// registers) beat more rows in flight per lane at lower occupancy
// (0.159 ms vs 0.17-0.30 ms for 2-8 rows at 2-6 CTAs per SM).
#ifndef CG_PN_U
#define CG_PN_U 1
#endif
#ifndef CG_PN_MINB
#define CG_PN_MINB 8
#endif

constexpr int kPThreads = 256;
constexpr int kPWide = 4;          // chunks in flight per lane on medium rows
constexpr int kPNarrow = CG_PN_U;  // rows in flight per lane group on short rows
constexpr uint64_t kTmaRowChunks = 256;  // rows this long go to the TMA pipeline

// Row r of the copy as a plain one-row job; obase = its first byte's offset
// in the copy.  Rows past the end become empty jobs (nothing is read).
__device__ __forceinline__ Geo row_geo(const PitchedJob &pj, const Image &img, uint32_t kind,
                                       uint64_t r) {
  uint64_t y = r, z = 0;
  if (pj.depth > 1) {
    z = r / pj.height;
    y = r - z * pj.height;
  }
  ScanJob j;
  j.kind = kind;
  j.mode = pj.mode;
  j.n = z < pj.depth && y < pj.height ? pj.width : 0;
  j.host_off = pj.host_start + z * pj.host_slice + y * pj.host_pitch;
  j.dev_src = pj.src_start + z * pj.src_slice + y * pj.src_pitch;
  j.dev_dst = pj.dst_start + z * pj.dst_slice + y * pj.dst_pitch;
  Geo g = make_geo(j, img);
  g.obase = (int64_t)(r * pj.width);
  return g;
}

// The input V window of chunk c when the warp is split into groups of P
// lanes: the lane after this one (same group) holds chunk c+1's first
// vector; the last lane of a group fetches it itself.  Every lane calls it.
// Both of the last lane's loads are issued before the shuffle waits on the
// first, so a group of one lane has its two loads in flight together.
__device__ __forceinline__ uint4 load_window_group(const Geo &g, int64_t c, bool last_in_group) {
  const uintptr_t a0 = g.vin_al + 16 * (uintptr_t)c;
  const uintptr_t a1 = a0 + 16;
  const bool in0 = a0 < g.vin_hi && a0 + 16 > g.vin_lo;
  const bool in1 = last_in_group && g.vin_r != 0 && a1 < g.vin_hi && a1 + 16 > g.vin_lo;
  const uint4 l0 = in0 ? ld_stream((const void *)a0) : make_uint4(0, 0, 0, 0);
  const uint4 own1 = in1 ? ld_stream((const void *)a1) : make_uint4(0, 0, 0, 0);
  uint4 l1;
  l1.x = __shfl_down_sync(CG_FULL, l0.x, 1);
  l1.y = __shfl_down_sync(CG_FULL, l0.y, 1);
  l1.z = __shfl_down_sync(CG_FULL, l0.z, 1);
  l1.w = __shfl_down_sync(CG_FULL, l0.w, 1);
  if (last_in_group) l1 = own1;
  return g.vin_r == 0 ? l0 : funnel16(l0, l1, g.vin_r);
}

// ------------------------------------------------------------ short rows

// Groups of P = 2^lp lanes; each group takes U rows per step: rows
// base + k*(32/P) + group, k < U.
template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kPThreads, CG_PN_MINB) scan_pitched_narrow_kernel(Image img, PitchedJob pj,
                                                                        RangeInfo ri,
                                                                        SingleScratch *scr,
                                                                        cg_report *out,
                                                                        uint32_t lp) {
  constexpr int U = kPNarrow;
  const int lane = threadIdx.x & 31;
  const uint32_t P = 1u << lp;
  const uint32_t ls = lane & (P - 1);
  const uint64_t groups = 32u >> lp;
  const uint64_t per_step = groups * U;
  const uint64_t rows = pj.height * pj.depth;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  LaneAcc la;
  lane_acc_reset(la);
  for (uint64_t base = warp * per_step; base < rows; base += nwarps * per_step) {
    Geo g[U];
    uint4 v[U];
    uint32_t a[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      g[k] = row_geo(pj, img, KIND, base + (uint64_t)k * groups + (lane >> lp));
      v[k] = make_uint4(0, 0, 0, 0);
      a[k] = 0xFFFFu;
      if (KIND == CG_HTOD || g[k].has_vin) v[k] = load_window_group(g[k], ls, ls == P - 1);
      if (KIND != CG_DTOD) a[k] = load_a16(A32, g[k].hb0 + 16 * (int64_t)ls, g[k].hlo, g[k].hhi);
    }
#pragma unroll
    for (int k = 0; k < U; k++)
      chunk_step<KIND, CARRY>(g[k], ls, v[k], a[k], valid_mask(16 * (int64_t)ls - g[k].ax, g[k].n),
                              la);
  }
  single_epilogue(la, scr, ri, out, 0u);
}

// ----------------------------------------------------------- medium rows

// Whole warps; item = (row, group of 32*U chunks), items in grid-stride
// order, (group, row) advanced incrementally by the grid's step.
struct WideStep {
  uint64_t groups;  // chunk groups per row
  uint64_t tg, tr;  // grid step: group advance, row advance
};

template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kPThreads) scan_pitched_wide_kernel(Image img, PitchedJob pj,
                                                                      RangeInfo ri,
                                                                      SingleScratch *scr,
                                                                      cg_report *out, WideStep ws) {
  constexpr int U = kPWide;
  const int lane = threadIdx.x & 31;
  const uint64_t rows = pj.height * pj.depth;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  uint64_t grp = warp % ws.groups;
  uint64_t r = warp / ws.groups;
  LaneAcc la;
  lane_acc_reset(la);
  while (r < rows) {  // warp-uniform
    const Geo g = row_geo(pj, img, KIND, r);
    const int64_t c0 = (int64_t)(grp * 32 * U) + lane;
    uint4 v[U];
    uint32_t a[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int64_t c = c0 + 32 * k;
      v[k] = make_uint4(0, 0, 0, 0);
      a[k] = 0xFFFFu;
      if (KIND == CG_HTOD || g.has_vin) v[k] = load_window_group(g, c, lane == 31);
      if (KIND != CG_DTOD) a[k] = load_a16(A32, g.hb0 + 16 * c, g.hlo, g.hhi);
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int64_t c = c0 + 32 * k;
      chunk_step<KIND, CARRY>(g, c, v[k], a[k], valid_mask(16 * c - g.ax, g.n), la);
    }
    grp += ws.tg;
    r += ws.tr;
    if (grp >= ws.groups) {
      grp -= ws.groups;
      r++;
    }
  }
  single_epilogue(la, scr, ri, out, 0u);
}

// ------------------------------------------------------------- long rows

// The plain copy's TMA pipeline over tiles t = (row, tile in row): each
// warp streams segments of seg_tiles consecutive tiles (its own first, then
// the next unclaimed one from the scratch's counter); lane 0 keeps kNS
// tiles in flight.
template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kTW * 32, 1)
    scan_pitched_tma_kernel(Image img, PitchedJob pj, RangeInfo ri, SingleScratch *scr,
                            cg_report *out, uint64_t tiles_per_row, uint64_t ntiles,
                            uint64_t seg_tiles) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t *wbase = smem + (size_t)wid * kWarpSmem;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kTW * kWarpSmem) + wid * kNS;
  uint64_t *segq = reinterpret_cast<uint64_t *>(smem + (size_t)kTW * kWarpSmem +
                                                 (size_t)kTW * kNS * 8) + wid * kSegQ;
  const uint64_t gw = (uint64_t)blockIdx.x * kTW + wid;
  const uint64_t nw = (uint64_t)gridDim.x * kTW;
  const uint64_t nseg = (ntiles + seg_tiles - 1) / seg_tiles;
  if (lane == 0) {
    for (int s = 0; s < kNS; s++) mbar_init(smem_addr(&bars[s]), 1);
    fence_mbar_init();
  }
  __syncwarp();
  SegSrc psrc{&scr->claim, segq, nw, 0, true};
  SegSrc csrc{&scr->claim, segq, nw, 0, false};
  uint64_t pseg = gw, cseg = gw;
  uint64_t pt = gw < nseg ? gw * seg_tiles : ntiles, ct = pt;
  uint64_t pend = pt + seg_tiles < ntiles ? pt + seg_tiles : ntiles, cend = pend;
  auto step = [&](uint64_t &seg, uint64_t &t, uint64_t &end, SegSrc &src) {
    if (++t < end) return;
    seg = src.next(seg, lane);
    t = seg < nseg ? seg * seg_tiles : ntiles;
    end = t + seg_tiles < ntiles ? t + seg_tiles : ntiles;
  };
  auto issue = [&](uint64_t t, int s) {
    const uint64_t r = t / tiles_per_row;
    const Geo g = row_geo(pj, img, KIND, r);
    issue_tile<KIND>(g, img.a_bits, (int64_t)(t - r * tiles_per_row) * kR * 32,
                     smem_addr(wbase + s * kStage), smem_addr(&bars[s]));
  };
  LaneAcc la;
  lane_acc_reset(la);
  uint32_t err = 0;
  int issued = 0;
  for (int s = 0; s < kNS && pt < ntiles; s++) {
    if (lane == 0) issue(pt, s);
    issued++;
    step(pseg, pt, pend, psrc);
  }
  uint32_t parity = 0;
  int s = 0;
  while (ct < ntiles) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), (parity >> s) & 1u);
    if (!__all_sync(CG_FULL, ok)) {
      err = 1;
      break;
    }
    parity ^= 1u << s;
    issued--;
    {
      const uint64_t r = ct / tiles_per_row;
      const Geo g = row_geo(pj, img, KIND, r);
      consume_tile<KIND, CARRY, 4, true>(g, (int64_t)(ct - r * tiles_per_row) * kR * 32,
                                wbase + s * kStage, lane, la);
    }
    __syncwarp();
    if (pt < ntiles) {
      if (lane == 0) {
        fence_proxy_async();
        issue(pt, s);
      }
      issued++;
      step(pseg, pt, pend, psrc);
    }
    step(cseg, ct, cend, csrc);
    s = s + 1 == kNS ? 0 : s + 1;
  }
  if (err) {  // drain: wait (bounded) for the copies this warp still has in flight
    for (int d = 0; d < issued; d++) {
      const int sd = (s + d) % kNS;
      mbar_wait_bounded(smem_addr(&bars[sd]), (parity >> sd) & 1u);
      parity ^= 1u << sd;
    }
  }
  single_epilogue(la, scr, ri, out, err);
}

// ------------------------------------------------ short, close rows: TMA

// Short rows that lie close together (a field of an array of records, the
// footnote's strided host read) are read as whole spans: a tile is R_T
// consecutive rows of one slice, and lane 0 bulk-copies the input V bytes
// and the host A bytes spanning them (gaps included: DRAM moves whole
// sectors anyway) into the warp's stage; groups of P lanes then classify
// and carry row after row out of shared memory.  The host picks R_T so
// both spans fit the stage's windows.
struct SpanTiles {
  uint64_t rows_per_tile;    // R_T
  uint64_t tiles_per_slice;  // ceil(height / R_T)
  uint64_t ntiles;
  uint32_t lp;               // log2 of the lanes per row
};

template <uint32_t KIND>
__device__ __forceinline__ void span_rows(const PitchedJob &pj, const SpanTiles &sp, uint64_t t,
                                          uint64_t *r_first, uint64_t *r_end) {
  const uint64_t z = t / sp.tiles_per_slice;
  const uint64_t y0 = (t - z * sp.tiles_per_slice) * sp.rows_per_tile;
  const uint64_t y1 = y0 + sp.rows_per_tile < pj.height ? y0 + sp.rows_per_tile : pj.height;
  *r_first = z * pj.height + y0;
  *r_end = z * pj.height + y1;
}

// Lane 0: queue tile t's V span and A span.
template <uint32_t KIND>
__device__ __forceinline__ void issue_span(const PitchedJob &pj, const Image &img,
                                           const SpanTiles &sp, uint64_t t, uint32_t st,
                                           uint32_t bar) {
  uint64_t r0, r1;
  span_rows<KIND>(pj, sp, t, &r0, &r1);
  const Geo g0 = row_geo(pj, img, KIND, r0);
  const Geo g1 = row_geo(pj, img, KIND, r1 - 1);
  uint32_t tx = 0, vbytes = 0, abytes = 0, voff = 0, aoff = 0;
  uintptr_t vsrc = 0;
  int64_t asrc = 0;
  if (KIND == CG_HTOD || g0.has_vin) {
    const uintptr_t vbeg = g0.vin_al;
    const uintptr_t lo = g0.vin_lo & ~(uintptr_t)15;
    uintptr_t hi = (g1.vin_hi + 15) & ~(uintptr_t)15;
    if (hi > vbeg + kVBytes) hi = vbeg + kVBytes;
    if (hi > lo) {
      vbytes = (uint32_t)(hi - lo);
      voff = (uint32_t)(lo - vbeg);
      vsrc = lo;
      tx += vbytes;
    }
  }
  if (KIND != CG_DTOD) {
    const int64_t aorig = floor16(g0.hb0 >> 3);
    const int64_t q0 = g0.hb0 > g0.hlo ? g0.hb0 : g0.hlo;
    const int64_t q1 = g1.hhi;
    if (q1 > q0) {
      const int64_t b0 = floor16(q0 >> 3);
      int64_t b1 = ceil16((q1 + 7) >> 3);
      if (b1 > aorig + (int64_t)kABytes) b1 = aorig + (int64_t)kABytes;
      abytes = (uint32_t)(b1 - b0);
      aoff = (uint32_t)(b0 - aorig);
      asrc = b0;
      tx += abytes;
    }
  }
  mbar_arrive_expect_tx(bar, tx);
  if (vbytes) bulk_g2s(st + voff, reinterpret_cast<const void *>(vsrc), vbytes, bar);
  if (abytes) bulk_g2s(st + kVBytes + aoff, img.a_bits + asrc, abytes, bar);
}

// A lane's walk over the rows of one tile: the row's anchor (the buffer the
// scan writes), input V and host positions advance by fixed steps (a tile
// lies in one slice), so each row's geometry is a few adds instead of a
// full row_geo.
struct RowCursor {
  uintptr_t anchor, vin;
  int64_t host;
  int64_t obase;
  uintptr_t d_anchor, d_vin;
  int64_t d_host, d_obase;
};

template <uint32_t KIND>
__device__ __forceinline__ RowCursor row_cursor(const PitchedJob &pj, const Image &img,
                                                uint64_t r, uint64_t step) {
  uint64_t y = r, z = 0;
  if (pj.depth > 1) {
    z = r / pj.height;
    y = r - z * pj.height;
  }
  const bool carry = pj.mode & kModeCarry;
  const uint64_t host_off = pj.host_start + z * pj.host_slice + y * pj.host_pitch;
  const uintptr_t host_v = reinterpret_cast<uintptr_t>(img.v) + host_off;
  const uintptr_t src = pj.src_start + z * pj.src_slice + y * pj.src_pitch;
  const uintptr_t dst = pj.dst_start + z * pj.dst_slice + y * pj.dst_pitch;
  RowCursor c;
  c.host = (int64_t)host_off;
  c.d_host = (int64_t)(step * pj.host_pitch);
  c.obase = (int64_t)(r * pj.width);
  c.d_obase = (int64_t)(step * pj.width);
  if (KIND == CG_HTOD) {
    c.vin = host_v;
    c.d_vin = step * pj.host_pitch;
  } else {
    c.vin = src;
    c.d_vin = step * pj.src_pitch;
  }
  if (KIND == CG_DTOH || (KIND == CG_HTOD && !carry)) {
    c.anchor = host_v;
    c.d_anchor = step * pj.host_pitch;
  } else if (carry) {
    c.anchor = dst;
    c.d_anchor = step * pj.dst_pitch;
  } else {
    c.anchor = src;
    c.d_anchor = step * pj.src_pitch;
  }
  return c;
}


// All lanes: the rows of tile t out of stage `sp_mem`.
template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ void consume_span(const PitchedJob &pj, const Image &img,
                                             const SpanTiles &sp, uint64_t t,
                                             const uint8_t *sp_mem, int lane, LaneAcc &la) {
  uint64_t r0, r1;
  span_rows<KIND>(pj, sp, t, &r0, &r1);
  const Geo g0 = row_geo(pj, img, KIND, r0);
  const uintptr_t vbeg = g0.vin_al;
  const int64_t aorig = floor16(g0.hb0 >> 3);
  const uint4 *vs = reinterpret_cast<const uint4 *>(sp_mem);
  const uint32_t *as = reinterpret_cast<const uint32_t *>(sp_mem + kVBytes);
  const uint32_t P = 1u << sp.lp;
  const uint64_t step = 32u >> sp.lp;
  const int64_t c = lane & (P - 1);
  uint64_t r = r0 + (lane >> sp.lp);
  if (r >= r1) return;
  RowCursor cur = row_cursor<KIND>(pj, img, r, step);
  const bool has_vin = g0.has_vin;
  // per row, in 32 bits: its V start from the stage's V window start (a
  // 16-byte-aligned address), its first host byte, which is also its first
  // A bit, from the A window's first bit, and its anchor alignment; only
  // the carry's store address and the copy offset stay 64-bit
  int32_t vrel = (int32_t)(cur.vin - vbeg);
  int32_t hrel = (int32_t)(cur.host - 8 * aorig);
  const int32_t d_vrel = (int32_t)cur.d_vin, d_hrel = (int32_t)cur.d_host;
  const int32_t c32 = (int32_t)c;
  Geo g;  // the fields chunk_step reads: n, ax, out_al, obase
  g.n = pj.width;
  for (; r < r1; r += step) {
    const int32_t ax = (int32_t)(cur.anchor & 15);
    g.ax = ax;
    g.out_al = reinterpret_cast<uint8_t *>(cur.anchor - (uintptr_t)ax);
    g.obase = cur.obase;
    uint4 V = make_uint4(0, 0, 0, 0);
    if (KIND == CG_HTOD || has_vin) {
      const int32_t vw = vrel - ax;  // aligned window start = vw rounded down to 16
      const int32_t k = (vw >> 4) + c32;
      V = vs[k];
      const int vin_r = vw & 15;
      if (vin_r) V = funnel16(V, vs[k + 1], vin_r);
    }
    uint32_t a16 = 0xFFFFu;
    if (KIND != CG_DTOD) {
      const int32_t qb = hrel - ax + 16 * c32;
      const int sh = qb & 31;
      const int wi = qb >> 5;
      const uint32_t w0 = as[wi];
      const uint32_t w1 = sh > 16 ? as[wi + 1] : 0u;
      a16 = __funnelshift_r(w0, w1, sh) & 0xFFFFu;
    }
    chunk_step<KIND, CARRY>(g, c, V, a16, valid_mask(16 * c - ax, g.n), la);
    cur.anchor += cur.d_anchor;
    vrel += d_vrel;
    hrel += d_hrel;
    cur.obase += cur.d_obase;
  }
}

template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kTW * 32, 1)
    scan_pitched_span_kernel(Image img, PitchedJob pj, RangeInfo ri, SingleScratch *scr,
                             cg_report *out, SpanTiles sp) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t *wbase = smem + (size_t)wid * kWarpSmem;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kTW * kWarpSmem) + wid * kNS;
  const uint64_t gw = (uint64_t)blockIdx.x * kTW + wid;
  const uint64_t nw = (uint64_t)gridDim.x * kTW;
  if (lane == 0) {
    for (int s = 0; s < kNS; s++) mbar_init(smem_addr(&bars[s]), 1);
    fence_mbar_init();
  }
  __syncwarp();
  LaneAcc la;
  lane_acc_reset(la);
  uint32_t err = 0;
  if (lane == 0)
    for (int s = 0; s < kNS; s++) {
      const uint64_t t = gw + (uint64_t)s * nw;
      if (t < sp.ntiles)
        issue_span<KIND>(pj, img, sp, t, smem_addr(wbase + s * kStage), smem_addr(&bars[s]));
    }
  uint32_t parity = 0;
  int s = 0;
  uint64_t t = gw;
  for (; t < sp.ntiles; t += nw) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), (parity >> s) & 1u);
    if (!__all_sync(CG_FULL, ok)) {
      err = 1;
      break;
    }
    parity ^= 1u << s;
    consume_span<KIND, CARRY>(pj, img, sp, t, wbase + s * kStage, lane, la);
    __syncwarp();
    const uint64_t tn = t + (uint64_t)kNS * nw;
    if (lane == 0 && tn < sp.ntiles) {
      fence_proxy_async();
      issue_span<KIND>(pj, img, sp, tn, smem_addr(wbase + s * kStage), smem_addr(&bars[s]));
    }
    s = s + 1 == kNS ? 0 : s + 1;
  }
  if (err) {  // drain: wait (bounded) for the copies this warp still has in flight
    for (int d = 0; d < kNS; d++) {
      const uint64_t td = t + (uint64_t)d * nw;
      if (td >= sp.ntiles) break;
      const int sd = (s + d) % kNS;
      mbar_wait_bounded(smem_addr(&bars[sd]), (parity >> sd) & 1u);
      parity ^= 1u << sd;
    }
  }
  single_epilogue(la, scr, ri, out, err);
}

// Rows per span tile when every row is read by `lanes` lanes (one chunk
// each), or 0 when fewer than two rows fit (then the register kernel reads
// row by row).  Bounds: every row's V window (its aligned start, one chunk
// per lane and one more vector) stays inside
// the stage's V window from the first row's aligned start, with 62 bytes of
// alignment slack; every row's A words (two per chunk position) inside the
// A window from the first row's aligned A byte, with slack.
static uint64_t span_rows_per_tile(const PitchedJob &job, uint64_t lanes) {
  if (job.height < 2) return 0;
  uint64_t rt = job.height;
  const bool reads_v = job.kind == CG_HTOD || (job.mode & kModeReadDev);
  if (reads_v) {
    const uint64_t pv = job.kind == CG_HTOD ? job.host_pitch : job.src_pitch;
    const int64_t room = (int64_t)kVBytes - 62 - 16 * (int64_t)lanes;
    if (room < 0 || pv == 0) return 0;
    const uint64_t r = (uint64_t)room / pv + 1;
    rt = r < rt ? r : rt;
  }
  if (job.kind != CG_DTOD) {
    const int64_t room = ((int64_t)kABytes - 32) * 8 - 15 - 16 * (int64_t)lanes;
    if (room < 0 || job.host_pitch == 0) return 0;
    const uint64_t r = (uint64_t)room / job.host_pitch + 1;
    rt = r < rt ? r : rt;
  }
  return rt >= 2 ? rt : 0;
}

// --------------------------------------------------------------- launch

template <uint32_t KIND, bool CARRY>
static cudaError_t launch_t(const Image &img, const PitchedJob &job, const RangeInfo &ri,
                            SingleScratch *scr, cg_report *out, int sm_count, uint64_t kmax,
                            bool tma_ok, cudaStream_t st) {
  const uint64_t rows = job.height * job.depth;
  const uint64_t wpc = kPThreads / 32;
  if (kmax >= kTmaRowChunks && tma_ok) {
    constexpr size_t smem = kSmemBytes + (size_t)kTW * kSegQ * 8;
    static KernelSetup setup;
    int per_sm = 1;
    const cudaError_t e = kernel_setup(setup, scan_pitched_tma_kernel<KIND, CARRY>, kTW * 32, smem,
                                       &per_sm);
    if (e != cudaSuccess) return e;
    const uint64_t tpr = (kmax + 32 * kR - 1) / (32 * kR);
    const uint64_t ntiles = rows * tpr;
    const uint64_t need = (ntiles + kTW - 1) / kTW;
    const uint64_t cap = (uint64_t)sm_count * per_sm;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    // segments of up to 16 tiles, at least about four per warp
    uint64_t seg_tiles = ntiles / (4 * (uint64_t)grid * kTW);
    seg_tiles = seg_tiles < 1 ? 1 : (seg_tiles > 16 ? 16 : seg_tiles);
    scan_pitched_tma_kernel<KIND, CARRY><<<grid, kTW * 32, smem, st>>>(img, job, ri, scr, out, tpr,
                                                                       ntiles, seg_tiles);
    return cudaGetLastError();
  }
  if (kmax > 32) {
    static KernelSetup setup;
    int per_sm = 1;
    const cudaError_t e = kernel_setup(setup, scan_pitched_wide_kernel<KIND, CARRY>, kPThreads, 0,
                                       &per_sm);
    if (e != cudaSuccess) return e;
    WideStep ws;
    ws.groups = (kmax + 32 * kPWide - 1) / (32 * kPWide);
    const uint64_t items = rows * ws.groups;
    const uint64_t need = (items + wpc - 1) / wpc;
    const uint64_t cap = (uint64_t)sm_count * per_sm;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    const uint64_t T = (uint64_t)grid * wpc;
    ws.tg = T % ws.groups;
    ws.tr = T / ws.groups;
    scan_pitched_wide_kernel<KIND, CARRY><<<grid, kPThreads, 0, st>>>(img, job, ri, scr, out, ws);
    return cudaGetLastError();
  }
  uint32_t lp = 0;
  while ((1ull << lp) < kmax) lp++;
  const uint64_t rt = tma_ok ? span_rows_per_tile(job, 1ull << lp) : 0;
  if (rt) {
    static KernelSetup setup;
    int span_per_sm = 1;
    const cudaError_t e = kernel_setup(setup, scan_pitched_span_kernel<KIND, CARRY>, kTW * 32,
                                       kSmemBytes, &span_per_sm);
    if (e != cudaSuccess) return e;
    SpanTiles sp;
    sp.rows_per_tile = rt;
    sp.tiles_per_slice = (job.height + rt - 1) / rt;
    sp.ntiles = sp.tiles_per_slice * job.depth;
    sp.lp = lp;
    const uint64_t need = (sp.ntiles + kTW - 1) / kTW;
    const uint64_t cap = (uint64_t)sm_count * span_per_sm;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    scan_pitched_span_kernel<KIND, CARRY><<<grid, kTW * 32, kSmemBytes, st>>>(img, job, ri, scr,
                                                                              out, sp);
    return cudaGetLastError();
  }
  static KernelSetup setup;
  int per_sm = 1;
  const cudaError_t e = kernel_setup(setup, scan_pitched_narrow_kernel<KIND, CARRY>, kPThreads, 0,
                                     &per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t per_warp = (32ull >> lp) * kPNarrow;
  const uint64_t need = (rows + per_warp * wpc - 1) / (per_warp * wpc);
  const uint64_t cap = (uint64_t)sm_count * per_sm;
  const unsigned grid = (unsigned)(need < cap ? need : cap);
  scan_pitched_narrow_kernel<KIND, CARRY><<<grid, kPThreads, 0, st>>>(img, job, ri, scr, out, lp);
  return cudaGetLastError();
}

cudaError_t launch_scan_pitched(const Image &img, const PitchedJob &job, const RangeInfo &ri,
                                SingleScratch *scr, cg_report *out, int sm_count,
                                uint64_t row_chunks, bool tma_ok, cudaStream_t st) {
  const bool carry = job.mode & kModeCarry;
  switch (job.kind) {
    case CG_HTOD:
      return carry ? launch_t<CG_HTOD, true>(img, job, ri, scr, out, sm_count, row_chunks, tma_ok, st)
                   : launch_t<CG_HTOD, false>(img, job, ri, scr, out, sm_count, row_chunks, tma_ok, st);
    case CG_DTOH:
      return carry ? launch_t<CG_DTOH, true>(img, job, ri, scr, out, sm_count, row_chunks, tma_ok, st)
                   : launch_t<CG_DTOH, false>(img, job, ri, scr, out, sm_count, row_chunks, tma_ok, st);
    default:
      return carry ? launch_t<CG_DTOD, true>(img, job, ri, scr, out, sm_count, row_chunks, tma_ok, st)
                   : launch_t<CG_DTOD, false>(img, job, ri, scr, out, sm_count, row_chunks, tma_ok, st);
  }
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

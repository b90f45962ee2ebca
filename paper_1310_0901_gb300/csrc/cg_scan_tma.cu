// cg_scan_tma.cu -- the single-copy scan with its loads on the TMA engine.
//
// Every warp runs its own pipeline of kNS shared-memory stages (16 warps
// per CTA, 2 stages of 5 KiB tiles: 16 warps hide the classification
// latency on error-dense data, 2 stages keep enough bytes in flight).  Lane 0
// issues 1-D bulk copies (cp.async.bulk, completion counted on an mbarrier)
// of the next tiles' V and A bytes; all 32 lanes wait on the stage's
// mbarrier, classify and carry the tile out of shared memory, and hand the
// stage back.  Bytes in flight no longer cost registers, so a few warps per
// SM keep HBM busy.  A tile is kR warp rows (kR x 512 bytes of the anchor
// grid).  Misaligned input streams are realigned when read from shared
// memory (two aligned 16-byte reads and a byte funnel shift).
//
// Every wait is bounded (about one second of %globaltimer); on expiry the
// warp stops, waits (bounded again) for its copies still in flight, and the
// report is flagged CG_F_INCOMPLETE.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_setup.h"
#include "cg_tma.cuh"
#include "cg_launch.h"

namespace cgi {

// A single copy is cut into segments of seg_tiles consecutive tiles: each
// warp streams its own segment (contiguous reads and writes) and then
// claims the next unclaimed one from the scratch's counter, which the last
// CTA resets.  Against tiles dealt to the warps in turn this took a 4 GiB
// host-to-device check with carry from 6.2 to 6.8 TB/s.
template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kTW * 32, 1)
    scan_single_tma_kernel(Image img, ScanJob job, RangeInfo ri, SingleScratch *scr,
                           cg_report *out, int64_t seg_tiles) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t *wbase = smem + (size_t)wid * kWarpSmem;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kTW * kWarpSmem) + wid * kNS;
  uint64_t *segq = reinterpret_cast<uint64_t *>(smem + (size_t)kTW * kWarpSmem +
                                                 (size_t)kTW * kNS * 8) + wid * kSegQ;
  const Geo g = make_geo(job, img);
  const bool aonly = a_only<KIND, CARRY>(g);  // super-tiles of A bits alone
  const int64_t rows = ((aonly ? super_chunks(g) : g.nchunks) + 31) >> 5;
  const int64_t ntiles = (rows + kR - 1) / kR;
  const uint64_t nseg = (uint64_t)((ntiles + seg_tiles - 1) / seg_tiles);
  const uint64_t gw = (uint64_t)blockIdx.x * kTW + wid;
  const uint64_t nw = (uint64_t)gridDim.x * kTW;
  if (lane == 0) {
    for (int s = 0; s < kNS; s++) mbar_init(smem_addr(&bars[s]), 1);
    fence_mbar_init();
  }
  __syncwarp();
  SegSrc psrc{&scr->claim, segq, nw, 0, true};
  SegSrc csrc{&scr->claim, segq, nw, 0, false};
  // producer and consumer positions: segment, tile, end of the segment
  uint64_t pseg = gw, cseg = gw;
  int64_t pt = (int64_t)gw * seg_tiles, ct = pt;
  int64_t pend = pt + seg_tiles < ntiles ? pt + seg_tiles : ntiles, cend = pend;
  auto step = [&](uint64_t &seg, int64_t &t, int64_t &end, SegSrc &src) {
    if (++t < end) return;
    seg = src.next(seg, lane);
    t = seg < nseg ? (int64_t)seg * seg_tiles : ntiles;
    end = t + seg_tiles < ntiles ? t + seg_tiles : ntiles;
  };
  auto issue = [&](int64_t t, int s, bool stall) {
    if (stall)  // injected: expect bytes, copy none
      mbar_arrive_expect_tx(smem_addr(&bars[s]), 16);
    else if (aonly)
      issue_tile_a_super(g, img.a_bits, t * kR * 32, smem_addr(wbase + s * kStage),
                         smem_addr(&bars[s]));
    else
      issue_tile<KIND>(g, img.a_bits, t * kR * 32, smem_addr(wbase + s * kStage),
                       smem_addr(&bars[s]));
  };
  LaneAcc la;
  lane_acc_reset(la);
  uint32_t err = 0;
  int issued = 0;
  for (int s = 0; s < kNS && pt < ntiles; s++) {
    if (lane == 0) issue(pt, s, (job.mode & kModeStall) && gw == 0 && s == 0);
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
    if (aonly)
      consume_tile_a_super(g, ct * kR * 32, wbase + s * kStage, lane, la);
    else
      consume_tile<KIND, CARRY>(g, ct * kR * 32, wbase + s * kStage, lane, la);
    __syncwarp();
    if (pt < ntiles) {
      if (lane == 0) {
        fence_proxy_async();
        issue(pt, s, false);
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


template <uint32_t KIND, bool CARRY>
static cudaError_t launch_tma_t(const Image &img, const ScanJob &job, const RangeInfo &ri,
                                SingleScratch *scr, cg_report *out, int grid, cudaStream_t st) {
  constexpr size_t smem = kSmemBytes + (size_t)kTW * kSegQ * 8;
  static KernelSetup setup;
  int per_sm = 1;
  const cudaError_t e = kernel_setup(setup, scan_single_tma_kernel<KIND, CARRY>, kTW * 32, smem,
                                     &per_sm);
  if (e != cudaSuccess) return e;
  // `grid` counts SM-sized units of work; fill every resident CTA slot
  const unsigned ctas = (unsigned)(grid * per_sm);
  // segments of up to 16 tiles (64 KiB of the anchor grid), and at least
  // about four per warp so that claims even out the end of the copy
  const uint64_t chunks = (job.n + 30) >> 4;  // an upper bound for any kind
  const int64_t tiles = (int64_t)((chunks + 32 * kR - 1) / (32 * kR));
  int64_t seg_tiles = tiles / (4 * (int64_t)ctas * kTW);
  seg_tiles = seg_tiles < 1 ? 1 : (seg_tiles > 16 ? 16 : seg_tiles);
  scan_single_tma_kernel<KIND, CARRY><<<ctas, kTW * 32, smem, st>>>(img, job, ri, scr, out,
                                                                    seg_tiles);
  return cudaGetLastError();
}

cudaError_t launch_scan_single_tma(const Image &img, const ScanJob &job, const RangeInfo &ri,
                                   SingleScratch *scr, cg_report *out, int grid,
                                   cudaStream_t st) {
  const bool carry = job.mode & kModeCarry;
  switch (job.kind) {
    case CG_HTOD:
      return carry ? launch_tma_t<CG_HTOD, true>(img, job, ri, scr, out, grid, st)
                   : launch_tma_t<CG_HTOD, false>(img, job, ri, scr, out, grid, st);
    case CG_DTOH:
      return carry ? launch_tma_t<CG_DTOH, true>(img, job, ri, scr, out, grid, st)
                   : launch_tma_t<CG_DTOH, false>(img, job, ri, scr, out, grid, st);
    default:
      return carry ? launch_tma_t<CG_DTOD, true>(img, job, ri, scr, out, grid, st)
                   : launch_tma_t<CG_DTOD, false>(img, job, ri, scr, out, grid, st);
  }
}

uint32_t scan_tma_tile_bytes() { return 512u * kR; }

int scan_single_tma_grid(int sm_count, uint64_t n) {
  // tiles of kR rows over kTW-warp CTAs, in SM units (the launch multiplies
  // by the CTAs resident per SM)
  const uint64_t tiles = ((n + 30) / 16 / 32 + kR) / kR + 1;
  const uint64_t ctas = (tiles + kTW - 1) / kTW;
  return (int)(ctas < (uint64_t)sm_count ? (ctas ? ctas : 1) : (uint64_t)sm_count);
}

}  // namespace cgi

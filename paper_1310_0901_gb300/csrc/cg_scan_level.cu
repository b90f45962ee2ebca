// cg_scan_level.cu -- one dependency level of a batch on the TMA engine.
//
// The level's copies are cut into segments; each warp runs its own
// pipeline of kNS shared-memory stages (as the single-copy kernel) over the
// segments it takes, classifies and carries each tile out of shared memory
// and adds its counts to the copy's accumulator.  Every wait is bounded;
// on expiry the warp drains its copies in flight and raises the batch's
// error flag.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_setup.h"
#include "cg_tma.cuh"
#include "cg_launch.h"

namespace cgi {

// ------------------------------------------------ batched: one level

// The tiles a warp processes in one level, in order: segment w first,
// then either segments w + W, w + 2W, ... (static) or, with a claim
// counter, the next unclaimed segment each time (dynamic: a warp that drew
// cheap segments takes more, so the level ends with every warp busy to its
// last segment).  Either way a warp's segments increase, and each
// segment's tiles are taken in turn.  The copy owning a segment is found by
// one binary search per warp, then by galloping forward from the previous
// copy.  Only the producer side of a warp walks this sequence (kNS tiles
// ahead): with each tile it issues it leaves a descriptor in the stage (the
// copy's order position and the tile's index), and the consumer side
// follows the descriptors.  (Claiming one segment ahead, to hide the
// atomic's latency, lengthened each level's tail: slower on error-dense
// batches.)
#ifndef CG_LEVEL_UNROLL
#define CG_LEVEL_UNROLL 2
#endif
constexpr int kLevelUnroll = CG_LEVEL_UNROLL;  // rows unrolled per consumed tile

struct SegIter {
  uint64_t s;      // current segment id
  uint64_t pos;    // order position of the current copy
  uint64_t first;  // its first segment id
  uint64_t next;   // first segment id of the next position (or ~0)
  uint32_t req;    // its request
  ScanJob job;
  Geo g;
  int64_t t, t_end;  // tile range of the segment
  int64_t rlo, rhi;  // rows of the copy the position covers (hi = -1: to the copy's end)
  bool valid;
};

// Segment claims of the level kernel's producer: static striding (no
// counter) or the next unclaimed segment from the level's counter.
struct LevelClaims {
  unsigned long long *ctr;
  uint64_t step;  // W
  __device__ __forceinline__ uint64_t next(uint64_t cur, int lane) {
    if (!ctr) return cur + step;
    uint64_t v = 0;
    if (lane == 0) v = step + atomicAdd(ctr, 1ull);
    return __shfl_sync(CG_FULL, v, 0);
  }
};

// A stage's tile as the producer issued it.
struct TileDesc {
  uint64_t pos;  // order position of its copy
  int64_t t;     // tile index within the copy
};

__device__ __forceinline__ void seg_set_pos(SegIter &it, const BatchPlan &p, const Image &img,
                                            uint64_t pos, uint64_t pos_end) {
  it.pos = pos;
  it.first = __ldg(p.seg_first + pos);
  it.next = pos + 1 < pos_end ? __ldg(p.seg_first + pos + 1) : ~0ull;
  it.req = __ldg(p.order + pos);
  const uint64_t pc = p.piece ? __ldg(p.piece + pos) : 0ull;
  it.rlo = pc ? (int64_t)(pc & 0xFFFFFFFFull) : 0;
  it.rhi = pc ? (int64_t)(pc >> 32) : -1;
  it.job = p.jobs[it.req];
  it.job.mode &= p.mode_mask;
  it.g = make_geo(it.job, img);
}

// last position in [lo, hi) whose first segment is <= s, given that
// position lo qualifies
__device__ __forceinline__ uint64_t seg_search(const BatchPlan &p, uint64_t lo, uint64_t hi,
                                               uint64_t s) {
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(p.seg_first + mid) <= s)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Settle on segment it.s (or the first non-empty one after it).
__device__ __forceinline__ void seg_settle(SegIter &it, const BatchPlan &p, const Image &img,
                                           uint64_t pos_end, uint64_t n_segs, LevelClaims &src,
                                           int lane) {
  const int64_t seg_rows = p.seg_chunks >> 5;
  while (it.s < n_segs) {
    if (it.s >= it.next) {  // gallop forward from the next position
      uint64_t lo = it.pos + 1, span = 1, hi = lo + 1;
      while (hi < pos_end && __ldg(p.seg_first + hi) <= it.s) {
        lo = hi;
        span <<= 1;
        hi = lo + span;
      }
      if (hi > pos_end) hi = pos_end;
      seg_set_pos(it, p, img, seg_search(p, lo, hi, it.s), pos_end);
    }
    const int64_t k = (int64_t)(it.s - it.first);
    const bool aonly = it.job.kind == CG_DTOH && !(it.job.mode & (kModeCarry | kModeReadDev));
    const int64_t rows =
        it.rhi >= 0 ? it.rhi : ((aonly ? super_chunks(it.g) : it.g.nchunks) + 31) >> 5;
    const int64_t r0 = it.rlo + k * seg_rows;
    const int64_t r1 = r0 + seg_rows < rows ? r0 + seg_rows : rows;
    if (r0 < r1) {
      it.t = r0 / kR;
      it.t_end = (r1 + kR - 1) / kR;
      it.valid = true;
      return;
    }
    it.s = src.next(it.s, lane);  // an empty trailing segment (the count was an upper bound)
  }
  it.valid = false;
}

__device__ __forceinline__ void seg_begin(SegIter &it, const BatchPlan &p, const Image &img,
                                          uint64_t pos_begin, uint64_t pos_end, uint64_t n_segs,
                                          uint64_t s, LevelClaims &src, int lane) {
  it.s = s;
  it.valid = false;
  if (s >= n_segs) return;
  seg_set_pos(it, p, img, seg_search(p, pos_begin, pos_end, s), pos_end);
  seg_settle(it, p, img, pos_end, n_segs, src, lane);
}

__device__ __forceinline__ void seg_advance(SegIter &it, const BatchPlan &p, const Image &img,
                                            uint64_t pos_end, uint64_t n_segs, LevelClaims &src,
                                            int lane) {
  if (++it.t < it.t_end) return;
  it.s = src.next(it.s, lane);
  seg_settle(it, p, img, pos_end, n_segs, src, lane);
}

__device__ __forceinline__ void seg_issue(const SegIter &it, const uint8_t *a_bits, uint32_t st,
                                          uint32_t bar) {
  const int64_t c0 = it.t * kR * 32;
  switch (it.job.kind) {
    case CG_HTOD:
      issue_tile<CG_HTOD>(it.g, a_bits, c0, st, bar);
      break;
    case CG_DTOH:
      if (!(it.job.mode & (kModeCarry | kModeReadDev)))
        issue_tile_a_super(it.g, a_bits, c0, st, bar);
      else
        issue_tile<CG_DTOH>(it.g, a_bits, c0, st, bar);
      break;
    default:
      issue_tile<CG_DTOD>(it.g, a_bits, c0, st, bar);
      break;
  }
}

__device__ __forceinline__ void tile_consume(const ScanJob &job, const Geo &g, int64_t t,
                                             const uint8_t *sp, int lane, LaneAcc &la) {
  const int64_t c0 = t * kR * 32;
  const bool carry = job.mode & kModeCarry;
  switch (job.kind) {
    case CG_HTOD:
      if (carry)
        consume_tile<CG_HTOD, true, kLevelUnroll>(g, c0, sp, lane, la);
      else
        consume_tile<CG_HTOD, false, kLevelUnroll>(g, c0, sp, lane, la);
      break;
    case CG_DTOH:
      if (carry)
        consume_tile<CG_DTOH, true, kLevelUnroll>(g, c0, sp, lane, la);
      else if (!(job.mode & kModeReadDev))
        consume_tile_a_super(g, c0, sp, lane, la);
      else
        consume_tile<CG_DTOH, false, kLevelUnroll>(g, c0, sp, lane, la);
      break;
    default:
      if (carry)
        consume_tile<CG_DTOD, true, kLevelUnroll>(g, c0, sp, lane, la);
      else
        consume_tile<CG_DTOD, false, kLevelUnroll>(g, c0, sp, lane, la);
      break;
  }
}

__global__ void __launch_bounds__(kTW * 32, 1)
    scan_level_tma_kernel(Image img, BatchPlan p, uint64_t pos_begin, uint64_t pos_end,
                          uint64_t n_segs, unsigned long long *claim, unsigned int *err_flag,
                          FinalizeHost fin) {
  // levels launched back to back may overlap: the next level's grid is
  // scheduled as this one's CTAs leave, runs its prologue (which reads only
  // the batch's plan), and waits for this grid before touching any shadow
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t *wbase = smem + (size_t)wid * kWarpSmem;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kTW * kWarpSmem) + wid * kNS;
  TileDesc *desc = reinterpret_cast<TileDesc *>(smem + (size_t)kTW * kWarpSmem +
                                                 (size_t)kTW * kNS * 8) + wid * kNS;
  const uint64_t gw = (uint64_t)blockIdx.x * kTW + wid;
  const uint64_t nw = (uint64_t)gridDim.x * kTW;
  if (lane == 0) {
    for (int s = 0; s < kNS; s++) mbar_init(smem_addr(&bars[s]), 1);
    fence_mbar_init();
  }
  __syncwarp();
  LevelClaims src{claim, nw};
  SegIter prod;
  seg_begin(prod, p, img, pos_begin, pos_end, n_segs, gw, src, lane);
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous level is complete
  auto issue = [&](int s) {  // lane 0: the producer's tile into stage s
    desc[s] = TileDesc{prod.pos, prod.t};
    seg_issue(prod, img.a_bits, smem_addr(wbase + s * kStage), smem_addr(&bars[s]));
  };
  int issued = 0;
  for (int s = 0; s < kNS && prod.valid; s++) {
    if (lane == 0) issue(s);
    issued++;
    seg_advance(prod, p, img, pos_end, n_segs, src, lane);
  }
  LaneAcc la;
  lane_acc_reset(la);
  uint32_t parity = 0;
  int stage = 0;
  bool failed = false;
  // the copy being consumed (cpos = ~0: none yet)
  uint64_t cpos = ~0ull;
  uint32_t creq = 0;
  ScanJob cjob{};
  Geo cgeo{};
  while (issued > 0) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[stage]), (parity >> stage) & 1u);
    if (!__all_sync(CG_FULL, ok)) {
      failed = true;
      break;
    }
    parity ^= 1u << stage;
    issued--;
    const TileDesc d = desc[stage];
    if (d.pos != cpos) {
      // a warp's tiles go forward through the level's copies, so it never
      // comes back to a copy it left: its counts for that copy are flushed
      // when the copy changes
      if (cpos != ~0ull) warp_flush(la, &p.acc[creq], lane);
      cpos = d.pos;
      creq = __ldg(p.order + cpos);
      cjob = p.jobs[creq];
      cjob.mode &= p.mode_mask;
      cgeo = make_geo(cjob, img);
    }
    tile_consume(cjob, cgeo, d.t, wbase + stage * kStage, lane, la);
    __syncwarp();
    if (prod.valid) {
      if (lane == 0) {
        fence_proxy_async();
        issue(stage);
      }
      issued++;
      seg_advance(prod, p, img, pos_end, n_segs, src, lane);
    }
    stage = stage + 1 == kNS ? 0 : stage + 1;
  }
  if (cpos != ~0ull) warp_flush(la, &p.acc[creq], lane);
  if (failed) {  // drain the copies still in flight, bounded
    for (int d = 0; d < issued; d++) {
      const int sd = (stage + d) % kNS;
      mbar_wait_bounded(smem_addr(&bars[sd]), (parity >> sd) & 1u);
      parity ^= 1u << sd;
    }
    if (lane == 0) atomicOr(err_flag, 1u);
  }
  if (fin.out) {  // the last CTA to finish writes every report to the host
    __shared__ bool s_last;
    __threadfence();  // this thread's accumulator atomics before the count
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(fin.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      for (uint64_t i = threadIdx.x; i < p.nreq; i += blockDim.x) {
        Acc a;
        a.n_unaddr = __ldcg(&p.acc[i].n_unaddr);
        a.n_undef = __ldcg(&p.acc[i].n_undef);
        a.first_unaddr = __ldcg(&p.acc[i].first_unaddr);
        a.first_undef = __ldcg(&p.acc[i].first_undef);
        cg_report r;
        assemble_report(&r, p.info[i], a);
        reinterpret_cast<cg_report *>(fin.out + 16)[i] = r;
      }
      if (threadIdx.x == 0) *reinterpret_cast<unsigned int *>(fin.out) = __ldcg(err_flag);
    }
  }
}

cudaError_t launch_scan_level_tma(const Image &img, const BatchPlan &p, uint64_t pos_begin,
                                  uint64_t pos_end, uint64_t n_segs, int max_ctas,
                                  unsigned long long *claim, unsigned int *err_flag, bool overlap,
                                  cudaStream_t st, const FinalizeHost &fin) {
  if (n_segs == 0 || pos_end <= pos_begin) return cudaSuccess;
  constexpr size_t smem = kSmemBytes + (size_t)kTW * kNS * sizeof(TileDesc);
  static KernelSetup setup;
  int per_sm = 1;
  const cudaError_t e = kernel_setup(setup, scan_level_tma_kernel, kTW * 32, smem, &per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t cap = (uint64_t)max_ctas * (uint64_t)per_sm;  // max_ctas counts SMs
  const uint64_t ctas = (n_segs + kTW - 1) / kTW;
  const unsigned g = (unsigned)(ctas < cap ? ctas : cap);
  if (overlap) {  // programmatic dependent launch after the previous level
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
    cfg.blockDim = dim3(kTW * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, scan_level_tma_kernel, img, p, pos_begin, pos_end, n_segs,
                              claim, err_flag, fin);
  }
  scan_level_tma_kernel<<<g, kTW * 32, smem, st>>>(img, p, pos_begin, pos_end, n_segs, claim,
                                                   err_flag, fin);
  return cudaGetLastError();
}

}  // namespace cgi

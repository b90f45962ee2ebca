// cg_devops.cpp -- the memset wrappers' check and kernel-argument checks.
//
// A memset is one range check on the host mirror plus a fill of the written
// bytes' V shadow with zeros (one launch).  The arguments of a kernel launch
// are checked together: their ranges on the host mirror (as single checks),
// then on the GPU the batched scan kernel counts the undefined bytes of
// in-range read arguments (one level: nothing is carried, every read sees
// the state before the launch), a finalize kernel writes the reports into
// pinned host memory, and a fill kernel defines the in-range write
// arguments.  One upload, three launches, one synchronisation.
#include <cuda_runtime.h>

#include "cg_ctx.h"

using namespace cgi;

namespace {

bool mul_over(uint64_t a, uint64_t b, uint64_t *out) { return __builtin_mul_overflow(a, b, out); }
bool add_over(uint64_t a, uint64_t b, uint64_t *out) { return __builtin_add_overflow(a, b, out); }

struct MemsetPlan {
  RangeInfo ri{};
  bool fill = false;
  uint64_t shadow = 0;
};

cg_status prepare_memset(cg_ctx *c, uint64_t dptr, uint64_t pitch, uint64_t width,
                         uint64_t height, MemsetPlan *M) {
  if (height > 1 && pitch < width) return set_error(CG_E_ARG, "pitch smaller than the row width");
  uint64_t n = 0;
  if (mul_over(width, height, &n)) return set_error(CG_E_WRAP, "width*height exceeds 64 bits");
  M->ri = RangeInfo{};
  M->ri.kind = CG_DTOD;
  M->ri.n = n;
  M->fill = false;
  if (n == 0) return CG_OK;  // R9
  uint64_t rows_span = 0, ext = 0;
  if (mul_over(height - 1, pitch, &rows_span) || add_over(rows_span, width, &ext))
    return set_error(CG_E_WRAP, "memset extent exceeds 64 bits");
  const bool ok = host_side(c, dptr, ext, &M->ri.found_dst, &M->ri.base_dst, &M->ri.size_dst,
                            &M->shadow, &M->ri.flags, CG_F_UNALLOC_DST, CG_F_OVERRUN_DST);
  M->fill = ok && c->cfg.carry;
  return CG_OK;
}

cg_status enqueue_memset(cg_ctx *c, const MemsetPlan &M, uint64_t pitch, uint64_t width,
                         uint64_t height, cg_report *rep_dev, cudaStream_t st) {
  CG_TRY(flush_fills(c, st));
  if (!M.fill && !rep_dev) return CG_OK;
  CG_CUDA(launch_fill_rows(reinterpret_cast<uint8_t *>(M.shadow), pitch, M.fill ? width : 0,
                           M.fill ? height : 0, 0x00, M.ri, rep_dev, c->sm_count, st));
  c->stats.kernels++;
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_check_memset(cg_ctx *c, uint64_t dptr, uint64_t pitch, uint64_t width,
                          uint64_t height, cg_report *rep, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !rep) return set_error(CG_E_ARG, "NULL argument");
  MemsetPlan M;
  CG_TRY(prepare_memset(c, dptr, pitch, width, height, &M));
  CG_TRY(enqueue_memset(c, M, pitch, width, height, nullptr, static_cast<cudaStream_t>(stream)));
  const Acc none{0, 0, kNone, kNone};
  assemble_report(rep, M.ri, none);
  count_stats(c, *rep);
  return CG_OK;
}

cg_status cg_check_memset_async(cg_ctx *c, uint64_t dptr, uint64_t pitch, uint64_t width,
                                uint64_t height, cg_report *rep_dev, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !rep_dev) return set_error(CG_E_ARG, "NULL argument");
  MemsetPlan M;
  CG_TRY(prepare_memset(c, dptr, pitch, width, height, &M));
  CG_TRY(enqueue_memset(c, M, pitch, width, height, rep_dev, static_cast<cudaStream_t>(stream)));
  c->stats.checks++;
  c->stats.bytes_checked += M.ri.n;
  return CG_OK;
}

cg_status cg_check_kernel_args(cg_ctx *c, const cg_karg *args, uint64_t nargs, cg_report *reps,
                               uint64_t *bad_index, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || (nargs && !args)) return set_error(CG_E_ARG, "NULL argument");
  for (uint64_t i = 0; i < nargs; i++) {
    const uint32_t a = args[i].access;
    if (a == 0 || (a & ~(CG_ARG_READ | CG_ARG_WRITE)) || args[i].reserved) {
      if (bad_index) *bad_index = i;
      return set_error(CG_E_ARG, "argument access must be CG_ARG_READ and/or CG_ARG_WRITE");
    }
  }
  if (nargs == 0) return CG_OK;
  if (nargs > 0xFFFFFFFFull) return set_error(CG_E_TOO_BIG, "at most 2^32-1 arguments per call");
  if (c->bb[0].ticket || c->bb[1].ticket)
    return set_error(CG_E_STATE, "batches still in flight (cg_batch_wait first)");
  NvtxRange range("cg kernel arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_TRY(flush_fills(c, st));
  // upload layout (16-byte aligned parts): jobs | range verdicts |
  // accumulators | order | scan segments | fill spans (pointer, bytes,
  // first group) | segment-claim counter | error flag; the last two zero
  const uint64_t o_info = round_up(nargs * sizeof(ScanJob), 16);
  const uint64_t o_acc = o_info + round_up(nargs * sizeof(RangeInfo), 16);
  const uint64_t o_order = o_acc + round_up(nargs * sizeof(Acc), 16);
  const uint64_t o_seg = o_order + round_up(nargs * 4, 16);
  const uint64_t o_fill = o_seg + round_up(nargs * 8, 16);
  const uint64_t o_claim = o_fill + round_up(3 * nargs * 8, 16);
  const uint64_t up = o_claim + 32;
  CG_TRY(c->k_in.ensure(up));
  CG_TRY(c->h_kin.ensure(up));
  // read-back (written by the finalize kernel into pinned memory): error
  // flag (16 bytes) | reports
  CG_TRY(c->h_kout.ensure(16 + nargs * sizeof(cg_report)));
  uint8_t *hp = c->h_kin.p;
  ScanJob *h_jobs = reinterpret_cast<ScanJob *>(hp);
  RangeInfo *h_info = reinterpret_cast<RangeInfo *>(hp + o_info);
  Acc *h_acc = reinterpret_cast<Acc *>(hp + o_acc);
  uint32_t *h_order = reinterpret_cast<uint32_t *>(hp + o_order);
  uint64_t *h_seg = reinterpret_cast<uint64_t *>(hp + o_seg);
  uint64_t *h_fptr = reinterpret_cast<uint64_t *>(hp + o_fill);
  uint64_t *h_fn = h_fptr + nargs, *h_fseg = h_fn + nargs;
  std::memset(hp + o_claim, 0, 32);
  const bool tma = c->cfg.scan_engine != 1 && !c->img_on_host;  // the scans read device memory only
  const uint64_t quantum = tma ? scan_tma_tile_bytes() : 2048;
  const uint64_t seg_bytes = std::max<uint64_t>(quantum, (65536 + quantum - 1) / quantum * quantum);
  const uint64_t seg_chunks = seg_bytes / 16;
  uint64_t segs = 0, fgroups = 0;
  // the range part of every argument on the host mirror (as single
  // checks): its read side as a copy source, its write side as a
  // destination (R23)
  for (uint64_t i = 0; i < nargs; i++) {
    const cg_karg &q = args[i];
    RangeInfo ri{};
    ri.kind = CG_DTOD;  // undefined bytes of a device source: the warning class
    ri.n = q.bytes;
    ScanJob j{};
    j.kind = CG_DTOD;
    j.n = q.bytes;
    uint64_t sh = 0, dsh = 0, fn = 0;
    if (q.access & CG_ARG_READ) {
      const bool ok = host_side(c, q.ptr, q.bytes, &ri.found_src, &ri.base_src, &ri.size_src, &sh,
                                &ri.flags, CG_F_UNALLOC_SRC, CG_F_OVERRUN_SRC);
      if (ok && q.bytes) {
        j.mode = kModeReadDev;
        j.dev_src = sh;
      }
    }
    if (q.access & CG_ARG_WRITE) {
      const bool ok = host_side(c, q.ptr, q.bytes, &ri.found_dst, &ri.base_dst, &ri.size_dst, &dsh,
                                &ri.flags, CG_F_UNALLOC_DST, CG_F_OVERRUN_DST);
      if (ok && c->cfg.carry) fn = q.bytes;
    }
    h_jobs[i] = j;
    h_info[i] = ri;
    h_acc[i] = Acc{0, 0, kNone, kNone};
    h_order[i] = (uint32_t)i;
    h_seg[i] = segs;
    if (j.mode & kModeReadDev) segs += (((q.bytes + 30) >> 4) + seg_chunks - 1) / seg_chunks;
    h_fptr[i] = dsh;
    h_fn[i] = fn;
    h_fseg[i] = fgroups;
    fgroups += fill_span_groups(fn);
  }
  uint8_t *dp = c->k_in.p;
  CG_CUDA(cudaMemcpyAsync(dp, hp, up, cudaMemcpyHostToDevice, st));
  BatchPlan plan{};
  plan.reqs = nullptr;
  plan.jobs = reinterpret_cast<ScanJob *>(dp);
  plan.info = reinterpret_cast<RangeInfo *>(dp + o_info);
  plan.acc = reinterpret_cast<Acc *>(dp + o_acc);
  plan.order = reinterpret_cast<const uint32_t *>(dp + o_order);
  plan.seg_first = reinterpret_cast<const uint64_t *>(dp + o_seg);
  plan.stage = nullptr;
  plan.nreq = nargs;
  plan.seg_chunks = (uint32_t)seg_chunks;
  plan.mode_mask = ~0u;
  const uint64_t *d_fill = reinterpret_cast<const uint64_t *>(dp + o_fill);
  unsigned long long *claim = reinterpret_cast<unsigned long long *>(dp + o_claim);
  unsigned int *d_err = reinterpret_cast<unsigned int *>(dp + o_claim + 16);
  if (segs) {  // one level: nothing is carried, every read sees the state before the launch
    if (tma)
      CG_CUDA(launch_scan_level_tma(c->img, plan, 0, nargs, segs, c->sm_count, claim, d_err, false,
                                    st));
    else
      CG_CUDA(launch_scan_level(c->img, plan, 0, nargs, segs, c->sm_count * 8, st));
    c->stats.kernels++;
  }
  CG_CUDA(launch_finalize_host(plan, d_err, c->h_kout.p, st));
  c->stats.kernels++;
  if (fgroups) {  // after the scan on the same stream
    CG_CUDA(launch_fill_spans(d_fill, d_fill + nargs, d_fill + 2 * nargs, nargs, fgroups, 0x00,
                              c->sm_count, st));
    c->stats.kernels++;
  }
  CG_CUDA(cudaStreamSynchronize(st));
  if (reinterpret_cast<const unsigned int *>(c->h_kout.p)[0])
    return set_error(CG_E_TIMEOUT, "a bounded wait in the scan kernel ran out");
  const cg_report *h_reps = reinterpret_cast<const cg_report *>(c->h_kout.p + 16);
  if (reps) std::memcpy(reps, h_reps, nargs * sizeof(cg_report));
  for (uint64_t i = 0; i < nargs; i++) count_stats(c, h_reps[i]);
  return CG_OK;
}

}  // extern "C"

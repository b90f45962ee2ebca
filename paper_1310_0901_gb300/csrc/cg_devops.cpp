// cg_devops.cpp -- the memset wrappers' check and kernel-argument checks.
//
// A memset is one range check on the host mirror plus a fill of the written
// bytes' V shadow with zeros (one launch).  The arguments of a kernel launch
// are checked together on the GPU: a lookup kernel over the device table
// gives every argument its verdicts, the batched scan kernels count the
// undefined bytes of in-range read arguments (one level: nothing is
// carried, every read sees the state before the launch), the finalize
// kernel builds the reports, and a fill kernel then defines the in-range
// write arguments.
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
  BatchBufs &K = c->bb[0];
  NvtxRange range("cg kernel arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_TRY(flush_fills(c, st));
  CG_TRY(ensure_device_table(c, st));
  CG_TRY(K.b_jobs.ensure(nargs));
  CG_TRY(K.b_info.ensure(nargs));
  CG_TRY(K.b_acc.ensure(nargs));
  CG_TRY(K.b_counts.ensure(nargs));
  const uint64_t nblocks = (nargs + kFinalizeItems - 1) / kFinalizeItems;
  CG_TRY(K.b_blocksums.ensure(nblocks + 1));
  // upload layout: arguments | order | scan segments | fill groups | the
  // scan's segment-claim counter (zero), then the fill spans (pointer,
  // bytes) the lookup writes on the device
  const uint64_t a_bytes = round_up(nargs * sizeof(cg_karg), 16);
  const uint64_t o_bytes = round_up(nargs * 4, 16);
  const uint64_t up = a_bytes + o_bytes + 16 * nargs + 16;
  CG_TRY(c->k_in.ensure(up + 16 * nargs));
  CG_TRY(c->h_kin.ensure(up));
  // read-back layout: reports | error flag
  const uint64_t r_bytes = round_up(nargs * sizeof(cg_report), 16);
  CG_TRY(c->k_out.ensure(r_bytes + 16));
  CG_TRY(c->h_kout.ensure(r_bytes + 16));
  uint8_t *hp = c->h_kin.p;
  std::memcpy(hp, args, nargs * sizeof(cg_karg));
  uint32_t *h_order = reinterpret_cast<uint32_t *>(hp + a_bytes);
  uint64_t *h_seg = reinterpret_cast<uint64_t *>(hp + a_bytes + o_bytes);
  uint64_t *h_fseg = h_seg + nargs;
  std::memset(hp + up - 16, 0, 16);
  const bool tma = c->cfg.scan_engine != 1;  // the scans read device memory only
  const uint64_t quantum = tma ? scan_tma_tile_bytes() : 2048;
  const uint64_t seg_bytes = std::max<uint64_t>(quantum, (65536 + quantum - 1) / quantum * quantum);
  const uint64_t seg_chunks = seg_bytes / 16;
  uint64_t segs = 0, fgroups = 0;
  for (uint64_t i = 0; i < nargs; i++) {
    h_order[i] = (uint32_t)i;
    h_seg[i] = segs;
    h_fseg[i] = fgroups;
    const uint64_t n = args[i].bytes;
    if ((args[i].access & CG_ARG_READ) && n) segs += (((n + 30) >> 4) + seg_chunks - 1) / seg_chunks;
    if (args[i].access & CG_ARG_WRITE) fgroups += fill_span_groups(n);
  }
  uint8_t *dp = c->k_in.p;
  const cg_karg *d_args = reinterpret_cast<const cg_karg *>(dp);
  uint32_t *d_order = reinterpret_cast<uint32_t *>(dp + a_bytes);
  uint64_t *d_seg = reinterpret_cast<uint64_t *>(dp + a_bytes + o_bytes);
  uint64_t *fill_seg = d_seg + nargs;
  unsigned long long *claim = reinterpret_cast<unsigned long long *>(dp + up - 16);
  uint64_t *fill_ptr = reinterpret_cast<uint64_t *>(dp + up), *fill_n = fill_ptr + nargs;
  cg_report *d_reps = reinterpret_cast<cg_report *>(c->k_out.p);
  unsigned int *d_err = reinterpret_cast<unsigned int *>(c->k_out.p + r_bytes);
  CG_CUDA(cudaMemcpyAsync(dp, hp, up, cudaMemcpyHostToDevice, st));
  BatchPlan plan{};
  plan.reqs = nullptr;  // only the lookup reads copies; the argument lookup has its own
  plan.order = d_order;
  plan.seg_first = d_seg;
  plan.stage = nullptr;
  plan.jobs = K.b_jobs.p;
  plan.info = K.b_info.p;
  plan.acc = K.b_acc.p;
  plan.nreq = nargs;
  plan.seg_chunks = (uint32_t)seg_chunks;
  plan.mode_mask = ~0u;
  DevTable dt{c->t_base.p, c->t_size.p, c->t_shadow.p, c->t_count};
  CG_CUDA(launch_karg_lookup(dt, plan, d_args, fill_ptr, fill_n, (int)c->cfg.carry, d_err, st));
  c->stats.kernels++;
  if (segs) {
    if (tma)
      CG_CUDA(launch_scan_level_tma(c->img, plan, 0, nargs, segs, c->sm_count, claim, d_err, false, st));
    else
      CG_CUDA(launch_scan_level(c->img, plan, 0, nargs, segs, c->sm_count * 8, st));
    c->stats.kernels++;
  }
  CG_CUDA(launch_finalize(plan, d_reps, K.b_counts.p, K.b_blocksums.p, kFinalizeItems, st));
  c->stats.kernels++;
  if (fgroups) {  // after the scans on the same stream: reads see the state before the launch
    CG_CUDA(launch_fill_spans(fill_ptr, fill_n, fill_seg, nargs, fgroups, 0x00, c->sm_count, st));
    c->stats.kernels++;
  }
  CG_CUDA(cudaMemcpyAsync(c->h_kout.p, c->k_out.p, r_bytes + 16, cudaMemcpyDeviceToHost, st));
  CG_CUDA(cudaStreamSynchronize(st));
  if (reinterpret_cast<const unsigned int *>(c->h_kout.p + r_bytes)[0])
    return set_error(CG_E_TIMEOUT, "a bounded wait in the scan kernel ran out");
  const cg_report *h_reps = reinterpret_cast<const cg_report *>(c->h_kout.p);
  if (reps) std::memcpy(reps, h_reps, nargs * sizeof(cg_report));
  for (uint64_t i = 0; i < nargs; i++) count_stats(c, h_reps[i]);
  return CG_OK;
}

}  // extern "C"

// cg_batch.cpp -- batched checks (cg_check_batch), the batch-split
// autotuner (cg_tune_batch) and the learned split chooser.
//
// A batch runs in phases: prepare (uploads, device lookup, level plan),
// split (cut every copy of every level into segments of the chosen size),
// levels (one persistent kernel per dependency level), finish (reports and
// records).  The tuner repeats split + levels per candidate segment size
// with the carry masked off, so trials leave the shadow untouched.
#include <cuda_runtime.h>

#include <cmath>

#include "cg_ctx.h"

using namespace cgi;

namespace {

struct StageCopy {
  int level;
  uint64_t src, dst, n, req;
};

struct BatchRun {
  const cg_copy *reqs = nullptr;
  uint64_t nreq = 0;
  BatchPlan plan{};
  std::vector<int> lvl;          // per request: the level of its first unit
  std::vector<PlanUnit> units;   // planning units (whole copies, pieces)
  uint64_t npos = 0;             // order positions (= units)
  int nlev = 0;
  std::vector<uint64_t> lev_start, lev_segs;
  std::vector<StageCopy> stages;
  const uint8_t *modes = nullptr;
  uint32_t *h_order = nullptr;
  uint64_t *h_segfirst = nullptr;
  uint64_t *h_piece = nullptr;
  bool tma = true;
  int grid = 1;
};

// `st` runs the batch; `look` runs its lookup (the same stream, or the side
// stream of an asynchronous submission so that the lookup does not queue
// behind the batch before it).
cg_status batch_prepare(cg_ctx *c, BatchBufs &K, const cg_copy *reqs, uint64_t nreq,
                        cudaStream_t st, cudaStream_t look, BatchRun &B) {
  B.reqs = reqs;
  B.nreq = nreq;
  CG_TRY(flush_fills(c, st));
  CG_TRY(ensure_device_table(c, look));  // only lookups read the device table
  CG_TRY(K.b_reqs.ensure(nreq));
  CG_TRY(K.b_stage.ensure(nreq));
  CG_TRY(K.b_jobs.ensure(nreq));
  CG_TRY(K.b_info.ensure(nreq));
  CG_TRY(K.b_acc.ensure(nreq));
  CG_TRY(K.b_reps.ensure(nreq));
  CG_TRY(K.b_counts.ensure(nreq));
  CG_TRY(K.b_modes.ensure(nreq));
  CG_TRY(K.b_err.ensure(1));
  const uint64_t upload_bytes = round_up(nreq * sizeof(cg_copy), 8) + nreq * 8 + 64;
  CG_TRY(K.h_stage_in.ensure(upload_bytes));
  CG_TRY(K.h_modes.ensure(nreq));
  cg_copy *h_reqs = reinterpret_cast<cg_copy *>(K.h_stage_in.p);
  uint64_t *h_stagep =
      reinterpret_cast<uint64_t *>(K.h_stage_in.p + round_up(nreq * sizeof(cg_copy), 8));
  std::memcpy(h_reqs, reqs, nreq * sizeof(cg_copy));

  // overlapping device->device copies are staged (R12); their source and
  // destination are looked up on the host mirror (they are rare)
  uint64_t stage_total = 0;
  std::memset(h_stagep, 0, nreq * sizeof(uint64_t));
  if (c->cfg.carry) {
    for (uint64_t i = 0; i < nreq; i++) {
      const cg_copy &q = reqs[i];
      if (q.kind != CG_DTOD || q.n == 0) continue;
      const uint64_t dist = q.src <= q.dst ? q.dst - q.src : q.src - q.dst;
      if (dist >= q.n) continue;
      uint64_t f, b, sz, sh, dsh;
      uint32_t fl = 0;
      const bool sok = host_side(c, q.src, q.n, &f, &b, &sz, &sh, &fl, 1, 2);
      const bool dok = host_side(c, q.dst, q.n, &f, &b, &sz, &dsh, &fl, 1, 2);
      if (!sok || !dok) continue;
      B.stages.push_back({0, sh, stage_total, q.n, i});
      h_stagep[i] = stage_total + 1;  // patched to an address below
      stage_total += round_up(q.n, 256);
    }
    if (stage_total) {
      CG_TRY(K.stage.ensure(stage_total));
      const uint64_t base = reinterpret_cast<uint64_t>(K.stage.p);
      for (uint64_t i = 0; i < nreq; i++)
        if (h_stagep[i]) h_stagep[i] = base + h_stagep[i] - 1;
      for (auto &sc : B.stages) sc.dst += base;
    }
  }
  CG_CUDA(cudaMemcpyAsync(K.b_reqs.p, h_reqs, nreq * sizeof(cg_copy), cudaMemcpyHostToDevice,
                          look));
  CG_CUDA(cudaMemcpyAsync(K.b_stage.p, h_stagep, nreq * 8, cudaMemcpyHostToDevice, look));
  BatchPlan &plan = B.plan;
  plan.reqs = K.b_reqs.p;
  plan.stage = K.b_stage.p;
  plan.jobs = K.b_jobs.p;
  plan.info = K.b_info.p;
  plan.acc = K.b_acc.p;
  plan.nreq = nreq;
  plan.mode_mask = ~0u;
  // device lookup first (a2): it decides which copies carry and read a
  // device source, which the level plan needs
  DevTable dt{c->t_base.p, c->t_size.p, c->t_shadow.p, c->t_count};
  const uint64_t t_lookup = now_ns();
  NvtxRange r_lookup("cg batch: lookup");
  CG_CUDA(launch_lookup(dt, plan, (int)c->cfg.strict_device_undef, (int)c->cfg.carry, look));
  CG_CUDA(launch_job_modes(plan, K.b_modes.p, look));
  c->stats.kernels += 2;
  CG_CUDA(cudaMemcpyAsync(K.h_modes.p, K.b_modes.p, nreq, cudaMemcpyDeviceToHost, look));
  CG_CUDA(cudaStreamSynchronize(look));  // the level kernels on st are issued after this
  B.modes = K.h_modes.p;
  const uint64_t t_plan = now_ns();
  c->stats.batch_lookup_ns += t_plan - t_lookup;
  // dependency levels, exact on validity, over planning units: whole
  // copies and, on the TMA engine, pieces of long host reads
  NvtxRange r_plan("cg batch: plan levels");
  B.tma = c->cfg.scan_engine != 1 && !c->img_on_host;
  const uint32_t pk = c->cfg.batch_piece_kib ? c->cfg.batch_piece_kib : 1024u;
  const uint64_t tile_rows = scan_tma_tile_bytes() / 512;
  const uint64_t piece_rows =
      (B.tma && pk != 0xFFFFFFFFu)
          ? std::max<uint64_t>(tile_rows, ((uint64_t)pk * 2) / tile_rows * tile_rows)
          : 0;
  B.units = plan_pieces(reqs, nreq, c->cfg.carry != 0, B.modes, c->img.n, piece_rows);
  B.npos = B.units.size();
  B.lvl.assign(nreq, 0);
  B.nlev = 0;
  bool any_piece = false;
  for (const PlanUnit &u : B.units) {
    B.nlev = std::max(B.nlev, u.level + 1);
    if (!u.rhi) B.lvl[u.req] = u.level;
    any_piece |= u.rhi != 0;
  }
  B.lev_start.assign(B.nlev + 1, 0);
  for (const PlanUnit &u : B.units) B.lev_start[u.level + 1]++;
  for (int l = 0; l < B.nlev; l++) B.lev_start[l + 1] += B.lev_start[l];
  // per position: request, first segment, piece (one pinned block)
  const uint64_t np = B.npos;
  CG_TRY(K.h_pos.ensure(round_up(np * 4, 8) + 2 * np * 8 + 64));
  B.h_order = reinterpret_cast<uint32_t *>(K.h_pos.p);
  B.h_segfirst = reinterpret_cast<uint64_t *>(K.h_pos.p + round_up(np * 4, 8));
  B.h_piece = B.h_segfirst + np;
  CG_TRY(K.b_order.ensure(np));
  CG_TRY(K.b_segfirst.ensure(np));
  if (any_piece) CG_TRY(K.b_piece.ensure(np));
  plan.order = K.b_order.p;
  plan.seg_first = K.b_segfirst.p;
  plan.piece = any_piece ? K.b_piece.p : nullptr;
  {
    // within a level, units in decreasing order of work (power-of-two
    // classes, stable): a level's segments are dealt to the warps in
    // turn, so the last turns hold the short segments of small units
    // and the level's tail is short (units of one level touch disjoint
    // shadow, so their order is free)
    std::vector<uint8_t> cls(np);
    uint64_t cnt[66] = {0};
    for (uint64_t k = 0; k < np; k++) {
      const PlanUnit &u = B.units[k];
      const cg_copy &q = reqs[u.req];
      uint64_t work = u.rhi ? 512ull * (u.rhi - u.rlo) : q.n;
      if (q.kind == CG_DTOD && !(B.modes[u.req] & (kModeCarry | kModeReadDev))) work = 0;
      if (B.tma && q.kind == CG_DTOH && !(B.modes[u.req] & kModeReadDev)) work = q.n >> 3;
      cls[k] = (uint8_t)(work ? 64 - __builtin_clzll(work) : 0);
      cnt[65 - cls[k]]++;
    }
    for (int k = 1; k < 66; k++) cnt[k] += cnt[k - 1];
    std::vector<uint32_t> by_work(np);
    for (uint64_t k = 0; k < np; k++) by_work[cnt[64 - cls[k]]++] = (uint32_t)k;
    std::vector<uint64_t> fill(B.lev_start.begin(), B.lev_start.end() - 1);
    for (uint32_t k : by_work) {
      const PlanUnit &u = B.units[k];
      const uint64_t pos = fill[u.level]++;
      B.h_order[pos] = u.req;
      B.h_piece[pos] = u.rhi ? ((uint64_t)u.rlo | ((uint64_t)u.rhi << 32)) : 0ull;
    }
  }
  for (auto &sc : B.stages) sc.level = B.lvl[sc.req];
  std::sort(B.stages.begin(), B.stages.end(),
            [](const StageCopy &a, const StageCopy &b) { return a.level < b.level; });
  c->stats.batch_plan_ns += now_ns() - t_plan;
  CG_CUDA(cudaMemcpyAsync(K.b_order.p, B.h_order, np * 4, cudaMemcpyHostToDevice, st));
  if (any_piece)
    CG_CUDA(cudaMemcpyAsync(K.b_piece.p, B.h_piece, np * 8, cudaMemcpyHostToDevice, st));
  CG_TRY(K.b_claim.ensure((uint64_t)B.nlev));
  int per_sm = (int)c->cfg.batch_ctas_per_sm;
  if (per_sm <= 0) per_sm = B.tma ? 1 : 8;
  B.grid = c->sm_count * per_sm;
  return CG_OK;
}

// Cut every copy into segments of seg_bytes (rounded to whole engine
// steps: one tile for the TMA engine, kU rows for register loads).
cg_status batch_split(cg_ctx *c, BatchBufs &K, BatchRun &B, uint64_t seg_bytes,
                      cudaStream_t st) {
  const uint64_t quantum = B.tma ? scan_tma_tile_bytes() : 2048;
  seg_bytes = std::max<uint64_t>(quantum, (seg_bytes + quantum - 1) / quantum * quantum);
  const uint64_t seg_chunks = seg_bytes / 16;
  B.plan.seg_chunks = (uint32_t)seg_chunks;
  B.lev_segs.assign(B.nlev, 0);
  for (int l = 0; l < B.nlev; l++) {
    uint64_t acc_segs = 0;
    for (uint64_t pos = B.lev_start[l]; pos < B.lev_start[l + 1]; pos++) {
      const uint32_t i = B.h_order[pos];
      const cg_copy &q = B.reqs[i];
      B.h_segfirst[pos] = acc_segs;
      if (B.h_piece[pos]) {  // rows [lo, hi) of the copy; segments are whole tiles
        const uint64_t rows = (B.h_piece[pos] >> 32) - (B.h_piece[pos] & 0xFFFFFFFFull);
        const uint64_t seg_rows = seg_chunks >> 5;
        acc_segs += (rows + seg_rows - 1) / seg_rows;
        continue;
      }
      const bool idle = q.kind == CG_DTOD && !(B.modes[i] & (kModeCarry | kModeReadDev));
      // the TMA engine walks a device->host copy with no valid source in
      // 128-byte super-chunks (its A bits alone)
      const bool aonly = B.tma && q.kind == CG_DTOH && !(B.modes[i] & kModeReadDev);
      const uint64_t chunks_ub = (q.n && !idle) ? (aonly ? (q.n + 254) >> 7 : (q.n + 30) >> 4) : 0;
      acc_segs += (chunks_ub + seg_chunks - 1) / seg_chunks;
    }
    B.lev_segs[l] = acc_segs;
  }
  CG_CUDA(cudaMemcpyAsync(K.b_segfirst.p, B.h_segfirst, B.npos * 8, cudaMemcpyHostToDevice, st));
  return CG_OK;
}

cg_status batch_levels(cg_ctx *c, BatchBufs &K, BatchRun &B, uint32_t mode_mask,
                       cudaStream_t st) {
  NvtxRange range("cg batch: enqueue level kernels");
  B.plan.mode_mask = mode_mask;
  const bool dry = !(mode_mask & kModeCarry);
  CG_CUDA(cudaMemsetAsync(K.b_err.p, 0, sizeof(unsigned int), st));
  if (B.tma)  // one segment-claim counter per level
    CG_CUDA(cudaMemsetAsync(K.b_claim.p, 0, (size_t)B.nlev * sizeof(unsigned long long), st));
  size_t sci = 0;
  for (int l = 0; l < B.nlev; l++) {
    for (; !dry && sci < B.stages.size() && B.stages[sci].level == l; sci++)
      CG_CUDA(cudaMemcpyAsync(reinterpret_cast<void *>(B.stages[sci].dst),
                              reinterpret_cast<const void *>(B.stages[sci].src), B.stages[sci].n,
                              cudaMemcpyDeviceToDevice, st));
    if (B.tma)
      CG_CUDA(launch_scan_level_tma(c->img, B.plan, B.lev_start[l], B.lev_start[l + 1],
                                    B.lev_segs[l], B.grid, K.b_claim.p + l, K.b_err.p, l > 0, st));
    else
      CG_CUDA(launch_scan_level(c->img, B.plan, B.lev_start[l], B.lev_start[l + 1], B.lev_segs[l],
                                B.grid, st));
    c->stats.kernels++;
  }
  return CG_OK;
}

const uint32_t kCandidatesKib[] = {4, 8, 16, 32, 64, 128, 256, 512, 1024};
constexpr int kNumCandidates = sizeof(kCandidatesKib) / sizeof(kCandidatesKib[0]);
const uint32_t kOnlineKib[] = {16, 32, 64, 128, 256};
constexpr uint32_t kNumOnline = sizeof(kOnlineKib) / sizeof(kOnlineKib[0]);

void features(const cg_copy *reqs, uint64_t nreq, float *f) {
  double s1 = 0, s2 = 0, total = 0;
  double bins[6] = {0, 0, 0, 0, 0, 0};
  double kinds[3] = {0, 0, 0};
  for (uint64_t i = 0; i < nreq; i++) {
    const double n = (double)reqs[i].n;
    const double l = std::log2(1.0 + n);
    s1 += l;
    s2 += l * l;
    total += n;
    const int b = n <= 4096.0 ? 0 : n <= 65536.0 ? 1 : n <= 1048576.0 ? 2
                  : n <= 4194304.0 ? 3 : n <= 16777216.0 ? 4 : 5;
    bins[b] += n;
    if (reqs[i].kind >= 1 && reqs[i].kind <= 3) kinds[reqs[i].kind - 1] += 1.0;
  }
  const double m = nreq ? s1 / nreq : 0.0;
  f[0] = (float)std::log2(1.0 + (double)nreq);
  f[1] = (float)m;
  f[2] = (float)std::sqrt(std::max(0.0, nreq ? s2 / nreq - m * m : 0.0));
  for (int k = 0; k < 6; k++) f[3 + k] = (float)(total > 0 ? bins[k] / total : 0.0);
  for (int k = 0; k < 3; k++) f[9 + k] = (float)(nreq ? kinds[k] / nreq : 0.0);
  f[12] = (float)std::log2(1.0 + total);
}

// The learned cost model: predicted log2(batch ms) for features f and a
// segment size; see cg_set_cost_model for the weight layout.
float predict(const cg_ctx *c, const float *f, uint32_t seg_kib) {
  const int D = CG_NFEAT + 1, H = (int)c->cost_hidden;
  const float *mu = c->cost_model.data();
  const float *sd = mu + D;
  const float *w1 = sd + D;
  const float *b1 = w1 + D * H;
  const float *w2 = b1 + H;
  const float *b2 = w2 + H;
  float x[CG_NFEAT + 1];
  for (int k = 0; k < CG_NFEAT; k++) x[k] = f[k];
  x[CG_NFEAT] = std::log2((float)seg_kib);
  for (int k = 0; k < D; k++) x[k] = (x[k] - mu[k]) / sd[k];
  float y = b2[0];
  for (int j = 0; j < H; j++) {
    float h = b1[j];
    for (int k = 0; k < D; k++) h += x[k] * w1[k * H + j];
    y += (h > 0.f ? h : 0.f) * w2[j];
  }
  return y;
}

// mean scaled distance between two feature vectors
float feature_distance(const float *a, const float *b) {
  float d = 0.f;
  for (int k = 0; k < CG_NFEAT; k++) {
    const float scale = (k == 0 || k == 12) ? 0.25f : (k == 1 || k == 2) ? 0.5f : 4.0f;
    d += std::fabs(a[k] - b[k]) * scale;
  }
  return d / CG_NFEAT;
}
constexpr float kClose = 0.5f;

// Segment size for a batch when the configuration leaves it open: a tuned
// entry close to this batch's features; else, with online tuning on, the
// next untried candidate for this shape (*source = 4: a trial, recorded when
// the batch finishes); else the learned model's argmin over the candidates;
// else 64 KiB.
uint32_t choose_kib(const cg_ctx *c, const cg_copy *reqs, uint64_t nreq, uint32_t *source) {
  float f[CG_NFEAT];
  features(reqs, nreq, f);
  float best_d = kClose;
  int best = -1;
  for (size_t e = 0; e < c->tuned_feat.size(); e++) {
    const float d = feature_distance(c->tuned_feat[e].data(), f);
    if (d < best_d) {
      best_d = d;
      best = (int)e;
    }
  }
  if (best >= 0) {
    if (source) *source = 1;
    return c->tuned_kib[best];
  }
  if (c->cfg.batch_autotune) {
    int slot = -1;
    best_d = kClose;
    for (size_t e = 0; e < c->online.size(); e++) {
      const float d = feature_distance(c->online[e].feat.data(), f);
      if (d < best_d) {
        best_d = d;
        slot = (int)e;
      }
    }
    const uint32_t next = slot >= 0 ? c->online[slot].next : 0;  // a new shape: the first
    if (source) *source = 4;
    return kOnlineKib[next < kNumOnline ? next : 0];
  }
  if (!c->cost_model.empty()) {
    uint32_t arg = 64;
    float lo = 0.f;
    for (int k = 0; k < kNumCandidates; k++) {
      const float y = predict(c, f, kCandidatesKib[k]);
      if (k == 0 || y < lo) {
        lo = y;
        arg = kCandidatesKib[k];
      }
    }
    if (source) *source = 2;
    return arg;
  }
  if (source) *source = 0;
  return 64;
}

// Record an online trial of segment size kib for the batch shape `f`; once
// every candidate has run, the fastest becomes a tuned entry.  The shape's
// entry is found again by its features (another batch may have finished
// in between), and a candidate timed twice does not skip one.
void online_record(cg_ctx *c, const float *f, uint32_t kib, float ms) {
  int slot = -1;
  float best_d = kClose;
  for (size_t e = 0; e < c->online.size(); e++) {
    const float d = feature_distance(c->online[e].feat.data(), f);
    if (d < best_d) {
      best_d = d;
      slot = (int)e;
    }
  }
  if (slot < 0) {
    for (size_t e = 0; e < c->tuned_feat.size(); e++)  // already settled
      if (feature_distance(c->tuned_feat[e].data(), f) < kClose) return;
    cg_ctx::OnlineTune t;
    t.feat.assign(f, f + CG_NFEAT);
    c->online.push_back(t);
    slot = (int)c->online.size() - 1;
  }
  cg_ctx::OnlineTune &t = c->online[slot];
  uint32_t idx = 0;
  while (idx < kNumOnline && kOnlineKib[idx] != kib) idx++;
  if (t.best_kib == 0 || ms < t.best_ms) {
    t.best_ms = ms;
    t.best_kib = kib;
  }
  t.next = std::max(t.next, idx + 1);
  if (t.next >= kNumOnline) {
    c->tuned_feat.push_back(t.feat);
    c->tuned_kib.push_back(t.best_kib);
    c->online.erase(c->online.begin() + slot);
  }
}

// Enqueue a batch into a free slot: host validation, the lookup (on `look`)
// and the level plan on the host, then the level kernels, reports, records
// and the copies of the results on `st`; K.done is recorded after them.
cg_status batch_submit(cg_ctx *c, const cg_copy *reqs, uint64_t nreq, uint64_t rec_cap,
                       uint64_t *bad_index, cudaStream_t st, cudaStream_t look, int *slot_out) {
  for (uint64_t i = 0; i < nreq; i++) {
    const cg_status s = validate(c, reqs[i]);
    if (s != CG_OK) {
      if (bad_index) *bad_index = i;
      return s;
    }
  }
  if (nreq > 0xFFFFFFFFull) return set_error(CG_E_TOO_BIG, "at most 2^32-1 requests per batch");
  int slot = -1;
  for (int k = 0; k < 2 && slot < 0; k++)
    if (!c->bb[k].ticket) slot = k;
  if (slot < 0) return set_error(CG_E_FULL, "two batches in flight: cg_batch_wait first");
  BatchBufs &K = c->bb[slot];
  NvtxRange range("cg batch: submit");
  K.t_begin = now_ns();
  BatchRun B;
  CG_TRY(batch_prepare(c, K, reqs, nreq, st, look, B));
  K.source = 3;
  K.kib = c->cfg.batch_segment_kib ? c->cfg.batch_segment_kib
                                   : choose_kib(c, reqs, nreq, &K.source);
  if (K.source == 4) {
    K.feat.resize(CG_NFEAT);
    features(reqs, nreq, K.feat.data());
  }
  CG_TRY(batch_split(c, K, B, (uint64_t)K.kib * 1024, st));
  if (!K.done) CG_CUDA(cudaEventCreateWithFlags(&K.done, cudaEventDisableTiming));
  if (!K.t0) CG_CUDA(cudaEventCreate(&K.t0));
  if (!K.t1) CG_CUDA(cudaEventCreate(&K.t1));
  K.nreq = nreq;
  K.nlev = B.nlev;
  K.nblocks = (nreq + kFinalizeItems - 1) / kFinalizeItems;
  CG_TRY(K.b_blocksums.ensure(K.nblocks + 1));
  K.dev_rec_cap = std::min<uint64_t>(rec_cap, nreq * CG_NFLAGS);
  CG_TRY(K.b_recs.ensure(std::max<uint64_t>(K.dev_rec_cap, 1)));
  CG_TRY(K.h_total.ensure(2));
  CG_TRY(K.h_reps.ensure(nreq));
  // the batch's device work: on `st` directly, or captured on the context's
  // capture stream into a CUDA graph that is then launched on `st`
  const bool graph = !c->cfg.batch_direct_launch;
  if (graph && !c->cap) CG_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  cudaStream_t es = graph ? c->cap : st;
  struct Capture {  // ends a capture left open by an error
    cudaStream_t s = nullptr;
    ~Capture() {
      if (!s) return;
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
  } open_capture;
  if (graph) {
    CG_CUDA(cudaStreamBeginCapture(es, cudaStreamCaptureModeRelaxed));
    open_capture.s = es;
  } else {
    CG_CUDA(cudaEventRecord(K.t0, st));
  }
  CG_TRY(batch_levels(c, K, B, ~0u, es));
  if (!graph) CG_CUDA(cudaEventRecord(K.t1, st));
  const int strict = (int)c->cfg.strict_device_undef;
  CG_CUDA(launch_finalize(B.plan, K.b_reps.p, K.b_counts.p, K.b_blocksums.p, kFinalizeItems, es));
  CG_CUDA(launch_scan_block_sums(K.b_blocksums.p, K.nblocks, nullptr, es));
  CG_CUDA(launch_emit_records(B.plan, K.b_reps.p, K.b_counts.p, K.b_blocksums.p, kFinalizeItems,
                              strict, K.b_recs.p, K.dev_rec_cap, es));
  c->stats.kernels += K.dev_rec_cap ? 3 : 2;
  CG_CUDA(cudaMemcpyAsync(K.h_total.p, K.b_blocksums.p + K.nblocks, 8, cudaMemcpyDeviceToHost,
                          es));
  CG_CUDA(cudaMemcpyAsync(K.h_total.p + 1, K.b_err.p, sizeof(unsigned int),
                          cudaMemcpyDeviceToHost, es));
  CG_CUDA(cudaMemcpyAsync(K.h_reps.p, K.b_reps.p, nreq * sizeof(cg_report),
                          cudaMemcpyDeviceToHost, es));
  if (graph) {
    cudaGraph_t g = nullptr;
    open_capture.s = nullptr;
    CG_CUDA(cudaStreamEndCapture(es, &g));
    cudaError_t e = cudaErrorUnknown;
    if (K.exec) {  // same shape as this slot's last batch: update in place
      cudaGraphExecUpdateResultInfo info{};
      e = cudaGraphExecUpdate(K.exec, g, &info);
      if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(K.exec);
        K.exec = nullptr;
      }
    }
    if (!K.exec) e = cudaGraphInstantiate(&K.exec, g, 0);
    cudaGraphDestroy(g);
    CG_CUDA(e);
    CG_CUDA(cudaEventRecord(K.t0, st));
    CG_CUDA(cudaGraphLaunch(K.exec, st));
    CG_CUDA(cudaEventRecord(K.t1, st));
  }
  CG_CUDA(cudaEventRecord(K.done, st));
  K.ticket = c->next_ticket++;
  *slot_out = slot;
  return CG_OK;
}

// Wait for the batch in `slot` and hand its results out; frees the slot.
cg_status batch_finish(cg_ctx *c, int slot, cg_report *reps, cg_err_record *recs,
                       uint64_t rec_cap, uint64_t *n_rec) {
  BatchBufs &K = c->bb[slot];
  NvtxRange range("cg batch: wait");
  struct Free {
    BatchBufs &k;
    ~Free() { k.ticket = 0; }
  } release_slot{K};
  CG_CUDA(cudaEventSynchronize(K.done));
  if (K.source == 4) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, K.t0, K.t1);
    online_record(c, K.feat.data(), K.kib, ms);
  }
  if (reinterpret_cast<const unsigned int *>(K.h_total.p + 1)[0])
    return set_error(CG_E_TIMEOUT, "a bounded wait in the batched scan kernel ran out");
  const uint64_t total = K.h_total.p[0];
  const uint64_t take = std::min(std::min(total, K.dev_rec_cap), rec_cap);
  if (take && recs) {
    // on the context's own non-blocking stream: a synchronous copy on the
    // legacy stream would also wait for the next batch's kernels
    if (!c->side) CG_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CG_TRY(K.h_recs.ensure(take));
    CG_CUDA(cudaMemcpyAsync(K.h_recs.p, K.b_recs.p, take * sizeof(cg_err_record),
                            cudaMemcpyDeviceToHost, c->side));
    CG_CUDA(cudaStreamSynchronize(c->side));
    std::memcpy(recs, K.h_recs.p, take * sizeof(cg_err_record));
  }
  if (reps) std::memcpy(reps, K.h_reps.p, K.nreq * sizeof(cg_report));
  {
    std::lock_guard<std::mutex> g(c->stats_mu);
    for (uint64_t i = 0; i < K.nreq; i++) count_stats(c, K.h_reps.p[i]);
    c->stats.batch_ns += now_ns() - K.t_begin;
    c->stats.batches++;
    c->stats.levels += (uint64_t)K.nlev;
  }
  if (n_rec) *n_rec = total;
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_get_tuned(const cg_ctx *c, float *feat, uint32_t *kib, uint32_t cap,
                       uint32_t *count) {
  if (!c || !count || (cap && (!feat || !kib))) return set_error(CG_E_ARG, "NULL argument");
  const uint32_t n = (uint32_t)c->tuned_kib.size();
  for (uint32_t e = 0; e < n && e < cap; e++) {
    std::memcpy(feat + (size_t)e * CG_NFEAT, c->tuned_feat[e].data(), CG_NFEAT * sizeof(float));
    kib[e] = c->tuned_kib[e];
  }
  *count = n;
  return CG_OK;
}

cg_status cg_add_tuned(cg_ctx *c, const float *feat, const uint32_t *kib, uint32_t count) {
  if (!c || (count && (!feat || !kib))) return set_error(CG_E_ARG, "NULL argument");
  for (uint32_t e = 0; e < count; e++)
    if (kib[e] == 0) return set_error(CG_E_ARG, "segment size 0");
  for (uint32_t e = 0; e < count; e++) {
    c->tuned_feat.emplace_back(feat + (size_t)e * CG_NFEAT, feat + (size_t)(e + 1) * CG_NFEAT);
    c->tuned_kib.push_back(kib[e]);
  }
  return CG_OK;
}

cg_status cg_check_batch(cg_ctx *c, const cg_copy *reqs, uint64_t nreq, cg_report *reps,
                         cg_err_record *recs, uint64_t rec_cap, uint64_t *n_rec,
                         uint64_t *bad_index, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || (nreq && !reqs) || !n_rec || (rec_cap && !recs))
    return set_error(CG_E_ARG, "NULL argument");
  if (nreq == 0) {
    *n_rec = 0;
    return CG_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int slot = -1;
  CG_TRY(batch_submit(c, reqs, nreq, rec_cap, bad_index, st, st, &slot));
  return batch_finish(c, slot, reps, recs, rec_cap, n_rec);
}

cg_status cg_check_batch_async(cg_ctx *c, const cg_copy *reqs, uint64_t nreq, uint64_t rec_cap,
                               uint64_t *ticket, uint64_t *bad_index, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !nreq || !reqs || !ticket) return set_error(CG_E_ARG, "NULL argument or empty batch");
  if (!c->side) CG_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  int slot = -1;
  CG_TRY(batch_submit(c, reqs, nreq, rec_cap, bad_index, static_cast<cudaStream_t>(stream),
                      c->side, &slot));
  *ticket = c->bb[slot].ticket;
  return CG_OK;
}

cg_status cg_batch_wait(cg_ctx *c, uint64_t ticket, cg_report *reps, cg_err_record *recs,
                        uint64_t rec_cap, uint64_t *n_rec) {
  if (!c || (rec_cap && !recs)) return set_error(CG_E_ARG, "NULL argument");
  for (int k = 0; k < 2; k++)
    if (ticket && c->bb[k].ticket == ticket) return batch_finish(c, k, reps, recs, rec_cap, n_rec);
  return set_error(CG_E_ARG, "no batch in flight with this ticket");
}

cg_status cg_batch_features(const cg_copy *reqs, uint64_t nreq, float *feat) {
  if (!feat || (nreq && !reqs)) return set_error(CG_E_ARG, "NULL argument");
  features(reqs, nreq, feat);
  return CG_OK;
}

cg_status cg_tune_batch(cg_ctx *c, const cg_copy *reqs, uint64_t nreq, const uint32_t *seg_kib,
                        uint32_t ncand, uint32_t repeats, uint32_t flags, float *ms,
                        uint32_t *best_kib, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !reqs || !nreq) return set_error(CG_E_ARG, "NULL argument or empty batch");
  for (uint64_t i = 0; i < nreq; i++) CG_TRY(validate(c, reqs[i]));
  const uint32_t *cand = seg_kib ? seg_kib : kCandidatesKib;
  const uint32_t nc = seg_kib ? ncand : (uint32_t)kNumCandidates;
  if (nc == 0) return set_error(CG_E_ARG, "no candidates");
  if (repeats == 0) repeats = 1;
  if (c->bb[0].ticket || c->bb[1].ticket)
    return set_error(CG_E_STATE, "batches still in flight (cg_batch_wait first)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchBufs &K = c->bb[0];
  BatchRun B;
  CG_TRY(batch_prepare(c, K, reqs, nreq, st, st, B));
  cudaEvent_t e0, e1;
  CG_CUDA(cudaEventCreate(&e0));
  CG_CUDA(cudaEventCreate(&e1));
  float best_ms = 0.f;
  uint32_t best = cand[0];
  cg_status status = CG_OK;
  for (uint32_t k = 0; k < nc && status == CG_OK; k++) {
    status = batch_split(c, K, B, (uint64_t)cand[k] * 1024, st);
    float lo = 0.f;
    for (uint32_t r = 0; r < repeats && status == CG_OK; r++) {
      cudaEventRecord(e0, st);
      status = batch_levels(c, K, B, ~kModeCarry, st);  // dry: the shadow is not written
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) status = set_error(CG_E_CUDA, "tuning run");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r == 0 || t < lo) lo = t;
    }
    if (ms) ms[k] = lo;
    if (k == 0 || lo < best_ms) {
      best_ms = lo;
      best = cand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CG_TRY(status);
  if (flags & CG_TUNE_REMEMBER) {
    std::vector<float> f(CG_NFEAT);
    features(reqs, nreq, f.data());
    c->tuned_feat.push_back(f);
    c->tuned_kib.push_back(best);
  }
  if (best_kib) *best_kib = best;
  return CG_OK;
}

cg_status cg_set_cost_model(cg_ctx *c, const float *weights, uint32_t hidden) {
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (!weights || hidden == 0) {
    c->cost_model.clear();
    c->cost_hidden = 0;
    return CG_OK;
  }
  if (hidden > 1024) return set_error(CG_E_TOO_BIG, "hidden layer above 1024 units");
  const size_t D = CG_NFEAT + 1;
  const size_t n = 2 * D + D * hidden + hidden + hidden + 1;
  for (size_t k = D; k < 2 * D; k++)
    if (!(weights[k] > 0.f)) return set_error(CG_E_ARG, "input scales must be positive");
  c->cost_model.assign(weights, weights + n);
  c->cost_hidden = hidden;
  return CG_OK;
}

cg_status cg_choose_segment(const cg_ctx *c, const cg_copy *reqs, uint64_t nreq,
                            uint32_t *seg_kib, uint32_t *source) {
  if (!c || !seg_kib || (nreq && !reqs)) return set_error(CG_E_ARG, "NULL argument");
  if (c->cfg.batch_segment_kib) {
    *seg_kib = c->cfg.batch_segment_kib;
    if (source) *source = 3;
    return CG_OK;
  }
  *seg_kib = choose_kib(c, reqs, nreq, source);
  return CG_OK;
}

}  // extern "C"

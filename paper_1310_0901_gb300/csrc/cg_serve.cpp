// cg_serve.cpp -- the serving loop: client rings, one scheduler thread,
// continuous batching of checks into rounds that overlap on the GPU.
//
// Order.  The scheduler admits requests one at a time and numbers them
// (result.seq); allocation events change the table at their place in that
// order and every check is looked up on the host mirror when it is
// admitted, so each request sees exactly the table state of its place in
// the order.  Checks admitted while earlier rounds are still on the GPU
// form the next round; a round is planned into dependency levels like a
// batch and runs on its own stream.  Two rounds run concurrently unless
// one reads or writes shadow that the other writes; then the later waits
// for the earlier (an event).  A freed allocation's shadow slot returns to
// the pool only after every round that may still use it has finished.
#include <cuda_runtime.h>

#include <atomic>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "cg_ctx.h"
#include "cg_race_index.h"

namespace cgi {

struct RaceEntry;

struct RingSlot {
  cg_request req;
  uint64_t submit_ns;
  std::atomic<uint32_t> state;  // 0 free, 1 submitted, 2 done, 3 collected
  cg_result res;
  RaceEntry *race = nullptr;  // its race-window entry (scheduler only)
};

struct ClientRing {
  std::unique_ptr<RingSlot[]> slots;
  uint64_t mask = 0;
  alignas(64) std::atomic<uint64_t> head{0};       // next index to submit (client)
  alignas(64) std::atomic<uint64_t> taken{0};      // next index to admit (scheduler)
  alignas(64) std::atomic<uint64_t> collected{0};  // all below collected (client)
  // 0: not inside cg_submit; 1: inside, timestamp not taken yet; else the
  // submit timestamp being published (lower bound for the race window)
  alignas(64) std::atomic<uint64_t> submitting{0};
};

// An admitted copy that moved data (valid device ranges), kept while a
// later copy of another client may still race with it.
struct RaceEntry {
  uint64_t seq;
  uint32_t client;
  uint32_t kind;
  uint64_t dst, src, n;
  uint64_t done_ns;  // 0 while in flight
};

static bool meets(uint64_t a, uint64_t na, uint64_t b, uint64_t nb) {
  return a < b + nb && b < a + na;
}

// q writes what r reads or writes, or reads what r writes (host offsets and
// device addresses are separate spaces)
static bool races_with(const RaceEntry &q, uint32_t kind, uint64_t dst, uint64_t src,
                       uint64_t n) {
  auto dsp = [](uint32_t k) { return k == CG_DTOH ? 0 : 1; };
  auto ssp = [](uint32_t k) { return k == CG_HTOD ? 0 : 1; };
  return (dsp(q.kind) == ssp(kind) && meets(q.dst, q.n, src, n)) ||
         (dsp(q.kind) == dsp(kind) && meets(q.dst, q.n, dst, n)) ||
         (ssp(q.kind) == dsp(kind) && meets(q.src, q.n, dst, n));
}

static int dst_space(uint32_t kind) { return kind == CG_DTOH ? 0 : 1; }
static int src_space(uint32_t kind) { return kind == CG_HTOD ? 0 : 1; }

struct Iv {
  uint64_t a, b;
};

// Shadow ranges a round reads and writes (host image offsets, device
// shadow addresses), for the cross-round hazard test.
struct Footprint {
  std::vector<Iv> hr, hw, dr, dw;
  void clear() {
    hr.clear();
    hw.clear();
    dr.clear();
    dw.clear();
  }
  void sort_all() {
    auto by_a = [](const Iv &x, const Iv &y) { return x.a < y.a; };
    std::sort(hr.begin(), hr.end(), by_a);
    std::sort(hw.begin(), hw.end(), by_a);
    std::sort(dr.begin(), dr.end(), by_a);
    std::sort(dw.begin(), dw.end(), by_a);
  }
};

// do two sorted interval lists intersect?
static bool meet(const std::vector<Iv> &x, const std::vector<Iv> &y) {
  size_t i = 0, j = 0;
  uint64_t xmax = 0, ymax = 0;  // furthest end seen so far on each side
  bool xs = false, ys = false;
  while (i < x.size() || j < y.size()) {
    const bool take_x = j >= y.size() || (i < x.size() && x[i].a <= y[j].a);
    if (take_x) {
      if (ys && x[i].a < ymax) return true;
      xmax = xs ? std::max(xmax, x[i].b) : x[i].b;
      xs = true;
      i++;
    } else {
      if (xs && y[j].a < xmax) return true;
      ymax = ys ? std::max(ymax, y[j].b) : y[j].b;
      ys = true;
      j++;
    }
  }
  return false;
}

static bool conflicts(const Footprint &n, const Footprint &o) {
  return meet(n.hr, o.hw) || meet(n.hw, o.hw) || meet(n.hw, o.hr) || meet(n.dr, o.dw) ||
         meet(n.dw, o.dw) || meet(n.dw, o.dr);
}

struct StageCopy {
  int level;
  uint64_t src, off, n;
};

struct RoundSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  // packed jobs | info | acc | order | seg_first | stage ptrs | error flag:
  // one upload per round (the flag zeroed)
  DevBuf<uint8_t> d_up;
  DevBuf<uint8_t> stage;
  PinBuf<uint8_t> h_up;
  PinBuf<uint8_t> h_down;  // error flag (16 bytes) | reports, written by the GPU
  bool busy = false;
  uint64_t id = 0;
  uint64_t bytes = 0;
  std::vector<RingSlot *> members;
  Footprint fp;
};

struct Deferred {
  uint64_t ptr, size, tag;  // release once every round up to `tag` is done
};

struct ServeEngine {
  cg_ctx *c = nullptr;
  std::mutex &stats_mu;
  cg_serve_config cfg{};
  std::vector<ClientRing> rings;
  std::vector<RoundSlot> rs;
  std::thread th;
  std::atomic<bool> stop{false};
  cg_serve_stats st{};
  uint64_t next_seq = 0;
  uint64_t next_round = 1;
  uint64_t rr = 0;
  uint64_t inflight_bytes = 0;
  std::vector<Deferred> deferred;
  // seq order; entries already dropped from the index keep their place
  // (n = 0) until everything before them is gone too
  // (entries are referred to by address: a deque keeps the addresses of
  // the others through push_back and pop_front)
  std::deque<RaceEntry> window;
  RaceIndex window_index;  // items: entry addresses
  // the window's finished entries in the order they finished, so done_ns
  // never decreases along it
  std::deque<RaceEntry *> done_order;
  cg_status fatal = CG_OK;

  ServeEngine(cg_ctx *ctx, size_t nclients) : c(ctx), stats_mu(ctx->stats_mu), rings(nclients) {}

  uint64_t done_upto() const {
    uint64_t lo = next_round;  // smallest busy round id
    for (const auto &r : rs)
      if (r.busy) lo = std::min(lo, r.id);
    return lo - 1;
  }

  void finish(RingSlot *sl, int32_t status) {
    sl->res.status = status;
    sl->res.submit_ns = sl->submit_ns;
    sl->res.done_ns = now_ns();
    sl->state.store(2, std::memory_order_release);
  }

  bool complete_rounds() {
    bool progress = false;
    for (auto &r : rs) {
      if (!r.busy) continue;
      const cudaError_t e = cudaEventQuery(r.done);
      if (e == cudaErrorNotReady) continue;
      const bool ok = e == cudaSuccess && *reinterpret_cast<const unsigned int *>(r.h_down.p) == 0;
      const cg_report *h_reps = reinterpret_cast<const cg_report *>(r.h_down.p + 16);
      if (e != cudaSuccess) cudaGetLastError();
      {
        std::lock_guard<std::mutex> g(stats_mu);
        for (size_t i = 0; i < r.members.size(); i++) {
          RingSlot *sl = r.members[i];
          const int64_t race = sl->res.report.race_seq;  // set at admission
          sl->res.report = h_reps[i];
          if (race >= 0) {
            sl->res.report.flags |= CG_F_CONCURRENT;
            sl->res.report.race_seq = race;
          }
          if (ok) count_stats(c, sl->res.report);
        }
      }
      for (RingSlot *sl : r.members) {
        finish(sl, ok ? CG_OK : (e == cudaSuccess ? CG_E_TIMEOUT : CG_E_CUDA));
        mark_done(sl);
      }
      inflight_bytes -= r.bytes;
      r.busy = false;
      r.members.clear();
      progress = true;
    }
    if (progress) release_deferred(done_upto());
    return progress;
  }

  // the window entry of a finished copy (if it moved data)
  void mark_done(RingSlot *sl) {
    RaceEntry *e = sl->race;
    sl->race = nullptr;
    if (!e || e->done_ns) return;
    e->done_ns = sl->res.done_ns;
    done_order.push_back(e);
  }

  // Drop finished copies that no request submitted from now on can race
  // with (those that finished no later than every future submit time).
  // The candidates come off the front of done_order, so a round's pruning
  // costs what it drops, however long the window has grown behind a
  // backlog.
  void prune_window() {
    if (done_order.empty()) return;
    uint64_t bound = now_ns();  // read before the clients' words
    for (auto &g : rings) {
      const uint64_t v = g.submitting.load(std::memory_order_seq_cst);
      if (v == 1) return;  // a timestamp is being taken: keep everything
      if (v) bound = std::min(bound, v);
      const uint64_t t = g.taken.load(std::memory_order_relaxed);
      if (t != g.head.load(std::memory_order_acquire))
        bound = std::min(bound, g.slots[t & g.mask].submit_ns);
    }
    while (!done_order.empty() && done_order.front()->done_ns <= bound) {
      RaceEntry *e = done_order.front();
      done_order.pop_front();
      const uint64_t item = reinterpret_cast<uint64_t>(e);
      window_index.remove(dst_space(e->kind), e->dst, e->n, item);
      window_index.remove(src_space(e->kind), e->src, e->n, item);
      e->n = 0;
    }
    while (!window.empty() && window.front().n == 0) window.pop_front();
  }

  void release_deferred(uint64_t upto) {
    size_t k = 0;
    for (size_t i = 0; i < deferred.size(); i++) {
      if (deferred[i].tag <= upto) {
        c->arena.release(deferred[i].ptr, deferred[i].size);
        c->fill_ptr.push_back(deferred[i].ptr);
        c->fill_size.push_back(deferred[i].size);
      } else {
        deferred[k++] = deferred[i];
      }
    }
    deferred.resize(k);
  }

  bool any_busy() const {
    for (const auto &r : rs)
      if (r.busy) return true;
    return false;
  }

  bool rings_empty() const {
    for (const auto &g : rings)
      if (g.taken.load(std::memory_order_relaxed) != g.head.load(std::memory_order_acquire))
        return false;
    return true;
  }

  // An allocation event or client request that never reaches the GPU.
  void apply_host_op(RingSlot *sl, uint64_t round_tag) {
    const cg_request &q = sl->req;
    sl->res.verdict = 0;
    if (q.op == CG_OP_ALLOC) {
      cg_status s = CG_OK;
      if (q.n == 0)
        s = CG_E_ZERO_SIZE;
      else if (q.dst + q.n < q.dst)
        s = CG_E_WRAP;
      else if (c->table.overlaps(q.dst, q.n))
        s = CG_E_OVERLAP;
      else {
        uint64_t sh = 0;
        s = c->arena.alloc(q.n, &sh);
        if (s == CG_OK) c->table.insert(q.dst, q.n, sh);
      }
      finish(sl, s);
    } else if (q.op == CG_OP_FREE) {
      uint64_t sz = 0, sh = 0;
      if (c->table.remove_base(q.dst, &sz, &sh)) {
        deferred.push_back({sh, sz, round_tag});
        sl->res.verdict = CG_FREE_OK;
      } else if (c->table.find(q.dst).ok) {
        sl->res.verdict = CG_FREE_INTERIOR;
      } else if (c->table.freed.count(q.dst)) {
        sl->res.verdict = CG_FREE_DOUBLE;
      } else {
        sl->res.verdict = CG_FREE_UNKNOWN;
      }
      finish(sl, CG_OK);
    } else {
      finish(sl, CG_E_ARG);
    }
  }

  // Mark a device range defined/undefined between rounds (no round is in
  // flight when this runs).
  void apply_mark(RingSlot *sl, cudaStream_t s) {
    const cg_request &q = sl->req;
    cg_status stt = CG_OK;
    if (q.n) {
      const AllocTable::Hit h = c->table.find(q.dst);
      if (!h.ok || q.n > h.base + h.size - q.dst) {
        stt = CG_E_RANGE;
      } else {
        cudaError_t e = cudaSuccess;
        if (flush_fills(c, s) != CG_OK) e = cudaErrorUnknown;
        if (e == cudaSuccess)
          e = cudaMemsetAsync(reinterpret_cast<void *>(h.shadow + (q.dst - h.base)),
                              q.op == CG_OP_MARK_DEFINED ? 0x00 : 0xFF, q.n, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) stt = CG_E_CUDA;
      }
    }
    finish(sl, stt);
  }

  // Admit what the rings hold into round slot R and launch it.  Returns
  // whether anything was admitted.
  bool build_round(RoundSlot &R) {
    const uint64_t round_id = next_round;
    prune_window();
    std::vector<RingSlot *> members;
    std::vector<cg_copy> copies;
    std::vector<ScanJob> jobs;
    std::vector<RangeInfo> infos;
    std::vector<uint8_t> modes;
    std::vector<StageCopy> stages;
    std::vector<uint64_t> stage_ptr;
    uint64_t stage_bytes = 0;
    uint64_t bytes = 0;
    bool progress = false, closed = false;
    const size_t nc = rings.size();
    bool any = true;
    while (any && !closed) {
      any = false;
      for (size_t k = 0; k < nc && !closed; k++) {
        ClientRing &ring = rings[(rr + k) % nc];
        uint64_t t = ring.taken.load(std::memory_order_relaxed);
        const uint64_t h = ring.head.load(std::memory_order_acquire);
        for (int take = 0; t < h && take < 64; take++) {
          RingSlot *sl = &ring.slots[t & ring.mask];
          const cg_request &q = sl->req;
          if (q.op == CG_OP_CHECK) {
            if (members.size() >= cfg.max_round) {
              closed = true;
              break;
            }
            if (!members.empty() && inflight_bytes + bytes + q.n > cfg.budget_bytes) {
              std::lock_guard<std::mutex> g(stats_mu);
              st.budget_stalls++;
              closed = true;
              break;
            }
            sl->res = cg_result{};
            sl->res.seq = next_seq++;
            sl->race = nullptr;
            const cg_copy cq{q.kind, 0, q.dst, q.src, q.n};
            cg_status s = validate(c, cq);
            if (s != CG_OK) {
              finish(sl, s);
            } else if (!admit_check(sl, (uint32_t)((rr + k) % nc), cq, members, copies, jobs, infos,
                                    modes, stages, stage_ptr, stage_bytes, bytes)) {
              // finished on the host (n == 0 or nothing readable)
            }
          } else if (q.op == CG_OP_MARK_DEFINED || q.op == CG_OP_MARK_UNDEFINED) {
            if (!members.empty() || any_busy()) {  // marks run between rounds
              closed = true;
              break;
            }
            sl->res = cg_result{};
            sl->res.seq = next_seq++;
            apply_mark(sl, R.stream);
          } else {
            sl->res = cg_result{};
            sl->res.seq = next_seq++;
            apply_host_op(sl, round_id);
          }
          t++;
          any = true;
          progress = true;
        }
        ring.taken.store(t, std::memory_order_release);
      }
    }
    rr = (rr + 1) % nc;
    if (members.empty()) return progress;
    if (launch(R, round_id, members, copies, jobs, infos, modes, stages, stage_ptr, stage_bytes,
               bytes) != CG_OK) {
      for (RingSlot *sl : members) {
        finish(sl, CG_E_CUDA);
        mark_done(sl);
      }
    }
    return true;
  }

  // Host part of one admitted check.  Returns true if it joins the round.
  bool admit_check(RingSlot *sl, uint32_t client, const cg_copy &q,
                   std::vector<RingSlot *> &members,
                   std::vector<cg_copy> &copies, std::vector<ScanJob> &jobs,
                   std::vector<RangeInfo> &infos, std::vector<uint8_t> &modes,
                   std::vector<StageCopy> &stages, std::vector<uint64_t> &stage_ptr,
                   uint64_t &stage_bytes, uint64_t &bytes) {
    RangeInfo ri{};
    ri.kind = q.kind;
    ri.n = q.n;
    ScanJob job{};
    job.kind = q.kind;
    job.n = q.n;
    job.host_off = q.kind == CG_HTOD ? q.src : (q.kind == CG_DTOH ? q.dst : 0);
    const Acc none{0, 0, kNone, kNone};
    if (q.n == 0) {
      assemble_report(&sl->res.report, ri, none);
      finish(sl, CG_OK);
      return false;
    }
    bool dst_ok = true, src_ok = true;
    uint64_t dsh = 0, ssh = 0;
    if (q.kind != CG_DTOH)
      dst_ok = host_side(c, q.dst, q.n, &ri.found_dst, &ri.base_dst, &ri.size_dst, &dsh, &ri.flags,
                         CG_F_UNALLOC_DST, CG_F_OVERRUN_DST);
    if (q.kind != CG_HTOD)
      src_ok = host_side(c, q.src, q.n, &ri.found_src, &ri.base_src, &ri.size_src, &ssh, &ri.flags,
                         CG_F_UNALLOC_SRC, CG_F_OVERRUN_SRC);
    bool overlap = false;
    if (q.kind == CG_DTOD) {
      const uint64_t dist = q.src <= q.dst ? q.dst - q.src : q.src - q.dst;
      overlap = dist < q.n;
      if (overlap) ri.flags |= CG_F_DTOD_OVERLAP;
    }
    if (q.kind != CG_HTOD && src_ok) {
      job.mode |= kModeReadDev;
      job.dev_src = ssh;
    }
    if (c->cfg.carry && dst_ok && src_ok) {
      job.mode |= kModeCarry;
      if (q.kind != CG_DTOH) job.dev_dst = dsh;
    }
    // concurrent accesses (Sec. 2 itemize): an earlier copy of another
    // client still outstanding when this one was submitted, touching the
    // same data
    int64_t race = -1;
    const bool moved = dst_ok && src_ok;
    if (moved) {
      // the smallest seq among the window entries near this copy's ranges
      // that meet the definition
      auto consider = [&](uint64_t item) {
        const RaceEntry &e = *reinterpret_cast<const RaceEntry *>(item);
        if (race >= 0 && (int64_t)e.seq >= race) return;
        if (e.client != client && (e.done_ns == 0 || e.done_ns > sl->submit_ns) &&
            races_with(e, q.kind, q.dst, q.src, q.n))
          race = (int64_t)e.seq;
      };
      // (the copy's own entry, met when both ranges lie in one space, is
      // of this client and so never a race)
      window.push_back({sl->res.seq, client, q.kind, q.dst, q.src, q.n, 0});
      sl->race = &window.back();
      const uint64_t item = reinterpret_cast<uint64_t>(sl->race);
      window_index.visit_add(dst_space(q.kind), q.dst, q.n, item, consider);
      window_index.visit_add(src_space(q.kind), q.src, q.n, item, consider);
    }
    if (q.kind == CG_DTOD && !(job.mode & (kModeCarry | kModeReadDev))) {
      assemble_report(&sl->res.report, ri, none);
      finish(sl, CG_OK);
      mark_done(sl);
      return false;
    }
    sl->res.report.race_seq = race;
    uint64_t sp = 0;
    if (overlap && (job.mode & kModeCarry)) {  // staged through the round's buffer
      stages.push_back({0, ssh, stage_bytes, q.n});
      sp = stage_bytes + 1;
      stage_bytes += round_up(q.n, 256);
    }
    members.push_back(sl);
    copies.push_back(q);
    jobs.push_back(job);
    infos.push_back(ri);
    modes.push_back((uint8_t)job.mode);
    stage_ptr.push_back(sp);
    bytes += q.n;
    return true;
  }

  cg_status launch(RoundSlot &R, uint64_t round_id, std::vector<RingSlot *> &members,
                   std::vector<cg_copy> &copies, std::vector<ScanJob> &jobs,
                   std::vector<RangeInfo> &infos, std::vector<uint8_t> &modes,
                   std::vector<StageCopy> &stages, std::vector<uint64_t> &stage_ptr,
                   uint64_t stage_bytes, uint64_t bytes) {
    NvtxRange range("cg serve: launch round");
    const uint64_t n = members.size();
    cudaStream_t s = R.stream;
    // dependency levels inside the round
    const std::vector<int> lvl = plan_levels(copies.data(), n, c->cfg.carry != 0, modes.data());
    int nlev = 0;
    for (int l : lvl) nlev = std::max(nlev, l + 1);
    std::vector<uint64_t> lev_start(nlev + 1, 0);
    for (int l : lvl) lev_start[l + 1]++;
    for (int l = 0; l < nlev; l++) lev_start[l + 1] += lev_start[l];
    // packed upload: jobs | info | acc | order | seg_first | stage
    const uint64_t o_jobs = 0;
    const uint64_t o_info = round_up(o_jobs + n * sizeof(ScanJob), 16);
    const uint64_t o_acc = round_up(o_info + n * sizeof(RangeInfo), 16);
    const uint64_t o_order = round_up(o_acc + n * sizeof(Acc), 16);
    const uint64_t o_seg = round_up(o_order + n * 4, 16);
    const uint64_t o_stage = round_up(o_seg + n * 8, 16);
    const uint64_t o_err = round_up(o_stage + n * 8, 16);
    const uint64_t total = o_err + 16;  // uploaded
    const uint64_t down = 16 + n * sizeof(cg_report);
    CG_TRY(R.h_up.ensure(total));
    CG_TRY(R.d_up.ensure(total));
    CG_TRY(R.h_down.ensure(down));
    if (stage_bytes) {
      CG_TRY(R.stage.ensure(stage_bytes));
      const uint64_t base = reinterpret_cast<uint64_t>(R.stage.p);
      for (auto &v : stage_ptr)
        if (v) v = base + v - 1;
      size_t k = 0;
      for (uint64_t i = 0; i < n; i++)
        if (stage_ptr[i]) {
          stages[k].level = lvl[i];
          stages[k].off += base;
          jobs[i].dev_src = stage_ptr[i];
          k++;
        }
    }
    uint8_t *h = R.h_up.p;
    std::memcpy(h + o_jobs, jobs.data(), n * sizeof(ScanJob));
    std::memcpy(h + o_info, infos.data(), n * sizeof(RangeInfo));
    Acc *ha = reinterpret_cast<Acc *>(h + o_acc);
    for (uint64_t i = 0; i < n; i++) ha[i] = Acc{0, 0, kNone, kNone};
    uint32_t *ho = reinterpret_cast<uint32_t *>(h + o_order);
    uint64_t *hs = reinterpret_cast<uint64_t *>(h + o_seg);
    std::memcpy(h + o_stage, stage_ptr.data(), n * 8);
    std::memset(h + o_err, 0, 16);
    {
      std::vector<uint64_t> fill(lev_start.begin(), lev_start.end() - 1);
      for (uint64_t i = 0; i < n; i++) ho[fill[lvl[i]]++] = (uint32_t)i;
    }
    const uint64_t quantum =
        (c->img_on_host || c->cfg.scan_engine == 1) ? 2048 : scan_tma_tile_bytes();
    uint64_t seg_bytes = (uint64_t)(c->cfg.batch_segment_kib ? c->cfg.batch_segment_kib : 64) * 1024;
    seg_bytes = std::max<uint64_t>(quantum, (seg_bytes + quantum - 1) / quantum * quantum);
    const uint64_t seg_chunks = seg_bytes / 16;
    std::vector<uint64_t> lev_segs(nlev, 0);
    for (int l = 0; l < nlev; l++) {
      uint64_t acc_segs = 0;
      for (uint64_t pos = lev_start[l]; pos < lev_start[l + 1]; pos++) {
        hs[pos] = acc_segs;
        acc_segs += (((copies[ho[pos]].n + 30) >> 4) + seg_chunks - 1) / seg_chunks;
      }
      lev_segs[l] = acc_segs;
    }
    // footprint for the cross-round hazard test
    R.fp.clear();
    for (uint64_t i = 0; i < n; i++) {
      const cg_copy &q = copies[i];
      const ScanJob &j = jobs[i];
      if (q.kind == CG_HTOD) R.fp.hr.push_back({q.src, q.src + q.n});
      if (q.kind == CG_DTOH && (j.mode & kModeCarry)) R.fp.hw.push_back({q.dst, q.dst + q.n});
      if (j.mode & kModeReadDev) {
        const uint64_t src_sh = stage_ptr[i] ? 0 : j.dev_src;
        if (src_sh) R.fp.dr.push_back({src_sh, src_sh + q.n});
      }
      if ((j.mode & kModeCarry) && q.kind != CG_DTOH) R.fp.dw.push_back({j.dev_dst, j.dev_dst + q.n});
    }
    for (const auto &sc : stages) R.fp.dr.push_back({sc.src, sc.src + sc.n});
    // shadow slots refilled by this round's stream count as its writes
    for (size_t k = 0; k < c->fill_ptr.size(); k++)
      R.fp.dw.push_back({c->fill_ptr[k], c->fill_ptr[k] + round_up(c->fill_size[k], 256)});
    R.fp.sort_all();
    bool waited = false;
    for (auto &o : rs) {
      if (&o == &R || !o.busy) continue;
      if (conflicts(R.fp, o.fp)) {
        CG_CUDA(cudaStreamWaitEvent(s, o.done, 0));
        waited = true;
      }
    }
    CG_TRY(flush_fills(c, s));
    CG_CUDA(cudaMemcpyAsync(R.d_up.p, h, total, cudaMemcpyHostToDevice, s));
    unsigned int *d_err = reinterpret_cast<unsigned int *>(R.d_up.p + o_err);
    BatchPlan plan{};
    plan.reqs = nullptr;
    plan.jobs = reinterpret_cast<ScanJob *>(R.d_up.p + o_jobs);
    plan.info = reinterpret_cast<RangeInfo *>(R.d_up.p + o_info);
    plan.acc = reinterpret_cast<Acc *>(R.d_up.p + o_acc);
    plan.order = reinterpret_cast<const uint32_t *>(R.d_up.p + o_order);
    plan.seg_first = reinterpret_cast<const uint64_t *>(R.d_up.p + o_seg);
    plan.stage = reinterpret_cast<const uint64_t *>(R.d_up.p + o_stage);
    plan.nreq = n;
    plan.seg_chunks = (uint32_t)seg_chunks;
    plan.mode_mask = ~0u;
    std::sort(stages.begin(), stages.end(),
              [](const StageCopy &a, const StageCopy &b) { return a.level < b.level; });
    size_t sci = 0;
    uint64_t kernels = 0;
    const bool tma = !(c->img_on_host || c->cfg.scan_engine == 1);
    // a one-level round of a few copies: the level kernel's last CTA writes
    // the reports (one launch less per round)
    FinalizeHost fin;
    if (tma && nlev == 1 && lev_segs[0] > 0 && n <= 512) {
      fin.out = R.h_down.p;
      fin.done = d_err + 1;  // zeroed by the upload with the flag
    }
    for (int l = 0; l < nlev; l++) {
      for (; sci < stages.size() && stages[sci].level == l; sci++)
        CG_CUDA(cudaMemcpyAsync(reinterpret_cast<void *>(stages[sci].off),
                                reinterpret_cast<const void *>(stages[sci].src), stages[sci].n,
                                cudaMemcpyDeviceToDevice, s));
      if (!tma)
        CG_CUDA(launch_scan_level(c->img, plan, lev_start[l], lev_start[l + 1], lev_segs[l],
                                  c->sm_count * 8, s));
      else
        CG_CUDA(launch_scan_level_tma(c->img, plan, lev_start[l], lev_start[l + 1], lev_segs[l],
                                      c->sm_count, nullptr, d_err, false, s, fin));
      kernels++;
    }
    if (!fin.out) {
      CG_CUDA(launch_finalize_host(plan, d_err, R.h_down.p, s));
      kernels++;
    }
    CG_CUDA(cudaEventRecord(R.done, s));
    R.busy = true;
    R.id = round_id;
    R.bytes = bytes;
    R.members.swap(members);
    next_round++;
    inflight_bytes += bytes;
    std::lock_guard<std::mutex> g(stats_mu);
    st.checks += n;
    st.rounds++;
    st.round_checks_max = std::max<uint64_t>(st.round_checks_max, n);
    st.bytes_checked += bytes;
    st.inflight_bytes_max = std::max(st.inflight_bytes_max, inflight_bytes);
    if (waited) st.conflict_waits++;
    c->stats.kernels += kernels;
    c->stats.levels += (uint64_t)nlev;
    return CG_OK;
  }

  void run() {
    uint32_t idle = 0;
    for (;;) {
      bool progress = complete_rounds();
      if (stop.load(std::memory_order_acquire) && rings_empty() && !any_busy()) break;
      for (auto &r : rs) {
        if (r.busy) continue;
        if (build_round(r)) progress = true;
        break;  // one round per pass keeps completions prompt
      }
      if (progress) {
        idle = 0;
      } else if (++idle > 64) {
        std::this_thread::yield();
      }
    }
    release_deferred(~0ull);
  }
};

}  // namespace cgi

using namespace cgi;

extern "C" {

cg_status cg_serve_start(cg_ctx *c, const cg_serve_config *cfg_in) {
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (c->serve) return set_error(CG_E_STATE, "already serving");
  cg_serve_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (!cfg.clients) cfg.clients = 8;
  if (!cfg.ring_capacity) cfg.ring_capacity = 4096;
  if (!cfg.max_round) cfg.max_round = 8192;
  if (!cfg.streams) cfg.streams = 4;
  if (!cfg.budget_bytes) cfg.budget_bytes = 8ull << 30;
  if (cfg.clients > 64 || cfg.streams > 8 || (cfg.ring_capacity & (cfg.ring_capacity - 1)) ||
      cfg.ring_capacity < 2)
    return set_error(CG_E_ARG, "clients <= 64, streams <= 8, ring_capacity a power of two >= 2");
  auto *e = new (std::nothrow) ServeEngine(c, cfg.clients);
  if (!e) return set_error(CG_E_NOMEM, "serve engine");
  e->cfg = cfg;
  for (auto &r : e->rings) {
    r.slots.reset(new (std::nothrow) RingSlot[cfg.ring_capacity]);
    if (!r.slots) {
      delete e;
      return set_error(CG_E_NOMEM, "client ring");
    }
    r.mask = cfg.ring_capacity - 1;
    for (uint32_t i = 0; i < cfg.ring_capacity; i++) r.slots[i].state.store(0);
  }
  e->rs.resize(cfg.streams);
  for (auto &r : e->rs) {
    cudaError_t err = cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
    if (err != cudaSuccess) {
      for (auto &x : e->rs) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.done) cudaEventDestroy(x.done);
      }
      delete e;
      return cuda_fail(err, "cg_serve_start");
    }
  }
  c->serve = e;
  e->th = std::thread([e] { e->run(); });
  return CG_OK;
}

cg_status cg_submit(cg_ctx *c, uint32_t client, const cg_request *req, uint64_t *ticket) {
  if (!c || !req || !ticket) return set_error(CG_E_ARG, "NULL argument");
  ServeEngine *e = c->serve;
  if (!e) return set_error(CG_E_STATE, "not serving");
  if (client >= e->rings.size()) return set_error(CG_E_ARG, "client index out of range");
  if (e->stop.load(std::memory_order_relaxed)) return set_error(CG_E_STATE, "stopping");
  ClientRing &r = e->rings[client];
  const uint64_t h = r.head.load(std::memory_order_relaxed);
  if (h - r.collected.load(std::memory_order_relaxed) > r.mask) return CG_E_FULL;
  RingSlot &sl = r.slots[h & r.mask];
  sl.req = *req;
  // the race window relies on this order: announce, then take the time
  r.submitting.store(1, std::memory_order_seq_cst);
  const uint64_t t = now_ns();
  r.submitting.store(t, std::memory_order_seq_cst);
  sl.submit_ns = t;
  sl.state.store(1, std::memory_order_relaxed);
  r.head.store(h + 1, std::memory_order_release);
  r.submitting.store(0, std::memory_order_release);
  *ticket = ((uint64_t)client << 56) | h;
  return CG_OK;
}

cg_status cg_poll(cg_ctx *c, uint64_t ticket, cg_result *out) {
  if (!c || !out) return set_error(CG_E_ARG, "NULL argument");
  ServeEngine *e = c->serve;
  if (!e) return set_error(CG_E_STATE, "not serving");
  const uint64_t client = ticket >> 56, idx = ticket & ((1ull << 56) - 1);
  if (client >= e->rings.size()) return set_error(CG_E_ARG, "unknown ticket");
  ClientRing &r = e->rings[client];
  const uint64_t col = r.collected.load(std::memory_order_relaxed);
  if (idx < col || idx >= r.head.load(std::memory_order_relaxed))
    return set_error(CG_E_ARG, "unknown or collected ticket");
  RingSlot &sl = r.slots[idx & r.mask];
  const uint32_t s = sl.state.load(std::memory_order_acquire);
  if (s == 3) return set_error(CG_E_ARG, "ticket already collected");
  if (s != 2) return CG_PENDING;
  *out = sl.res;
  sl.state.store(3, std::memory_order_relaxed);
  uint64_t k = col;
  while (k < r.head.load(std::memory_order_relaxed) &&
         r.slots[k & r.mask].state.load(std::memory_order_relaxed) == 3) {
    r.slots[k & r.mask].state.store(0, std::memory_order_relaxed);
    k++;
  }
  r.collected.store(k, std::memory_order_release);
  return CG_OK;
}

cg_status cg_wait(cg_ctx *c, uint64_t ticket, uint32_t timeout_ms, cg_result *out) {
  const uint64_t t0 = now_ns();
  for (uint32_t it = 0;; it++) {
    const cg_status s = cg_poll(c, ticket, out);
    if (s != CG_PENDING) return s;
    if ((uint64_t)timeout_ms * 1000000ull < now_ns() - t0)
      return set_error(CG_E_TIMEOUT, "result not ready in time");
    if (it > 256) std::this_thread::yield();
  }
}

cg_status cg_serve_replay(cg_ctx *c, const cg_request *reqs, const uint32_t *client,
                          const uint64_t *arrival_ns, uint64_t n, cg_result *results) {
  if (!c || (n && (!reqs || !client || !arrival_ns || !results)))
    return set_error(CG_E_ARG, "NULL argument");
  ServeEngine *e = c->serve;
  if (!e) return set_error(CG_E_STATE, "not serving");
  const uint32_t nc = (uint32_t)e->rings.size();
  for (uint64_t i = 0; i < n; i++)
    if (client[i] >= nc) return set_error(CG_E_ARG, "client index out of range");
  std::atomic<int> failed{CG_OK};
  const uint64_t start = now_ns();
  auto worker = [&](uint32_t me) {
    std::deque<std::pair<uint64_t, uint64_t>> pending;  // (ticket, index)
    auto collect = [&](bool block) {
      while (!pending.empty()) {
        cg_result r;
        const cg_status s = block ? cg_wait(c, pending.front().first, 600000, &r)
                                  : cg_poll(c, pending.front().first, &r);
        if (s == CG_PENDING) return;
        if (s != CG_OK) {
          failed.store(s);
          return;
        }
        results[pending.front().second] = r;
        pending.pop_front();
      }
    };
    for (uint64_t i = 0; i < n && failed.load() == CG_OK; i++) {
      if (client[i] != me) continue;
      while (now_ns() - start < arrival_ns[i]) collect(false);
      uint64_t t = 0;
      for (;;) {
        const cg_status s = cg_submit(c, me, &reqs[i], &t);
        if (s == CG_OK) break;
        if (s != CG_E_FULL) {
          failed.store(s);
          return;
        }
        collect(false);
        std::this_thread::yield();
      }
      pending.emplace_back(t, i);
      collect(false);
    }
    collect(true);
  };
  std::vector<std::thread> ts;
  for (uint32_t k = 0; k < nc; k++) ts.emplace_back(worker, k);
  for (auto &t : ts) t.join();
  return (cg_status)failed.load();
}

cg_status cg_serve_stop(cg_ctx *c, cg_serve_stats *out) {
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  ServeEngine *e = c->serve;
  if (!e) return set_error(CG_E_STATE, "not serving");
  e->stop.store(true, std::memory_order_release);
  e->th.join();
  for (auto &r : e->rs) {
    cudaStreamSynchronize(r.stream);
    cudaStreamDestroy(r.stream);
    cudaEventDestroy(r.done);
    r.d_up.release();
    r.stage.release();
    r.h_up.release();
    r.h_down.release();
  }
  if (out) {
    std::lock_guard<std::mutex> g(e->stats_mu);
    *out = e->st;
    out->requests = e->next_seq;
  }
  c->serve = nullptr;
  delete e;
  return CG_OK;
}

}  // extern "C"

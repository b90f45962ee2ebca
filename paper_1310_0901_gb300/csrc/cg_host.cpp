// cg_host.cpp -- host runtime of libcg: the C ABI entry points of cg.h
// (the structures they use are in cg_ctx.h).
#include <cuda_runtime.h>

#include "cg_ctx.h"

using namespace cgi;

// ------------------------------------------------------------- errors

static thread_local std::string g_last_error;

cg_status cgi::set_error(cg_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

void cgi::set_error_text(const char *msg) { g_last_error = msg; }

cg_status cgi::cuda_fail(cudaError_t e, const char *what) {
  return set_error(CG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

// An endpoint of a range, tagged with its owner's index and slot.
struct Ep {
  uint64_t v;
  uint32_t req;
  uint32_t slot;
};

// Rank of each endpoint's value among the distinct values, written to
// idx[stride * req + slot]; returns the number of distinct values.  Large
// sets sort by LSD radix (11-bit digits, skipping digits no two keys differ
// in), small ones directly (only the ranks matter, so ties may go either way).
int compress_endpoints(std::vector<Ep> &e, int32_t *idx, int stride) {
  if (e.size() < 1024) {
    std::sort(e.begin(), e.end(), [](const Ep &a, const Ep &b) { return a.v < b.v; });
  } else {
    std::vector<Ep> tmp(e.size());
    uint64_t any = 0, all = ~0ull;
    for (const Ep &x : e) {
      any |= x.v;
      all &= x.v;
    }
    const uint64_t differ = any ^ all;
    for (int shift = 0; shift < 64; shift += 11) {
      if (((differ >> shift) & 2047) == 0) continue;
      uint32_t cnt[2048] = {0};
      for (const Ep &x : e) cnt[(x.v >> shift) & 2047]++;
      uint32_t sum = 0;
      for (int d = 0; d < 2048; d++) {
        const uint32_t c = cnt[d];
        cnt[d] = sum;
        sum += c;
      }
      for (const Ep &x : e) tmp[cnt[(x.v >> shift) & 2047]++] = x;
      e.swap(tmp);
    }
  }
  int rank = -1;
  uint64_t prev = 0;
  for (size_t k = 0; k < e.size(); k++) {
    if (k == 0 || e[k].v != prev) rank++;
    prev = e[k].v;
    idx[(size_t)stride * e[k].req + e[k].slot] = rank;
  }
  return rank + 1;
}

}  // namespace

// Dependency levels for sequential semantics (R15): a copy's level is one
// more than the highest level of any earlier copy it conflicts with (it
// reads what that copy writes, writes what it reads, or writes what it
// writes).  With `modes` (the device lookup's per-copy job modes) a copy
// writes its destination only if it carries and reads a device source only
// if that source is valid; without, every copy is taken to read its source
// and write its destination.  Levels run in order; copies within a level
// touch disjoint shadow.
std::vector<int> cgi::plan_levels(const cg_copy *reqs, uint64_t nreq, bool carry,
                                  const uint8_t *modes) {
  std::vector<int> lvl(nreq, 0);
  if (!carry || nreq < 2) return lvl;
  auto end_of = [](uint64_t a, uint64_t n) { return a + n < a ? ~0ull : a + n; };
  auto reads_dev = [&](uint64_t i) { return !modes || (modes[i] & kModeReadDev); };
  auto writes = [&](uint64_t i) { return !modes || (modes[i] & kModeCarry); };
  // endpoints of every range, tagged (request, slot): slots 0/1 host read,
  // 2/3 host write, 4/5 device read, 6/7 device write
  std::vector<Ep> he, de;
  he.reserve(2 * nreq);
  de.reserve(2 * nreq);
  for (uint64_t i = 0; i < nreq; i++) {
    const cg_copy &q = reqs[i];
    if (q.n == 0) continue;
    const uint32_t r = (uint32_t)i;
    if (q.kind == CG_HTOD) {
      he.push_back({q.src, r, 0});
      he.push_back({q.src + q.n, r, 1});
      if (writes(i)) {
        de.push_back({q.dst, r, 6});
        de.push_back({end_of(q.dst, q.n), r, 7});
      }
    } else if (q.kind == CG_DTOH) {
      if (writes(i)) {
        he.push_back({q.dst, r, 2});
        he.push_back({q.dst + q.n, r, 3});
      }
      if (reads_dev(i)) {
        de.push_back({q.src, r, 4});
        de.push_back({end_of(q.src, q.n), r, 5});
      }
    } else {
      if (reads_dev(i)) {
        de.push_back({q.src, r, 4});
        de.push_back({end_of(q.src, q.n), r, 5});
      }
      if (writes(i)) {
        de.push_back({q.dst, r, 6});
        de.push_back({end_of(q.dst, q.n), r, 7});
      }
    }
  }
  std::vector<int32_t> idx(8 * nreq, -1);
  LevelTree ht, dt;
  ht.init(compress_endpoints(he, idx.data(), 8));
  dt.init(compress_endpoints(de, idx.data(), 8));
  for (uint64_t i = 0; i < nreq; i++) {
    if (reqs[i].n == 0) continue;
    const int32_t *x = &idx[8 * i];
    int l = -1;
    if (x[0] >= 0) l = std::max(l, ht.query(x[0], x[1], false));
    if (x[2] >= 0) l = std::max(l, ht.query(x[2], x[3], true));
    if (x[4] >= 0) l = std::max(l, dt.query(x[4], x[5], false));
    if (x[6] >= 0) l = std::max(l, dt.query(x[6], x[7], true));
    l += 1;
    if (x[0] >= 0) ht.update_r(x[0], x[1], l);
    if (x[2] >= 0) ht.update_w(x[2], x[3], l);
    if (x[4] >= 0) dt.update_r(x[4], x[5], l);
    if (x[6] >= 0) dt.update_w(x[6], x[7], l);
    lvl[i] = l;
  }
  return lvl;
}

namespace {

// Conflicts in the host space, exact, per 64 KiB block of the host image.
// A block keeps the highest write and read levels of every unit that
// touched it (w_any, r_any), of the units that covered it whole (w_full,
// r_full), and the exact ranges of up to kCap units that touched it only
// in part.  A range meets an earlier unit iff, in a block it covers whole,
// that block's *_any levels say so, or, in a block at one of its ends, the
// unit covered the block whole or is one of the block's partial entries
// that overlaps it.  A block with more partial entries than kCap falls
// back to its *_any levels (conservative: it may order units that do not
// overlap).  Cost per unit: the blocks it spans plus two short scans.
struct HostConflicts {
  static constexpr int kShift = 16;
  static constexpr int kCap = 8;
  struct Entry {
    uint64_t lo, hi;
    int level;
    bool write;
  };
  struct Slot {
    int n = 0;
    bool over = false;
    Entry e[kCap];
  };
  std::vector<int> w_any, r_any, w_full, r_full;
  std::vector<int32_t> slot_of;  // -1: no partial entries
  std::vector<Slot> slots;

  explicit HostConflicts(uint64_t host_n) {
    const size_t nb = (size_t)(host_n >> kShift) + 2;
    w_any.assign(nb, -1);
    r_any.assign(nb, -1);
    w_full.assign(nb, -1);
    r_full.assign(nb, -1);
    slot_of.assign(nb, -1);
  }
  // highest level of an earlier unit that writes within [a, b), or (write)
  // reads or writes within it
  int query(uint64_t a, uint64_t b, bool write) const {
    int l = -1;
    if (b <= a) return l;
    const uint64_t k0 = a >> kShift, k1 = (b - 1) >> kShift;
    // the blocks the range covers whole: everything that touched them
    const uint64_t f0 = (a + (1ull << kShift) - 1) >> kShift, f1 = b >> kShift;
    for (uint64_t k = f0; k < f1; k++) {
      l = std::max(l, w_any[k]);
      if (write) l = std::max(l, r_any[k]);
    }
    // the blocks at its ends that it covers in part
    auto edge = [&](uint64_t k) {
      const int32_t sl = slot_of[k];
      if (sl >= 0 && slots[sl].over) {
        l = std::max(l, w_any[k]);
        if (write) l = std::max(l, r_any[k]);
        return;
      }
      l = std::max(l, w_full[k]);
      if (write) l = std::max(l, r_full[k]);
      if (sl < 0) return;
      const Slot &s = slots[sl];
      for (int j = 0; j < s.n; j++)
        if ((s.e[j].write || write) && s.e[j].lo < b && a < s.e[j].hi)
          l = std::max(l, s.e[j].level);
    };
    if (k0 < f0 || f0 >= f1) edge(k0);
    if (k1 != k0 && k1 >= f1) edge(k1);
    return l;
  }
  void update(uint64_t a, uint64_t b, bool write, int level) {
    if (b <= a) return;
    const uint64_t k0 = a >> kShift, k1 = (b - 1) >> kShift;
    const uint64_t f0 = (a + (1ull << kShift) - 1) >> kShift, f1 = b >> kShift;
    std::vector<int> &any = write ? w_any : r_any;
    std::vector<int> &full = write ? w_full : r_full;
    for (uint64_t k = f0; k < f1; k++) {
      any[k] = std::max(any[k], level);
      full[k] = std::max(full[k], level);
    }
    auto edge = [&](uint64_t k) {
      any[k] = std::max(any[k], level);
      if (slot_of[k] < 0) {
        slot_of[k] = (int32_t)slots.size();
        slots.emplace_back();
      }
      Slot &s = slots[slot_of[k]];
      if (s.n < kCap)
        s.e[s.n++] = Entry{a, b, level, write};
      else
        s.over = true;
    };
    if (k0 < f0 || f0 >= f1) edge(k0);
    if (k1 != k0 && k1 >= f1) edge(k1);
  }
};

}  // namespace

// Dependency levels over planning units (R15).  A host->device copy that
// carries nothing only reads its host bytes; a long one is cut into pieces
// of piece_rows rows of its anchor grid (the host buffer, 16-byte aligned,
// so the anchor offset is the host offset mod 16), each planned as a unit
// of its own: a piece waits only for the writes it overlaps, not for every
// write the whole copy overlaps.  The pieces of a copy add to the same
// report (counts and first offsets are sums and minima).
//
// Conflicts in the host space are tracked per 64 KiB block of the host
// image (HostConflicts: exact unless a block holds many partial ranges,
// and linear in the bytes planned); the device space keeps the exact
// interval tree.
std::vector<PlanUnit> cgi::plan_pieces(const cg_copy *reqs, uint64_t nreq, bool carry,
                                       const uint8_t *modes, uint64_t host_n,
                                       uint64_t piece_rows) {
  std::vector<PlanUnit> units;
  units.reserve(nreq + nreq / 4);
  auto reads_dev = [&](uint64_t i) { return !modes || (modes[i] & kModeReadDev); };
  auto writes = [&](uint64_t i) { return !modes || (modes[i] & kModeCarry); };
  for (uint64_t i = 0; i < nreq; i++) {
    const cg_copy &q = reqs[i];
    const uint64_t ax = q.src & 15;
    const uint64_t rows = (((ax + q.n + 15) >> 4) + 31) >> 5;
    if (carry && piece_rows && q.kind == CG_HTOD && !writes(i) && rows > piece_rows + piece_rows / 2) {
      for (uint64_t r = 0; r < rows; r += piece_rows)
        units.push_back({(uint32_t)i, (uint32_t)r, (uint32_t)std::min(rows, r + piece_rows), 0});
    } else {
      units.push_back({(uint32_t)i, 0u, 0u, 0});
    }
  }
  if (!carry) return units;  // nothing is written: every unit at level 0
  // host bytes [lo, hi) a unit reads or writes (0, 0: none)
  auto host_range = [&](const PlanUnit &u, bool &is_write) -> std::pair<uint64_t, uint64_t> {
    const cg_copy &q = reqs[u.req];
    is_write = false;
    if (q.n == 0) return {0, 0};
    if (q.kind == CG_HTOD) {
      if (!u.rhi) return {q.src, q.src + q.n};
      const int64_t ax = (int64_t)(q.src & 15);
      const int64_t b0 = std::max<int64_t>(0, 512 * (int64_t)u.rlo - ax);
      const int64_t b1 = std::min<int64_t>((int64_t)q.n, 512 * (int64_t)u.rhi - ax);
      return {q.src + (uint64_t)b0, q.src + (uint64_t)b1};
    }
    if (q.kind == CG_DTOH && writes(u.req)) {
      is_write = true;
      return {q.dst, q.dst + q.n};
    }
    return {0, 0};
  };
  HostConflicts hc(host_n);
  // device space: the exact tree over compressed endpoints
  auto end_of = [](uint64_t a, uint64_t n) { return a + n < a ? ~0ull : a + n; };
  std::vector<Ep> de;
  de.reserve(4 * nreq);
  for (const PlanUnit &u : units) {
    const cg_copy &q = reqs[u.req];
    if (q.n == 0 || u.rhi) continue;
    if ((q.kind == CG_DTOH || q.kind == CG_DTOD) && reads_dev(u.req)) {
      de.push_back({q.src, u.req, 0});
      de.push_back({end_of(q.src, q.n), u.req, 1});
    }
    if ((q.kind == CG_HTOD || q.kind == CG_DTOD) && writes(u.req)) {
      de.push_back({q.dst, u.req, 2});
      de.push_back({end_of(q.dst, q.n), u.req, 3});
    }
  }
  std::vector<int32_t> rk(4 * nreq, -1);
  LevelTree dt;
  dt.init(compress_endpoints(de, rk.data(), 4));
  for (PlanUnit &u : units) {
    const cg_copy &q = reqs[u.req];
    if (q.n == 0) continue;
    bool hwrite = false;
    const auto h = host_range(u, hwrite);
    int l = hc.query(h.first, h.second, hwrite);
    const bool drd = !u.rhi && (q.kind == CG_DTOH || q.kind == CG_DTOD) && reads_dev(u.req);
    const bool dwr = !u.rhi && (q.kind == CG_HTOD || q.kind == CG_DTOD) && writes(u.req);
    int r0 = 0, r1 = 0, w0 = 0, w1 = 0;
    if (drd) {
      r0 = rk[4 * (size_t)u.req];
      r1 = rk[4 * (size_t)u.req + 1];
      l = std::max(l, dt.query(r0, r1, false));
    }
    if (dwr) {
      w0 = rk[4 * (size_t)u.req + 2];
      w1 = rk[4 * (size_t)u.req + 3];
      l = std::max(l, dt.query(w0, w1, true));
    }
    l += 1;
    hc.update(h.first, h.second, hwrite, l);
    if (drd) dt.update_r(r0, r1, l);
    if (dwr) dt.update_w(w0, w1, l);
    u.level = l;
  }
  return units;
}

// Queue 0xFF refills of released shadow ranges on `st`.
cg_status cgi::flush_fills(cg_ctx *c, cudaStream_t st) {
  const uint64_t n = c->fill_ptr.size();
  if (n == 0) return CG_OK;
  if (n <= 8) {
    for (uint64_t i = 0; i < n; i++)
      CG_CUDA(cudaMemsetAsync(reinterpret_cast<void *>(c->fill_ptr[i]), 0xFF,
                              round_up(c->fill_size[i], 256), st));
  } else {
    CG_TRY(c->h_fill.ensure(2 * n));
    CG_TRY(c->d_fill.ensure(2 * n));
    for (uint64_t i = 0; i < n; i++) {
      c->h_fill.p[i] = c->fill_ptr[i];
      c->h_fill.p[n + i] = round_up(c->fill_size[i], 256);
    }
    CG_CUDA(cudaMemcpyAsync(c->d_fill.p, c->h_fill.p, 2 * n * sizeof(uint64_t),
                            cudaMemcpyHostToDevice, st));
    CG_CUDA(launch_fill(c->d_fill.p, c->d_fill.p + n, n, 0xFF, st));
    c->stats.kernels++;
    // the pinned list is reused by the next flush: wait for this copy
    CG_CUDA(cudaStreamSynchronize(st));
  }
  c->fill_ptr.clear();
  c->fill_size.clear();
  return CG_OK;
}

// Bring the device copy of the table up to date.  While the device copy
// is tracked, only the registrations and the freed bases since its last
// update are uploaded, and the merge kernel builds the new table on the
// device; otherwise (first use, or too many changes) the host merges and
// the whole table is uploaded.
cg_status cgi::ensure_device_table(cg_ctx *c, cudaStream_t st) {
  AllocTable &t = c->table;
  if (t.dev_track) {
    const uint64_t m = t.dev_added.size(), d = t.dev_removed.size();
    if (m == 0 && d == 0) return CG_OK;
    if (d <= c->t_count && c->t_count - d + m == t.live) {
      const uint64_t n_new = t.live;
      CG_TRY(c->t_base2.ensure(n_new));
      CG_TRY(c->t_size2.ensure(n_new));
      CG_TRY(c->t_shadow2.ensure(n_new));
      CG_TRY(c->t_delta.ensure(3 * m + d));
      if (!c->t_ev) CG_CUDA(cudaEventCreateWithFlags(&c->t_ev, cudaEventDisableTiming));
      CG_CUDA(cudaEventSynchronize(c->t_ev));  // the staging buffer's last copy is done
      CG_TRY(c->h_tdelta.ensure(3 * m + d));
      uint64_t *h = c->h_tdelta.p;
      uint64_t k = 0;
      for (const auto &e : t.dev_added) {
        h[k] = e.first;
        h[m + k] = e.second.first;
        h[2 * m + k] = e.second.second;
        k++;
      }
      std::copy(t.dev_removed.begin(), t.dev_removed.end(), h + 3 * m);
      std::sort(h + 3 * m, h + 3 * m + d);
      if (3 * m + d)
        CG_CUDA(cudaMemcpyAsync(c->t_delta.p, h, (3 * m + d) * 8, cudaMemcpyHostToDevice, st));
      const uint64_t *dd = c->t_delta.p;
      DevTable old{c->t_base.p, c->t_size.p, c->t_shadow.p, c->t_count};
      CG_CUDA(launch_table_merge(old, dd, dd + m, dd + 2 * m, m, dd + 3 * m, d, c->t_base2.p,
                                 c->t_size2.p, c->t_shadow2.p, c->sm_count, st));
      CG_CUDA(cudaEventRecord(c->t_ev, st));
      c->stats.kernels++;
      c->stats.table_merges++;
      std::swap(c->t_base.p, c->t_base2.p);
      std::swap(c->t_base.cap, c->t_base2.cap);
      std::swap(c->t_size.p, c->t_size2.p);
      std::swap(c->t_size.cap, c->t_size2.cap);
      std::swap(c->t_shadow.p, c->t_shadow2.p);
      std::swap(c->t_shadow.cap, c->t_shadow2.cap);
      c->t_count = n_new;
      t.dev_synced();
      return CG_OK;
    }
  }
  if (!t.delta.empty() || t.dead) t.merge();
  if (c->t_ev) CG_CUDA(cudaEventSynchronize(c->t_ev));  // a merge may still write t_base
  const uint64_t n = t.base.size();
  CG_TRY(c->t_base.ensure(n));
  CG_TRY(c->t_size.ensure(n));
  CG_TRY(c->t_shadow.ensure(n));
  if (n) {
    CG_CUDA(cudaMemcpyAsync(c->t_base.p, t.base.data(), n * 8, cudaMemcpyHostToDevice, st));
    CG_CUDA(cudaMemcpyAsync(c->t_size.p, t.size.data(), n * 8, cudaMemcpyHostToDevice, st));
    CG_CUDA(cudaMemcpyAsync(c->t_shadow.p, t.shadow.data(), n * 8, cudaMemcpyHostToDevice, st));
    CG_CUDA(cudaStreamSynchronize(st));  // host vectors may change after return
  }
  c->t_count = n;
  c->stats.table_uploads++;
  t.dev_synced();
  return CG_OK;
}

cg_status cgi::validate(const cg_ctx *c, const cg_copy &q) {
  if (q.kind != CG_HTOD && q.kind != CG_DTOH && q.kind != CG_DTOD)
    return set_error(CG_E_KIND, "copy kind must be CG_HTOD, CG_DTOH or CG_DTOD");
  if (q.reserved != 0) return set_error(CG_E_ARG, "cg_copy.reserved must be 0");
  if (q.kind != CG_DTOD) {
    if (!c->img_bound) return set_error(CG_E_NO_HOST, "no host shadow image bound");
    const uint64_t h = q.kind == CG_HTOD ? q.src : q.dst;
    if (h > c->img.n || q.n > c->img.n - h)
      return set_error(CG_E_HOST_RANGE, "host range outside the bound host image");
  }
  return CG_OK;
}

// Host-mirror lookup of one device side (Sec. 2 itemize; R7, R8).
bool cgi::host_side(const cg_ctx *c, uint64_t p, uint64_t n, uint64_t *found, uint64_t *abase,
                      uint64_t *asize, uint64_t *shadow, uint32_t *flags, uint32_t f_unalloc,
                      uint32_t f_overrun) {
  const AllocTable::Hit h = c->table.find(p);
  if (!h.ok) {
    *found = *abase = *asize = *shadow = 0;
    *flags |= f_unalloc;
    return false;
  }
  *found = h.base + h.size - p;
  *abase = h.base;
  *asize = h.size;
  *shadow = h.shadow + (p - h.base);
  if (n > *found) {
    *flags |= f_overrun;
    return false;
  }
  return true;
}

// --------------------------------------------------------------- C ABI

void cgi::count_stats(cg_ctx *c, const cg_report &r) {
  c->stats.checks++;
  c->stats.bytes_checked += r.expected;
  for (int b = 0; b < CG_NFLAGS; b++)
    if (r.flags & (1u << b)) c->stats.errors[b]++;
}

extern "C" {

cg_status cg_config_default(cg_config *cfg) {
  if (!cfg) return set_error(CG_E_ARG, "cfg is NULL");
  std::memset(cfg, 0, sizeof *cfg);
  cfg->carry = 1;
  return CG_OK;
}

const char *cg_last_error(void) { return g_last_error.c_str(); }

const char *cg_version(void) { return "0.1.0"; }

cg_status cg_create(cg_ctx **out, const cg_config *cfg) {
  if (!out) return set_error(CG_E_ARG, "out is NULL");
  *out = nullptr;
  cg_ctx *c = new (std::nothrow) cg_ctx();
  if (!c) return set_error(CG_E_NOMEM, "context");
  if (cfg)
    c->cfg = *cfg;
  else
    cg_config_default(&c->cfg);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch, sizeof(SingleScratch));
  if (e == cudaSuccess) e = cudaHostAlloc(&c->h_result, sizeof(cg_report), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c->d_result, c->h_result, 0);
  if (e == cudaSuccess) e = launch_init_single_scratch(c->d_scratch, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cg_status st = cuda_fail(e, "cg_create");
    cg_destroy(c);
    return st;
  }
  c->arena.slab_bytes = c->cfg.shadow_slab_bytes ? round_up(c->cfg.shadow_slab_bytes, 1 << 20)
                                                 : (1ull << 30);
  c->arena.budget = c->cfg.shadow_budget_bytes;
  *out = c;
  return CG_OK;
}

cg_status cg_destroy(cg_ctx *c) {
  if (!c) return CG_OK;
  if (c->serve) cg_serve_stop(c, nullptr);
  cudaDeviceSynchronize();
  if (c->d_scratch) cudaFree(c->d_scratch);
  if (c->h_result) cudaFreeHost(c->h_result);
  c->stage.release();
  c->d_fill.release();
  c->h_fill.release();
  c->t_base.release();
  c->t_size.release();
  c->t_shadow.release();
  c->t_base2.release();
  c->t_size2.release();
  c->t_shadow2.release();
  c->t_delta.release();
  c->h_tdelta.release();
  if (c->t_ev) cudaEventDestroy(c->t_ev);
  c->bb[0].release();
  c->bb[1].release();
  c->k_in.release();
  c->h_kin.release();
  c->h_kout.release();
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cap) cudaStreamDestroy(c->cap);
  c->arena.release_all();
  delete c;
  return CG_OK;
}

// The device's view of a pointer: device and managed memory as is, mapped
// pinned host memory through its device pointer; anything else (pageable
// host memory) is refused.
static cg_status device_view(const void *p, const void **out, bool *on_host) {
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(CG_E_ARG, "pointer unknown to CUDA");
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *out = p;
    *on_host = false;
    return CG_OK;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *out = at.devicePointer;
    *on_host = true;
    return CG_OK;
  }
  return set_error(CG_E_ARG, "host memory the device cannot read (pin and map it)");
}

cg_status cg_bind_host_shadow(cg_ctx *c, const uint8_t *a_bits_dev, uint8_t *v_dev,
                              uint64_t n_bytes) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (n_bytes && (!a_bits_dev || !v_dev)) return set_error(CG_E_ARG, "image pointer is NULL");
  if ((reinterpret_cast<uintptr_t>(a_bits_dev) & 15) || (reinterpret_cast<uintptr_t>(v_dev) & 15))
    return set_error(CG_E_ALIGN, "host shadow arrays must be 16-byte aligned");
  if (n_bytes % 128) return set_error(CG_E_ALIGN, "host image size must be a multiple of 128");
  const void *a = a_bits_dev, *v = v_dev;
  bool a_host = false, v_host = false;
  if (n_bytes) {
    CG_TRY(device_view(a_bits_dev, &a, &a_host));
    CG_TRY(device_view(v_dev, &v, &v_host));
    if ((reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(v) & 15))
      return set_error(CG_E_ALIGN, "host shadow arrays must be 16-byte aligned");
  }
  c->img.a_bits = static_cast<const uint8_t *>(a);
  c->img.v = const_cast<uint8_t *>(static_cast<const uint8_t *>(v));
  c->img.n = n_bytes;
  c->img_bound = true;
  c->img_on_host = a_host || v_host;
  return CG_OK;
}

cg_status cg_upload_host_shadow(cg_ctx *c, const uint8_t *a_bits_host, const uint8_t *v_host,
                                uint64_t off, uint64_t n, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !a_bits_host || !v_host) return set_error(CG_E_ARG, "NULL argument");
  if (!c->img_bound) return set_error(CG_E_NO_HOST, "no host shadow image bound");
  if ((off | n) & 7) return set_error(CG_E_ALIGN, "off and n must be multiples of 8");
  if (off > c->img.n || n > c->img.n - off) return set_error(CG_E_HOST_RANGE, "range outside image");
  if (n == 0) return CG_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_CUDA(cudaMemcpyAsync(c->img.v + off, v_host + off, n, cudaMemcpyHostToDevice, st));
  CG_CUDA(cudaMemcpyAsync(const_cast<uint8_t *>(c->img.a_bits) + off / 8, a_bits_host + off / 8,
                          n / 8, cudaMemcpyHostToDevice, st));
  return CG_OK;
}

cg_status cg_register_alloc(cg_ctx *c, uint64_t dptr, uint64_t size) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (size == 0) return set_error(CG_E_ZERO_SIZE, "zero-size allocation");
  if (dptr + size < dptr) return set_error(CG_E_WRAP, "allocation wraps 2^64");
  if (c->table.overlaps(dptr, size))
    return set_error(CG_E_OVERLAP, "allocation overlaps a live allocation");
  if (c->fault_pending & CG_FAULT_SHADOW_ALLOC) {
    c->fault_pending &= ~CG_FAULT_SHADOW_ALLOC;
    return set_error(CG_E_NOMEM, "shadow allocation failed (injected fault)");
  }
  uint64_t sh = 0;
  CG_TRY(c->arena.alloc(size, &sh));
  c->table.insert(dptr, size, sh);
  return CG_OK;
}

cg_status cg_inject_fault(cg_ctx *c, uint32_t fault) {
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (fault & ~(CG_FAULT_STALL_COPY | CG_FAULT_SHADOW_ALLOC))
    return set_error(CG_E_ARG, "unknown fault");
  c->fault_pending |= fault;
  return CG_OK;
}

cg_status cg_register_allocs(cg_ctx *c, const uint64_t *dptr, const uint64_t *size,
                             uint64_t count, cg_status *st_out) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || (count && (!dptr || !size))) return set_error(CG_E_ARG, "NULL argument");
  cg_status first = CG_OK;
  for (uint64_t i = 0; i < count; i++) {
    const cg_status s = cg_register_alloc(c, dptr[i], size[i]);
    if (st_out) st_out[i] = s;
    if (s != CG_OK && first == CG_OK) first = s;
  }
  return first;
}

cg_status cg_free(cg_ctx *c, uint64_t dptr, uint32_t *verdict) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !verdict) return set_error(CG_E_ARG, "NULL argument");
  uint64_t sz = 0, sh = 0;
  if (c->table.remove_base(dptr, &sz, &sh)) {
    c->arena.release(sh, sz);
    c->fill_ptr.push_back(sh);
    c->fill_size.push_back(sz);
    *verdict = CG_FREE_OK;
    return CG_OK;
  }
  if (c->table.find(dptr).ok)
    *verdict = CG_FREE_INTERIOR;
  else if (c->table.freed.count(dptr))
    *verdict = CG_FREE_DOUBLE;
  else
    *verdict = CG_FREE_UNKNOWN;
  return CG_OK;
}

static cg_status mark(cg_ctx *c, uint64_t dptr, uint64_t n, int value, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (n == 0) return CG_OK;
  const AllocTable::Hit h = c->table.find(dptr);
  if (!h.ok || n > h.base + h.size - dptr)
    return set_error(CG_E_RANGE, "range not inside one live allocation");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_TRY(flush_fills(c, st));
  CG_CUDA(cudaMemsetAsync(reinterpret_cast<void *>(h.shadow + (dptr - h.base)), value, n, st));
  return CG_OK;
}

cg_status cg_mark_defined(cg_ctx *c, uint64_t dptr, uint64_t n, void *stream) {
  return mark(c, dptr, n, 0x00, stream);
}

cg_status cg_mark_undefined(cg_ctx *c, uint64_t dptr, uint64_t n, void *stream) {
  return mark(c, dptr, n, 0xFF, stream);
}

cg_status cg_read_device_shadow(cg_ctx *c, uint64_t dptr, uint64_t n, uint8_t *out) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || (n && !out)) return set_error(CG_E_ARG, "NULL argument");
  if (n == 0) return CG_OK;
  const AllocTable::Hit h = c->table.find(dptr);
  if (!h.ok || n > h.base + h.size - dptr)
    return set_error(CG_E_RANGE, "range not inside one live allocation");
  CG_TRY(flush_fills(c, 0));
  CG_CUDA(cudaDeviceSynchronize());
  CG_CUDA(cudaMemcpy(out, reinterpret_cast<const void *>(h.shadow + (dptr - h.base)), n,
                     cudaMemcpyDeviceToHost));
  return CG_OK;
}

static int single_grid(const cg_ctx *c, const ScanJob &job) {
  const uint64_t chunks = (job.n + 30) >> 4;
  const uint64_t groups = (chunks + 32 * 4 - 1) / (32 * 4);  // kU rows of 32 chunks per warp
  const uint64_t ctas_needed = (groups + 7) / 8;             // 8 warps per CTA
  int per_sm = (int)c->cfg.scan_ctas_per_sm;
  if (per_sm <= 0) per_sm = scan_single_max_ctas_per_sm(job.kind, job.mode);
  const uint64_t cap = (uint64_t)c->sm_count * (uint64_t)per_sm;
  const uint64_t g = std::min<uint64_t>(std::max<uint64_t>(ctas_needed, 1), cap);
  return (int)g;
}


// Host part of one check: validation (a1), the device-range lookup on the
// host mirror (a2) and the scan job.  *trivial is set when no byte needs
// reading (n == 0, or a device->device copy whose source has no shadow).
static cg_status prepare_single(cg_ctx *c, const cg_copy &q, RangeInfo *ri, ScanJob *job,
                                bool *overlap_stage, uint64_t *stage_src, bool *trivial) {
  CG_TRY(validate(c, q));
  *ri = RangeInfo{};
  ri->kind = q.kind;
  ri->n = q.n;
  *job = ScanJob{};
  job->kind = q.kind;
  job->n = q.n;
  job->host_off = q.kind == CG_HTOD ? q.src : (q.kind == CG_DTOH ? q.dst : 0);
  *overlap_stage = false;
  *trivial = q.n == 0;  // R9
  if (q.n == 0) return CG_OK;
  bool dst_ok = true, src_ok = true;
  uint64_t dsh = 0, ssh = 0;
  if (q.kind != CG_DTOH)
    dst_ok = host_side(c, q.dst, q.n, &ri->found_dst, &ri->base_dst, &ri->size_dst, &dsh,
                       &ri->flags, CG_F_UNALLOC_DST, CG_F_OVERRUN_DST);
  if (q.kind != CG_HTOD)
    src_ok = host_side(c, q.src, q.n, &ri->found_src, &ri->base_src, &ri->size_src, &ssh,
                       &ri->flags, CG_F_UNALLOC_SRC, CG_F_OVERRUN_SRC);
  bool overlap = false;
  if (q.kind == CG_DTOD) {
    const uint64_t dist = q.src <= q.dst ? q.dst - q.src : q.src - q.dst;
    overlap = dist < q.n;
    if (overlap) ri->flags |= CG_F_DTOD_OVERLAP;
  }
  if (q.kind != CG_HTOD && src_ok) {
    job->mode |= kModeReadDev;
    job->dev_src = ssh;
  }
  if (c->cfg.carry && dst_ok && src_ok) {
    job->mode |= kModeCarry;
    if (q.kind != CG_DTOH) job->dev_dst = dsh;
  }
  if (q.kind == CG_DTOD && !(job->mode & (kModeCarry | kModeReadDev))) *trivial = true;
  if (overlap && (job->mode & kModeCarry)) {  // R12: read the whole source first
    *overlap_stage = true;
    *stage_src = ssh;
  }
  return CG_OK;
}

// Device part: flush queued refills, stage an overlapping source, launch
// the scan; the kernel's last CTA writes the report to `out`.
static cg_status enqueue_single(cg_ctx *c, const RangeInfo &ri, ScanJob job, bool stage,
                                uint64_t stage_src, cg_report *out, cudaStream_t st) {
  NvtxRange range("cg check copy");
  CG_TRY(flush_fills(c, st));
  if (stage) {
    CG_TRY(c->stage.ensure(round_up(job.n, 256)));
    CG_CUDA(cudaMemcpyAsync(c->stage.p, reinterpret_cast<const void *>(stage_src), job.n,
                            cudaMemcpyDeviceToDevice, st));
    job.dev_src = reinterpret_cast<uint64_t>(c->stage.p);
  }
  if (c->cfg.scan_engine == 1 || c->img_on_host) {  // bulk copies read device memory only
    CG_CUDA(launch_scan_single(c->img, job, ri, c->d_scratch, out, single_grid(c, job), st));
  } else {
    if ((c->fault_pending & CG_FAULT_STALL_COPY) && job.n) {
      job.mode |= kModeStall;
      c->fault_pending &= ~CG_FAULT_STALL_COPY;
    }
    CG_CUDA(launch_scan_single_tma(c->img, job, ri, c->d_scratch, out,
                                   scan_single_tma_grid(c->sm_count, job.n), st));
  }
  c->stats.kernels++;
  c->stats.checks++;
  c->stats.bytes_checked += job.n;
  return CG_OK;
}

cg_status cg_check_copy(cg_ctx *c, const cg_copy *req, cg_report *rep, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !req || !rep) return set_error(CG_E_ARG, "NULL argument");
  RangeInfo ri;
  ScanJob job;
  bool stage, trivial;
  uint64_t stage_src = 0;
  CG_TRY(prepare_single(c, *req, &ri, &job, &stage, &stage_src, &trivial));
  if (trivial) {
    const Acc none{0, 0, kNone, kNone};
    assemble_report(rep, ri, none);
    count_stats(c, *rep);
    return CG_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_TRY(enqueue_single(c, ri, job, stage, stage_src, c->d_result, st));
  CG_CUDA(cudaStreamSynchronize(st));
  std::memcpy(rep, c->h_result, sizeof(cg_report));
  if (rep->flags & CG_F_INCOMPLETE)
    return set_error(CG_E_TIMEOUT, "a bounded wait in the scan kernel ran out");
  c->stats.checks--;  // counted again with its flags below
  c->stats.bytes_checked -= job.n;
  count_stats(c, *rep);
  return CG_OK;
}

cg_status cg_check_copy_async(cg_ctx *c, const cg_copy *req, cg_report *rep_dev, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !req || !rep_dev) return set_error(CG_E_ARG, "NULL argument");
  RangeInfo ri;
  ScanJob job;
  bool stage, trivial;
  uint64_t stage_src = 0;
  CG_TRY(prepare_single(c, *req, &ri, &job, &stage, &stage_src, &trivial));
  if (trivial) {  // the kernel with no chunks only writes the report
    job.mode = 0;
    job.kind = CG_DTOD;
  }
  return enqueue_single(c, ri, job, stage, stage_src, rep_dev, static_cast<cudaStream_t>(stream));
}

cg_status cg_plan_units(const cg_copy *reqs, uint64_t nreq, uint32_t carry, const uint8_t *modes,
                        uint64_t host_n, uint64_t piece_rows, uint32_t *req, uint32_t *row_lo,
                        uint32_t *row_hi, int32_t *level, uint64_t cap, uint64_t *n_units) {
  if ((nreq && !reqs) || !n_units || (cap && (!req || !row_lo || !row_hi || !level)))
    return set_error(CG_E_ARG, "NULL argument");
  for (uint64_t i = 0; i < nreq; i++) {
    const cg_copy &q = reqs[i];
    const bool host = q.kind == CG_HTOD || q.kind == CG_DTOH;
    const uint64_t h = q.kind == CG_HTOD ? q.src : q.dst;
    if (host && (h > host_n || q.n > host_n - h))
      return set_error(CG_E_HOST_RANGE, "host range outside the host image");
  }
  const std::vector<PlanUnit> u = plan_pieces(reqs, nreq, carry != 0, modes, host_n, piece_rows);
  *n_units = u.size();
  if (u.size() > cap) return set_error(CG_E_TOO_BIG, "more units than cap");
  for (size_t k = 0; k < u.size(); k++) {
    req[k] = u[k].req;
    row_lo[k] = u[k].rlo;
    row_hi[k] = u[k].rhi;
    level[k] = u[k].level;
  }
  return CG_OK;
}

cg_status cg_plan_levels(const cg_copy *reqs, uint64_t nreq, uint32_t carry, const uint8_t *modes,
                         int32_t *level, uint32_t *n_levels) {
  if ((nreq && (!reqs || !level))) return set_error(CG_E_ARG, "NULL argument");
  const std::vector<int> lvl = plan_levels(reqs, nreq, carry != 0, modes);
  int top = -1;
  for (uint64_t i = 0; i < nreq; i++) {
    level[i] = lvl[i];
    top = std::max(top, lvl[i]);
  }
  if (n_levels) *n_levels = (uint32_t)(top + 1);
  return CG_OK;
}

cg_status cg_get_stats(const cg_ctx *c, cg_stats *out) {
  if (!c || !out) return set_error(CG_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> g(const_cast<cg_ctx *>(c)->stats_mu);
  *out = c->stats;
  out->live_allocs = c->table.live;
  out->shadow_bytes = c->arena.held;
  return CG_OK;
}

cg_status cg_device_table(cg_ctx *c, uint64_t *base, uint64_t *size, uint64_t *shadow,
                          uint64_t cap, uint64_t *count, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !count || (cap && (!base || !size))) return set_error(CG_E_ARG, "NULL argument");
  if (c->bb[0].ticket || c->bb[1].ticket)
    return set_error(CG_E_STATE, "batches still in flight (cg_batch_wait first)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_TRY(ensure_device_table(c, st));
  const uint64_t k = std::min<uint64_t>(cap, c->t_count);
  if (k) {
    CG_CUDA(cudaMemcpyAsync(base, c->t_base.p, k * 8, cudaMemcpyDeviceToHost, st));
    CG_CUDA(cudaMemcpyAsync(size, c->t_size.p, k * 8, cudaMemcpyDeviceToHost, st));
    if (shadow) CG_CUDA(cudaMemcpyAsync(shadow, c->t_shadow.p, k * 8, cudaMemcpyDeviceToHost, st));
  }
  CG_CUDA(cudaStreamSynchronize(st));
  *count = c->t_count;
  return CG_OK;
}

cg_status cg_format_report(const cg_report *r, uint32_t kind, char *buf, size_t cap) {
  if (!r || !buf || cap == 0) return set_error(CG_E_ARG, "NULL argument");
  const char *dir = kind == CG_HTOD ? "host->device" : kind == CG_DTOH ? "device->host"
                                                                       : "device->device";
  std::string s;
  char line[320];
  if (r->flags == 0) {
    std::snprintf(line, sizeof line, "%s copy of %llu bytes: no findings", dir,
                  (unsigned long long)r->expected);
    s += line;
  }
  auto add = [&](const char *t) {
    if (!s.empty()) s += "\n";
    s += t;
  };
  if (r->flags & CG_F_UNALLOC_DST) {
    std::snprintf(line, sizeof line, "%s copy of %llu bytes: destination pointer lies in no live allocation",
                  dir, (unsigned long long)r->expected);
    add(line);
  }
  if (r->flags & CG_F_UNALLOC_SRC) {
    std::snprintf(line, sizeof line, "%s copy of %llu bytes: source pointer lies in no live allocation",
                  dir, (unsigned long long)r->expected);
    add(line);
  }
  if (r->flags & CG_F_OVERRUN_DST) {
    std::snprintf(line, sizeof line,
                  "%s copy of %llu bytes overruns its destination allocation: only %llu bytes "
                  "from the pointer to its end",
                  dir, (unsigned long long)r->expected, (unsigned long long)r->found_dst);
    add(line);
  }
  if (r->flags & CG_F_OVERRUN_SRC) {
    std::snprintf(line, sizeof line,
                  "%s copy of %llu bytes overruns its source allocation: only %llu bytes from "
                  "the pointer to its end",
                  dir, (unsigned long long)r->expected, (unsigned long long)r->found_src);
    add(line);
  }
  if (r->flags & CG_F_HOST_UNADDR) {
    std::snprintf(line, sizeof line, "%s copy: %llu host bytes not addressable, first at offset %lld",
                  dir, (unsigned long long)r->n_unaddr, (long long)r->first_unaddr_off);
    add(line);
  }
  if (r->flags & CG_F_HOST_UNDEF) {
    std::snprintf(line, sizeof line,
                  "%s copy: %llu host bytes (partly) undefined, first at offset %lld", dir,
                  (unsigned long long)r->n_undef, (long long)r->first_undef_off);
    add(line);
  }
  if (r->flags & CG_F_DEV_UNDEF_SRC) {
    std::snprintf(line, sizeof line,
                  "%s copy (warning): %llu device source bytes (partly) undefined, first at "
                  "offset %lld",
                  dir, (unsigned long long)r->n_undef, (long long)r->first_undef_off);
    add(line);
  }
  if (r->flags & CG_F_DTOD_OVERLAP) add("device->device copy (warning): source and destination overlap");
  std::snprintf(buf, cap, "%s", s.c_str());
  return CG_OK;
}

}  // extern "C"

// cg_ctx.h -- the context of libcg and the host-side structures behind it
// (allocation table, device shadow pool, dependency planner), shared by the
// C ABI (cg_host.cpp) and the serving engine (cg_serve.cpp).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "cg_internal.h"
#include "cg_launch.h"

namespace cgi {

// ------------------------------------------------------------- errors

cg_status set_error(cg_status st, const std::string &msg);
cg_status cuda_fail(cudaError_t e, const char *what);

#define CG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cgi::cuda_fail(e_, #call); \
  } while (0)

#define CG_TRY(call)            \
  do {                          \
    cg_status s_ = (call);      \
    if (s_ != CG_OK) return s_; \
  } while (0)

inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

inline uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// -------------------------------------------------- device shadow pool

// Device V shadow of every live allocation (R6: all 0xFF on registration).
// Slabs of device memory are carved best-fit in 256-byte units; free space
// is kept at 0xFF, so a new allocation's shadow needs no initialisation.
// Released ranges are refilled with 0xFF (queued, flushed on the next
// stream operation of the context).
class ShadowArena {
 public:
  uint64_t slab_bytes = 1ull << 30;
  uint64_t budget = 0;
  uint64_t held = 0;

  ~ShadowArena() { release_all(); }

  void release_all() {
    for (auto &s : slabs_)
      if (s.base) cudaFree(s.base);
    slabs_.clear();
    by_size_.clear();
    free_by_off_.clear();
    slab_index_.clear();
    held = 0;
  }

  cg_status alloc(uint64_t size, uint64_t *out) {
    const uint64_t sz = round_up(size, 256);
    if (sz > slab_bytes / 2) {  // its own slab
      if (budget && held + sz > budget) return set_error(CG_E_NOMEM, "shadow budget exceeded");
      uint8_t *p = nullptr;
      cudaError_t e = cudaMalloc(&p, sz);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CG_E_NOMEM, std::string("shadow slab: ") + cudaGetErrorString(e));
      }
      e = cudaMemset(p, 0xFF, sz);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(shadow)");
      add_slab(p, sz, true);
      held += sz;
      *out = reinterpret_cast<uint64_t>(p);
      return CG_OK;
    }
    auto it = by_size_.lower_bound(sz);
    if (it == by_size_.end()) {
      if (budget && held + slab_bytes > budget) return set_error(CG_E_NOMEM, "shadow budget exceeded");
      uint8_t *p = nullptr;
      cudaError_t e = cudaMalloc(&p, slab_bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(CG_E_NOMEM, std::string("shadow slab: ") + cudaGetErrorString(e));
      }
      e = cudaMemset(p, 0xFF, slab_bytes);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(shadow)");
      const uint32_t si = add_slab(p, slab_bytes, false);
      held += slab_bytes;
      insert_free(si, 0, slab_bytes);
      it = by_size_.lower_bound(sz);
    }
    const uint64_t bsize = it->first;
    const uint32_t si = it->second.first;
    const uint64_t off = it->second.second;
    by_size_.erase(it);
    free_by_off_[si].erase(off);
    if (bsize > sz) insert_free(si, off + sz, bsize - sz);
    *out = reinterpret_cast<uint64_t>(slabs_[si].base) + off;
    return CG_OK;
  }

  // The caller queues the 0xFF refill of [ptr, ptr+size) before reuse.
  void release(uint64_t ptr, uint64_t size) {
    const uint64_t sz = round_up(size, 256);
    auto it = slab_index_.upper_bound(ptr);
    --it;
    const uint32_t si = it->second;
    Slab &s = slabs_[si];
    if (s.dedicated) {
      cudaFree(s.base);  // synchronises the device; dedicated slabs are rare
      held -= s.size;
      slab_index_.erase(it);
      s.base = nullptr;
      s.size = 0;
      return;
    }
    uint64_t off = ptr - reinterpret_cast<uint64_t>(s.base);
    uint64_t len = sz;
    auto &fm = free_by_off_[si];
    auto nx = fm.lower_bound(off);
    if (nx != fm.end() && nx->first == off + len) {  // merge with the next block
      len += nx->second;
      erase_free(si, nx->first, nx->second);
      nx = fm.lower_bound(off);
    }
    if (nx != fm.begin()) {  // merge with the previous block
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        off = pv->first;
        len += pv->second;
        erase_free(si, pv->first, pv->second);
      }
    }
    insert_free(si, off, len);
  }

 private:
  struct Slab {
    uint8_t *base;
    uint64_t size;
    bool dedicated;
  };
  std::vector<Slab> slabs_;
  std::multimap<uint64_t, std::pair<uint32_t, uint64_t>> by_size_;  // size -> (slab, off)
  std::vector<std::map<uint64_t, uint64_t>> free_by_off_;           // per slab: off -> size
  std::map<uint64_t, uint32_t> slab_index_;                         // base -> slab

  uint32_t add_slab(uint8_t *p, uint64_t size, bool dedicated) {
    slabs_.push_back({p, size, dedicated});
    free_by_off_.emplace_back();
    const uint32_t si = (uint32_t)(slabs_.size() - 1);
    slab_index_[reinterpret_cast<uint64_t>(p)] = si;
    return si;
  }
  void insert_free(uint32_t si, uint64_t off, uint64_t len) {
    free_by_off_[si][off] = len;
    by_size_.insert({len, {si, off}});
  }
  void erase_free(uint32_t si, uint64_t off, uint64_t len) {
    free_by_off_[si].erase(off);
    auto r = by_size_.equal_range(len);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second.first == si && it->second.second == off) {
        by_size_.erase(it);
        break;
      }
  }
};

// A named NVTX range for profilers (ncu --nvtx, nsys) around a host phase;
// a few instructions when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------- allocation table

// The list of live device allocations (Fig. 2 caption) as a sorted main
// array (size 0 = tombstone of a freed entry) plus an ordered delta of
// recent registrations, merged into the main array in bulk.
class AllocTable {
 public:
  std::vector<uint64_t> base, size, shadow;  // main, sorted by base
  std::map<uint64_t, std::pair<uint64_t, uint64_t>> delta;  // base -> (size, shadow)
  std::set<uint64_t> freed;
  uint64_t dead = 0;
  uint64_t live = 0;
  uint64_t version = 0;
  // Changes since the device copy was last brought up to date, while it is
  // tracked (dev_track): registrations it lacks, and bases it still holds
  // that were freed.  Kept by base, so the host's own merges do not matter.
  bool dev_track = false;
  std::map<uint64_t, std::pair<uint64_t, uint64_t>> dev_added;
  std::vector<uint64_t> dev_removed;

  void dev_synced() {
    dev_track = true;
    dev_added.clear();
    dev_removed.clear();
  }
  void dev_stale() {
    dev_track = false;
    dev_added.clear();
    dev_removed.clear();
  }
  uint64_t dev_limit() const { return std::max<uint64_t>(65536, live / 4); }

  struct Hit {
    bool ok;
    uint64_t base, size, shadow;
  };

  Hit find(uint64_t addr) const {
    auto ub = std::upper_bound(base.begin(), base.end(), addr);
    if (ub != base.begin()) {
      const size_t j = (size_t)(ub - base.begin()) - 1;
      if (size[j] && addr - base[j] < size[j]) return {true, base[j], size[j], shadow[j]};
    }
    auto it = delta.upper_bound(addr);
    if (it != delta.begin()) {
      --it;
      if (addr - it->first < it->second.first)
        return {true, it->first, it->second.first, it->second.second};
    }
    return {false, 0, 0, 0};
  }

  bool overlaps(uint64_t b, uint64_t s) const {  // [b, b+s), no wrap
    auto ub = std::upper_bound(base.begin(), base.end(), b);
    if (ub != base.begin()) {
      const size_t j = (size_t)(ub - base.begin()) - 1;
      if (size[j] && b - base[j] < size[j]) return true;
    }
    for (auto k = ub; k != base.end() && *k < b + s; ++k)
      if (size[(size_t)(k - base.begin())]) return true;
    auto it = delta.upper_bound(b);
    if (it != delta.end() && it->first < b + s) return true;
    if (it != delta.begin()) {
      --it;
      if (b - it->first < it->second.first) return true;
    }
    return false;
  }

  void insert(uint64_t b, uint64_t s, uint64_t sh) {
    delta[b] = {s, sh};
    live++;
    version++;
    if (dev_track) {
      dev_added[b] = {s, sh};
      if (dev_added.size() > dev_limit()) dev_stale();
    }
    freed.erase(freed.lower_bound(b), freed.lower_bound(b + s));  // R13
    if (delta.size() > std::max<uint64_t>(4096, base.size() / 8)) merge();
  }

  // Remove the live allocation whose base is exactly b.
  bool remove_base(uint64_t b, uint64_t *sz, uint64_t *sh) {
    auto lb = std::lower_bound(base.begin(), base.end(), b);
    if (lb != base.end() && *lb == b) {
      const size_t j = (size_t)(lb - base.begin());
      if (size[j]) {
        *sz = size[j];
        *sh = shadow[j];
        size[j] = 0;
        dead++;
        goto removed;
      }
    }
    {
      auto it = delta.find(b);
      if (it == delta.end()) return false;
      *sz = it->second.first;
      *sh = it->second.second;
      delta.erase(it);
    }
  removed:
    live--;
    version++;
    if (dev_track && dev_added.erase(b) == 0) {
      dev_removed.push_back(b);
      if (dev_removed.size() > dev_limit()) dev_stale();
    }
    freed.insert(b);
    if (dead > 1024 && dead > base.size() / 4) merge();
    return true;
  }

  void merge() {
    if (delta.empty() && dead == 0) return;
    std::vector<uint64_t> nb, ns, nh;
    nb.reserve(live);
    ns.reserve(live);
    nh.reserve(live);
    auto it = delta.begin();
    for (size_t j = 0; j <= base.size(); j++) {
      const uint64_t limit = j < base.size() ? base[j] : ~0ull;
      while (it != delta.end() && (j == base.size() || it->first < limit)) {
        nb.push_back(it->first);
        ns.push_back(it->second.first);
        nh.push_back(it->second.second);
        ++it;
      }
      if (j < base.size() && size[j]) {
        nb.push_back(base[j]);
        ns.push_back(size[j]);
        nh.push_back(shadow[j]);
      }
    }
    base.swap(nb);
    size.swap(ns);
    shadow.swap(nh);
    delta.clear();
    dead = 0;
  }
};

// ---------------------------------------------------- batch planner

// Range-chmax / range-max segment tree over the elementary intervals of one
// address space, holding two values per leaf: the highest level of a copy
// that wrote it (w) and of one that read it (r).  Values only grow, so a
// chmax never has to be pushed down: each node keeps the max of its
// subtree (sub) and the chmax applied to its whole subtree (tag); a range
// max is the max of `sub` over the covering nodes and of `tag` over the
// ancestors of the range's two end leaves.  Iterative, bottom-up.
class LevelTree {
 public:
  void init(int n) {
    size_t m = 1;
    while (m < (size_t)std::max(1, n)) m <<= 1;
    m_ = m;
    nodes_.assign(2 * m, Node{-1, -1, -1, -1});
  }
  // max of w (and of r when want_r) over leaves [l, r)
  int query(int l, int r, bool want_r) const {
    if (l >= r) return -1;
    int v = -1;
    size_t a = l + m_, b = r + m_;
    const size_t a0 = a, b0 = b - 1;
    while (a < b) {
      if (a & 1) v = std::max(v, sub(nodes_[a++], want_r));
      if (b & 1) v = std::max(v, sub(nodes_[--b], want_r));
      a >>= 1;
      b >>= 1;
    }
    // tags of the end leaves' ancestors; the two paths join below the root
    size_t i = a0 >> 1, j = b0 >> 1;
    for (; i != j; i >>= 1, j >>= 1) {
      v = std::max(v, tag(nodes_[i], want_r));
      v = std::max(v, tag(nodes_[j], want_r));
    }
    for (; i; i >>= 1) v = std::max(v, tag(nodes_[i], want_r));
    return v;
  }
  void update_w(int l, int r, int v) { update(l, r, v, true); }
  void update_r(int l, int r, int v) { update(l, r, v, false); }

 private:
  struct Node {
    int sw, sr, tw, tr;  // subtree maxima, whole-subtree chmax tags
  };
  size_t m_ = 1;
  std::vector<Node> nodes_;
  static int sub(const Node &n, bool want_r) { return want_r ? std::max(n.sw, n.sr) : n.sw; }
  static int tag(const Node &n, bool want_r) { return want_r ? std::max(n.tw, n.tr) : n.tw; }
  void update(int l, int r, int v, bool is_w) {
    if (l >= r) return;
    size_t a = l + m_, b = r + m_;
    const size_t a0 = a, b0 = b - 1;
    auto apply = [&](Node &n) {
      if (is_w) {
        n.sw = std::max(n.sw, v);
        n.tw = std::max(n.tw, v);
      } else {
        n.sr = std::max(n.sr, v);
        n.tr = std::max(n.tr, v);
      }
    };
    while (a < b) {
      if (a & 1) apply(nodes_[a++]);
      if (b & 1) apply(nodes_[--b]);
      a >>= 1;
      b >>= 1;
    }
    // ancestors of the end leaves, level by level (children before their
    // parent; the two paths join below the root): subtree max = max(own
    // tag, children's)
    auto rebuild = [&](size_t i) {
      Node &n = nodes_[i];
      const Node &c0 = nodes_[2 * i], &c1 = nodes_[2 * i + 1];
      if (is_w)
        n.sw = std::max(n.tw, std::max(c0.sw, c1.sw));
      else
        n.sr = std::max(n.tr, std::max(c0.sr, c1.sr));
    };
    size_t i = a0 >> 1, j = b0 >> 1;
    for (; i != j; i >>= 1, j >>= 1) {
      rebuild(i);
      rebuild(j);
    }
    for (; i; i >>= 1) rebuild(i);
  }
};

std::vector<int> plan_levels(const cg_copy *reqs, uint64_t nreq, bool carry,
                             const uint8_t *modes = nullptr);

// A batch cut into planning units: whole copies, and pieces of the copies
// that only read host bytes (host->device copies that carry nothing).
struct PlanUnit {
  uint32_t req;
  uint32_t rlo, rhi;  // rows [rlo, rhi) of the copy's anchor grid; rhi = 0: the whole copy
  int level;
};
// The units of a batch with their dependency levels (sequential semantics,
// as plan_levels; see cg_host.cpp).  piece_rows: rows per piece (a
// multiple of the tile's rows), 0 = whole copies only.
std::vector<PlanUnit> plan_pieces(const cg_copy *reqs, uint64_t nreq, bool carry,
                                  const uint8_t *modes, uint64_t host_n, uint64_t piece_rows);

// --------------------------------------------------------------- context

template <typename T>
struct DevBuf {
  T *p = nullptr;
  uint64_t cap = 0;
  cg_status ensure(uint64_t n) {
    if (n <= cap) return CG_OK;
    uint64_t c = std::max<uint64_t>(n, cap * 2);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max<uint64_t>(1, c) * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(CG_E_NOMEM, std::string("device buffer: ") + cudaGetErrorString(e));
    }
    cap = c;
    return CG_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

template <typename T>
struct PinBuf {
  T *p = nullptr;
  uint64_t cap = 0;
  cg_status ensure(uint64_t n) {
    if (n <= cap) return CG_OK;
    uint64_t c = std::max<uint64_t>(n, cap * 2);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMallocHost(&p, std::max<uint64_t>(1, c) * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(CG_E_NOMEM, std::string("pinned buffer: ") + cudaGetErrorString(e));
    }
    cap = c;
    return CG_OK;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
  }
};

// Per-batch buffers (device, and pinned host staging), one set per slot.
struct BatchBufs {
  DevBuf<cg_copy> b_reqs;
  DevBuf<uint32_t> b_order;
  DevBuf<uint64_t> b_segfirst, b_stage, b_piece;
  DevBuf<ScanJob> b_jobs;
  DevBuf<RangeInfo> b_info;
  DevBuf<Acc> b_acc;
  DevBuf<cg_report> b_reps;
  DevBuf<uint32_t> b_counts;
  DevBuf<uint64_t> b_blocksums;
  DevBuf<cg_err_record> b_recs;
  DevBuf<unsigned int> b_err;
  DevBuf<unsigned long long> b_claim;  // per-level segment-claim counters
  DevBuf<uint8_t> b_modes;
  DevBuf<uint8_t> stage;  // overlapping device->device sources
  PinBuf<uint8_t> h_modes;
  PinBuf<uint8_t> h_stage_in;  // pinned upload staging (requests, stage pointers)
  PinBuf<uint8_t> h_pos;       // per order position: request, first segment, piece
  PinBuf<cg_report> h_reps;
  PinBuf<cg_err_record> h_recs;
  PinBuf<uint64_t> h_total;
  // a batch in flight in this slot (asynchronous submission)
  uint64_t ticket = 0;        // 0: free
  cudaEvent_t done = nullptr;  // recorded after its results' copies
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // around its level kernels
  cudaGraphExec_t exec = nullptr;           // the batch's kernels as a CUDA graph
  uint64_t nreq = 0, nblocks = 0, dev_rec_cap = 0, t_begin = 0;
  int nlev = 0;
  uint32_t source = 0, kib = 0;
  std::vector<float> feat;    // features, kept for an online trial's record
  void release() {
    b_reqs.release();
    b_order.release();
    b_segfirst.release();
    b_piece.release();
    b_stage.release();
    b_jobs.release();
    b_info.release();
    b_acc.release();
    b_reps.release();
    b_counts.release();
    b_blocksums.release();
    b_recs.release();
    b_err.release();
    b_claim.release();
    b_modes.release();
    stage.release();
    h_modes.release();
    h_stage_in.release();
    h_pos.release();
    h_reps.release();
    h_recs.release();
    h_total.release();
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    if (done) cudaEventDestroy(done);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    done = t0 = t1 = nullptr;
    ticket = 0;
  }
};

struct ServeEngine;

}  // namespace cgi

struct cg_ctx {
  cg_config cfg{};
  int device = 0;
  int sm_count = 1;
  cgi::Image img{nullptr, nullptr, 0};
  bool img_bound = false;
  bool img_on_host = false;  // image in mapped pinned host memory: register engine
  cgi::ShadowArena arena;
  cgi::AllocTable table;
  cgi::SingleScratch *d_scratch = nullptr;
  cg_report *h_result = nullptr;  // mapped pinned
  cg_report *d_result = nullptr;
  cgi::DevBuf<uint8_t> stage;
  std::vector<uint64_t> fill_ptr, fill_size;
  cgi::DevBuf<uint64_t> d_fill;
  cgi::PinBuf<uint64_t> h_fill;
  cgi::DevBuf<uint64_t> t_base, t_size, t_shadow;
  uint64_t t_count = 0;
  // incremental updates: the merge kernel writes the other buffer set from
  // the uploaded registrations and freed bases (t_delta, staged in h_tdelta)
  cgi::DevBuf<uint64_t> t_base2, t_size2, t_shadow2, t_delta;
  cgi::PinBuf<uint64_t> h_tdelta;
  cudaEvent_t t_ev = nullptr;  // the last table update's copies and merge
  // batch buffers: two slots, so that a batch can be planned while the one
  // before it still runs (slot 0 also serves the synchronous paths)
  cgi::BatchBufs bb[2];
  cudaStream_t side = nullptr;  // lookups of batches submitted asynchronously
  cudaStream_t cap = nullptr;   // where a batch's kernels are captured into a graph
  uint64_t next_ticket = 1;
  // batch split choice: tuned entries (features -> segment KiB) and the
  // learned cost model's weights (empty = none)
  std::vector<std::vector<float>> tuned_feat;
  std::vector<uint32_t> tuned_kib;
  std::vector<float> cost_model;
  uint32_t cost_hidden = 0;
  struct OnlineTune {
    std::vector<float> feat;
    uint32_t next = 0;  // index of the next candidate to try
    uint32_t best_kib = 0;
    float best_ms = 0.f;
  };
  std::vector<OnlineTune> online;
  // kernel-argument checks: one upload (jobs | range verdicts |
  // accumulators | order | scan segments | fill spans | claim counter |
  // error flag) and the pinned buffer the finalize kernel writes (error
  // flag | reports)
  cgi::DevBuf<uint8_t> k_in;
  cgi::PinBuf<uint8_t> h_kin, h_kout;
  // device arrays (Fig. 2's second list): handle -> dimensions and shadow
  struct ArrayInfo {
    uint64_t w, h, d;
    uint64_t shadow;  // dense, row-major
  };
  std::unordered_map<uint64_t, ArrayInfo> arrays;
  std::unordered_set<uint64_t> freed_arrays;
  uint32_t fault_pending = 0;  // CG_FAULT_* bits injected for the next operation
  cg_stats stats{};
  std::mutex stats_mu;                // guards stats while serving
  cgi::ServeEngine *serve = nullptr;  // non-null while serving
};

namespace cgi {

cg_status flush_fills(cg_ctx *c, cudaStream_t st);
cg_status ensure_device_table(cg_ctx *c, cudaStream_t st);
cg_status validate(const cg_ctx *c, const cg_copy &q);
bool host_side(const cg_ctx *c, uint64_t p, uint64_t n, uint64_t *found, uint64_t *abase,
               uint64_t *asize, uint64_t *shadow, uint32_t *flags, uint32_t f_unalloc,
               uint32_t f_overrun);
void count_stats(cg_ctx *c, const cg_report &r);

}  // namespace cgi

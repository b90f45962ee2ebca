// cg_race_index.h -- the serving engine's index of its race window (host
// only; no CUDA).
#pragma once
#include <stdint.h>

#include <cstddef>
#include <vector>

namespace cgi {

// The items listed under one block, in the order they were added.  Up to
// kInline items stay in place (a removal shifts the few behind it); a list
// that outgrows them moves to a heap vector with a moving head (a removal
// at the front only moves the head; the vector is compacted once most of
// it is dead).  Most blocks hold one or two items, so a lookup usually
// touches one cache line and no heap memory.
struct BlockList {
  static constexpr uint32_t kInline = 4;
  uint64_t key;
  uint32_t n;     // items in place (while big is null)
  uint32_t head;  // first live item of *big
  uint64_t in[kInline];
  std::vector<uint64_t> *big;

  template <typename F>
  void each(F &&f) const {
    if (big) {
      for (size_t i = head; i < big->size(); i++) f((*big)[i]);
    } else {
      for (uint32_t i = 0; i < n; i++) f(in[i]);
    }
  }
  void push(uint64_t item) {
    if (!big) {
      if (n < kInline) {
        in[n++] = item;
        return;
      }
      big = new std::vector<uint64_t>(in, in + n);
      head = 0;
      n = 0;
    }
    big->push_back(item);
  }
  // drop one occurrence of item; true when no item is left
  bool remove(uint64_t item) {
    if (!big) {
      for (uint32_t i = 0; i < n; i++)
        if (in[i] == item) {
          for (uint32_t j = i + 1; j < n; j++) in[j - 1] = in[j];
          n--;
          break;
        }
      return n == 0;
    }
    std::vector<uint64_t> &v = *big;
    for (size_t i = head; i < v.size(); i++)
      if (v[i] == item) {
        if (i == head)
          head++;
        else
          v.erase(v.begin() + (ptrdiff_t)i);
        break;
      }
    if (head == v.size()) return true;
    if (head >= 32 && 2 * (size_t)head >= v.size()) {
      v.erase(v.begin(), v.begin() + (ptrdiff_t)head);
      head = 0;
    }
    return false;
  }
  void release() {
    delete big;
    big = nullptr;
    n = 0;
    head = 0;
  }
};

// Block key -> BlockList, open addressing with linear probing in a
// power-of-two table kept at most half full; a deleted slot is refilled by
// shifting back the entries of its probe run (no tombstones), so lookups
// stay short however many entries came and went.
class ListMap {
 public:
  static constexpr uint64_t kFree = ~0ull;  // never a key: space < 2, block < 2^58

  ListMap() { resize(1u << 10); }
  ~ListMap() {
    for (auto &s : t_)
      if (s.key != kFree) s.release();
  }
  ListMap(const ListMap &) = delete;
  ListMap &operator=(const ListMap &) = delete;

  const BlockList *find(uint64_t k) const {
    for (size_t i = home(k);; i = (i + 1) & mask_) {
      if (t_[i].key == k) return &t_[i];
      if (t_[i].key == kFree) return nullptr;
    }
  }
  // the list of k, created empty if absent (a reference valid until the
  // next get or erase)
  BlockList &get(uint64_t k) {
    if (2 * (used_ + 1) > t_.size()) resize(2 * t_.size());
    size_t i = home(k);
    for (; t_[i].key != kFree; i = (i + 1) & mask_)
      if (t_[i].key == k) return t_[i];
    BlockList &s = t_[i];
    s.key = k;
    s.n = 0;
    s.head = 0;
    s.big = nullptr;
    used_++;
    return s;
  }
  // drop one occurrence of item from k's list; the list goes when empty
  void remove(uint64_t k, uint64_t item) {
    size_t i = home(k);
    for (;; i = (i + 1) & mask_) {
      if (t_[i].key == kFree) return;
      if (t_[i].key == k) break;
    }
    if (!t_[i].remove(item)) return;
    t_[i].release();
    // backward shift: an entry further along the run moves into the hole
    // unless its home lies cyclically in (hole, its slot]
    size_t hole = i;
    for (size_t j = (i + 1) & mask_; t_[j].key != kFree; j = (j + 1) & mask_) {
      const size_t h = home(t_[j].key);
      const bool stays = hole <= j ? (hole < h && h <= j) : (hole < h || h <= j);
      if (stays) continue;
      t_[hole] = t_[j];
      hole = j;
    }
    t_[hole].key = kFree;
    t_[hole].big = nullptr;
    used_--;
  }
  size_t size() const { return used_; }

 private:
  size_t home(uint64_t k) const {
    return (size_t)((k * 0x9E3779B97F4A7C15ull) >> (64 - bits_)) & mask_;
  }
  void resize(size_t cap) {
    std::vector<BlockList> old;
    old.swap(t_);
    t_.resize(cap);
    for (auto &s : t_) {
      s.key = kFree;
      s.big = nullptr;
    }
    mask_ = cap - 1;
    bits_ = 0;
    while (((size_t)1 << bits_) < cap) bits_++;
    for (const auto &s : old) {
      if (s.key == kFree) continue;
      size_t i = home(s.key);
      while (t_[i].key != kFree) i = (i + 1) & mask_;
      t_[i] = s;
    }
  }
  std::vector<BlockList> t_;
  size_t used_ = 0;
  size_t mask_ = 0;
  unsigned bits_ = 0;
};

// The race window's entries indexed by the blocks of the spaces their ranges
// touch (space 0: host image offsets, 1: device addresses), so that a new
// copy meets only the entries near its own ranges instead of scanning the
// whole window (which, with a backlog, holds every copy finished since the
// oldest waiting request was submitted).  A short range (at most kSmallMax
// blocks of 64 KiB) is listed under those blocks and under the 64 MiB
// blocks it touches (a list of its own); a long range only under its 64 MiB
// blocks.  Two ranges that meet share a block of the shorter one's kind,
// so a short range looks up its small blocks and the long entries of its
// large blocks, and a long range every entry of its large blocks: the
// common short lookups never walk the short entries of a whole 64 MiB
// block.  An entry is an opaque 64-bit item (the serving engine passes the
// address of its window entry); each list holds items in the order they
// were added, and entries leave about in that order, so a removal finds
// its item near the front.  Candidates are then checked exactly.
struct RaceIndex {
  static constexpr int kSmallShift = 16, kLargeShift = 26;
  static constexpr uint64_t kSmallMax = 64;
  ListMap small, large_short, large_long;
  static uint64_t key(int space, uint64_t block) { return ((uint64_t)space << 62) | block; }
  static bool is_long(uint64_t a, uint64_t n) {
    return ((a + n - 1) >> kSmallShift) - (a >> kSmallShift) + 1 > kSmallMax;
  }
  void add(int space, uint64_t a, uint64_t n, uint64_t item) {
    if (!n) return;
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++)
        small.get(key(space, b)).push(item);
    ListMap &big = lg ? large_long : large_short;
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++)
      big.get(key(space, b)).push(item);
  }
  void remove(int space, uint64_t a, uint64_t n, uint64_t item) {
    if (!n) return;
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++)
        small.remove(key(space, b), item);
    ListMap &big = lg ? large_long : large_short;
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++)
      big.remove(key(space, b), item);
  }
  // candidates() and then add() in one pass over the keys (so each list is
  // looked up once); f may also see `item` itself when both of a copy's
  // ranges lie in one space
  template <typename F>
  void visit_add(int space, uint64_t a, uint64_t n, uint64_t item, F &&f) {
    if (!n) return;
    auto walk_if = [&](const ListMap &m, uint64_t k) {
      if (const BlockList *l = m.find(k)) l->each(f);
    };
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++) {
        BlockList &l = small.get(key(space, b));
        l.each(f);
        l.push(item);
      }
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++) {
      const uint64_t k = key(space, b);
      if (lg) {
        BlockList &l = large_long.get(k);
        l.each(f);
        walk_if(large_short, k);
        l.push(item);
      } else {
        walk_if(large_long, k);
        large_short.get(k).push(item);
      }
    }
  }
  // f(item) for every entry that may touch [a, a+n) of `space` (some twice)
  template <typename F>
  void candidates(int space, uint64_t a, uint64_t n, F &&f) const {
    if (!n) return;
    auto walk_if = [&](const ListMap &m, uint64_t k) {
      if (const BlockList *l = m.find(k)) l->each(f);
    };
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++)
        walk_if(small, key(space, b));
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++) {
      walk_if(large_long, key(space, b));
      if (lg) walk_if(large_short, key(space, b));
    }
  }
};

}  // namespace cgi

// cg_race_index.h -- the serving engine's index of its race window (host
// only; no CUDA).
#pragma once
#include <stdint.h>

#include <cstddef>
#include <unordered_map>
#include <vector>

namespace cgi {

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
  // items in the order they were added; those before `head` are removed
  // (a removal at the front only moves head; the vector is compacted once
  // most of it is dead)
  struct List {
    std::vector<uint64_t> v;
    size_t head = 0;
  };
  using Map = std::unordered_map<uint64_t, List>;
  Map small, large_short, large_long;
  static uint64_t key(int space, uint64_t block) { return ((uint64_t)space << 62) | block; }
  static bool is_long(uint64_t a, uint64_t n) {
    return ((a + n - 1) >> kSmallShift) - (a >> kSmallShift) + 1 > kSmallMax;
  }
  void add(int space, uint64_t a, uint64_t n, uint64_t item) {
    if (!n) return;
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++)
        small[key(space, b)].v.push_back(item);
    Map &big = lg ? large_long : large_short;
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++)
      big[key(space, b)].v.push_back(item);
  }
  static void erase_from(Map &m, uint64_t k, uint64_t item) {
    auto it = m.find(k);
    if (it == m.end()) return;
    List &l = it->second;
    for (size_t i = l.head; i < l.v.size(); i++)
      if (l.v[i] == item) {
        if (i == l.head)
          l.head++;
        else
          l.v.erase(l.v.begin() + (ptrdiff_t)i);
        break;
      }
    if (l.head == l.v.size()) {
      m.erase(it);
    } else if (l.head >= 32 && 2 * l.head >= l.v.size()) {
      l.v.erase(l.v.begin(), l.v.begin() + (ptrdiff_t)l.head);
      l.head = 0;
    }
  }
  void remove(int space, uint64_t a, uint64_t n, uint64_t item) {
    if (!n) return;
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++)
        erase_from(small, key(space, b), item);
    Map &big = lg ? large_long : large_short;
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++)
      erase_from(big, key(space, b), item);
  }
  // candidates() and then add() in one pass over the keys (so each list is
  // looked up once); f may also see `item` itself when both of a copy's
  // ranges lie in one space
  template <typename F>
  void visit_add(int space, uint64_t a, uint64_t n, uint64_t item, F &&f) {
    if (!n) return;
    auto walk = [&](const List &l) {
      for (size_t i = l.head; i < l.v.size(); i++) f(l.v[i]);
    };
    auto walk_if = [&](const Map &m, uint64_t k) {
      auto it = m.find(k);
      if (it != m.end()) walk(it->second);
    };
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++) {
        List &l = small[key(space, b)];
        walk(l);
        l.v.push_back(item);
      }
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++) {
      const uint64_t k = key(space, b);
      if (lg) {
        List &l = large_long[k];
        walk(l);
        walk_if(large_short, k);
        l.v.push_back(item);
      } else {
        walk_if(large_long, k);
        large_short[k].v.push_back(item);
      }
    }
  }
  // f(item) for every entry that may touch [a, a+n) of `space` (some twice)
  template <typename F>
  void candidates(int space, uint64_t a, uint64_t n, F &&f) const {
    if (!n) return;
    auto walk = [&](const Map &m, uint64_t k) {
      auto it = m.find(k);
      if (it != m.end())
        for (size_t i = it->second.head; i < it->second.v.size(); i++) f(it->second.v[i]);
    };
    const bool lg = is_long(a, n);
    if (!lg)
      for (uint64_t b = a >> kSmallShift; b <= (a + n - 1) >> kSmallShift; b++)
        walk(small, key(space, b));
    for (uint64_t b = a >> kLargeShift; b <= (a + n - 1) >> kLargeShift; b++) {
      walk(large_long, key(space, b));
      if (lg) walk(large_short, key(space, b));
    }
  }
};

}  // namespace cgi

"""The serving engine's race-window index (cg_race_index.h) against brute
force: over random sequences of adds (plain, or fused with a lookup),
removals and lookups of short and long ranges in two address spaces, every
live entry whose range meets a lookup's range is among the lookup's
candidates, and no removed entry is.
The index only narrows the exact check, so this is what its correctness
rests on.  Built with g++ and AddressSanitizer where available; CPU only."""
from __future__ import annotations

import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1310_0901_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>
#include "cg_race_index.h"

struct E { int space; uint64_t a, n, seq; bool live; };

static uint64_t rng_state = 88172645463325252ull;
static uint64_t rnd() {  // xorshift64
  rng_state ^= rng_state << 13; rng_state ^= rng_state >> 7; rng_state ^= rng_state << 17;
  return rng_state;
}
static uint64_t pick_len() {
  switch (rnd() % 4) {
    case 0: return 1 + rnd() % 64;
    case 1: return 1 + rnd() % (1u << 16);
    case 2: return 1 + rnd() % (4u << 20);            // up to about the long threshold
    default: return (4u << 20) + rnd() % (300u << 20);  // long ranges
  }
}
int main(int argc, char **argv) {
  rng_state += (uint64_t)atoi(argv[1]);
  const uint64_t span = argc > 2 ? strtoull(argv[2], 0, 10) : (1ull << 31);
  cgi::RaceIndex ix;
  std::vector<E> es;
  uint64_t seq = 0, checked = 0;
  for (int step = 0; step < 6000; step++) {
    const uint64_t r = rnd() % 10;
    if (r < 5) {  // add; half of them through visit_add, which must also find every meeting entry
      E e{(int)(rnd() % 2), rnd() % span, pick_len(), seq++, true};
      if (rnd() % 2) {
        ix.add(e.space, e.a, e.n, e.seq);
      } else {
        std::set<uint64_t> got;
        ix.visit_add(e.space, e.a, e.n, e.seq, [&](uint64_t s) { got.insert(s); });
        for (const E &o : es)
          if (o.live && o.space == e.space && o.a < e.a + e.n && e.a < o.a + o.n) {
            if (!got.count(o.seq)) {
              printf("MISSED (visit_add) seq %llu\n", (unsigned long long)o.seq);
              return 1;
            }
            checked++;
          } else if (!o.live && got.count(o.seq)) {
            printf("STALE (visit_add) seq %llu\n", (unsigned long long)o.seq);
            return 1;
          }
      }
      es.push_back(e);
    } else if (r < 8 && !es.empty()) {  // remove, mostly among the oldest
      const size_t k = rnd() % 3 ? rnd() % (es.size() < 8 ? es.size() : 8) : rnd() % es.size();
      for (size_t i = 0, live = 0; i < es.size(); i++) {
        if (!es[i].live) continue;
        if (live++ == k) {
          ix.remove(es[i].space, es[i].a, es[i].n, es[i].seq);
          es[i].live = false;
          break;
        }
      }
    } else {  // look up
      const int space = (int)(rnd() % 2);
      const uint64_t a = rnd() % span, n = pick_len();
      std::set<uint64_t> got;
      ix.candidates(space, a, n, [&](uint64_t s) { got.insert(s); });
      for (const E &e : es) {
        const bool meets = e.space == space && e.a < a + n && a < e.a + e.n;
        if (e.live && meets && !got.count(e.seq)) {
          printf("MISSED seq %llu\n", (unsigned long long)e.seq);
          return 1;
        }
        if (!e.live && got.count(e.seq)) {
          printf("STALE seq %llu\n", (unsigned long long)e.seq);
          return 1;
        }
        checked += e.live && meets;
      }
    }
  }
  printf("OK %llu\n", (unsigned long long)checked);
  return 0;
}
'''


def _asan_ok() -> bool:
    p = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True)
    path = p.stdout.strip()
    return p.returncode == 0 and os.path.isabs(path) and os.path.exists(path)


@pytest.mark.timeout(300)
def test_race_index_candidates_cover_every_meeting_entry(tmp_path):
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    flags = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all"] if _asan_ok() else []
    subprocess.run(["g++", "-std=c++17", "-O1", "-g", *flags, "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    total = 0
    for seed, span in ((1, 1 << 31), (2, 1 << 31), (3, 1 << 27), (4, 1 << 40)):
        p = subprocess.run([str(exe), str(seed), str(span)], capture_output=True, text=True,
                           timeout=200)
        assert p.returncode == 0 and p.stdout.startswith("OK"), p.stdout + p.stderr
        total += int(p.stdout.split()[1])
    assert total > 1000  # lookups that met live entries

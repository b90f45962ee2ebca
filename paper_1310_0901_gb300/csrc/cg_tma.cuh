// cg_tma.cuh -- the TMA tile pipeline pieces shared by the scan kernels:
// tile geometry, the mbarrier / bulk-copy PTX, and the per-tile producer
// (issue_tile: lane 0 queues a tile's V and A bytes) and consumer
// (consume_tile: every lane classifies and carries from shared memory).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_device.cuh"

#ifndef CG_TMA_R
#define CG_TMA_R 10
#endif
#ifndef CG_TMA_NS
#define CG_TMA_NS 2
#endif
#ifndef CG_TMA_WARPS
#define CG_TMA_WARPS 16
#endif

namespace cgi {

constexpr int kR = CG_TMA_R;       // warp rows per tile
constexpr int kNS = CG_TMA_NS;     // stages per warp
constexpr int kTW = CG_TMA_WARPS;  // warps per CTA
constexpr uint32_t kVBytes = 16u * (32u * kR + 1u);                 // V window of a tile
constexpr uint32_t kABytes = 64u * kR + 64u;                        // A window of a tile
constexpr uint32_t kStage = ((kVBytes + kABytes) + 127u) & ~127u;  // one stage
constexpr uint32_t kWarpSmem = kNS * kStage;
constexpr size_t kSmemBytes = (size_t)kTW * kWarpSmem + (size_t)kTW * kNS * 8 + 128;
constexpr uint64_t kWaitLimitNs = 1000000000ull;
// rows of a device->host carry tile whose merge reads go out together
constexpr int kMergeRows = kR % 5 == 0 ? 5 : (kR % 4 == 0 ? 4 : (kR % 3 == 0 ? 3 : 2));
static_assert(kR % kMergeRows == 0, "merge groups must tile the rows");

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for a stage; false if about one second passes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ int64_t floor16(int64_t x) { return x & ~(int64_t)15; }
__device__ __forceinline__ int64_t ceil16(int64_t x) { return (x + 15) & ~(int64_t)15; }

// Lane 0: queue the V and A bytes of the tile starting at anchor chunk c0
// into the stage at `st` (shared address), completion on `bar`.
template <uint32_t KIND>
__device__ __forceinline__ void issue_tile(const Geo &g, const uint8_t *a_bytes, int64_t c0,
                                           uint32_t st, uint32_t bar) {
  if (c0 >= 1 && c0 + 32 * kR + 2 <= g.nchunks) {
    // An interior tile: neither window reaches past the copy's ends, so no
    // clipping -- the whole V window, and the A bytes from the one holding
    // the tile's first bit (the same copies as the general form below)
    const bool v = KIND == CG_HTOD || g.has_vin;
    const int64_t p0 = g.hb0 + 16 * c0;
    const int64_t aorig = floor16(p0 >> 3);
    const uint32_t abytes =
        KIND != CG_DTOD ? (uint32_t)(ceil16((p0 + 512 * kR + 39) >> 3) - aorig) : 0u;
    mbar_arrive_expect_tx(bar, (v ? kVBytes : 0u) + abytes);
    if (v) bulk_g2s(st, reinterpret_cast<const void *>(g.vin_al + 16 * (uintptr_t)c0), kVBytes, bar);
    if (abytes) bulk_g2s(st + kVBytes, a_bytes + aorig, abytes, bar);
    return;
  }
  uint32_t tx = 0, vbytes = 0, abytes = 0, voff = 0, aoff = 0;
  uintptr_t vsrc = 0;
  int64_t asrc = 0;
  if (KIND == CG_HTOD || g.has_vin) {
    // aligned V chunks of the tile, clipped to the chunks the copy touches
    const uintptr_t vbeg = g.vin_al + 16 * (uintptr_t)c0;
    const uintptr_t vend = vbeg + kVBytes;
    const uintptr_t lo_lim = g.vin_lo & ~(uintptr_t)15;
    const uintptr_t hi_lim = (g.vin_hi + 15) & ~(uintptr_t)15;
    const uintptr_t lo = vbeg > lo_lim ? vbeg : lo_lim;
    const uintptr_t hi = vend < hi_lim ? vend : hi_lim;
    if (hi > lo) {
      vbytes = (uint32_t)(hi - lo);
      voff = (uint32_t)(lo - vbeg);
      vsrc = lo;
      tx += vbytes;
    }
  }
  if (KIND != CG_DTOD) {
    // A bytes holding bits [p0, p1 + 32), clipped to the copy's host bits
    const int64_t p0 = g.hb0 + 16 * c0;
    const int64_t p1 = p0 + 512 * kR;
    const int64_t aorig = floor16(p0 >> 3);
    const int64_t q0 = p0 > g.hlo ? p0 : g.hlo;
    const int64_t q1 = (p1 + 32) < g.hhi ? (p1 + 32) : g.hhi;
    if (q1 > q0) {
      const int64_t b0 = floor16(q0 >> 3);
      const int64_t b1 = ceil16((q1 + 7) >> 3);
      abytes = (uint32_t)(b1 - b0);
      aoff = (uint32_t)(b0 - aorig);
      asrc = b0;
      tx += abytes;
    }
  }
  mbar_arrive_expect_tx(bar, tx);
  if (vbytes) bulk_g2s(st + voff, reinterpret_cast<const void *>(vsrc), vbytes, bar);
  if (abytes) bulk_g2s(st + kVBytes + aoff, a_bytes + asrc, abytes, bar);
}

// ---------------------------------------------------- A-bits-only tiles

// A device->host copy whose source range is invalid reads no V and carries
// nothing: only its destination's A bits decide (unaddressable or good).
// The whole-copy kernels give such a copy tiles of kR*32 "super-chunks" of
// 128 bytes (32 KiB of copy, 4 KiB of A bits per tile) so that each bulk
// copy is as large as a V tile; the chunk index c of these tiles counts
// super-chunks on the same anchor grid (copy offset 128*c - ax).
template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ bool a_only(const Geo &g) {
  return KIND == CG_DTOH && !CARRY && !g.has_vin;
}

__device__ __forceinline__ int64_t super_chunks(const Geo &g) {
  return (g.ax + (int64_t)g.n + 127) >> 7;
}

// Lane 0: queue the A bytes of super-tile c0 (host bits [p0, p0 + 32768 +
// 32), clipped to the copy's) into the stage from its start.
__device__ __forceinline__ void issue_tile_a_super(const Geo &g, const uint8_t *a_bytes,
                                                   int64_t c0, uint32_t st, uint32_t bar) {
  const int64_t p0 = g.hb0 + 128 * c0;
  const int64_t aorig = floor16(p0 >> 3);
  const int64_t q0 = p0 > g.hlo ? p0 : g.hlo;
  const int64_t pe = p0 + 4096 * kR + 32;
  const int64_t q1 = pe < g.hhi ? pe : g.hhi;
  uint32_t bytes = 0;
  int64_t b0 = 0;
  if (q1 > q0) {
    b0 = floor16(q0 >> 3);
    const int64_t b1 = ceil16((q1 + 7) >> 3);
    bytes = (uint32_t)(b1 - b0);
  }
  mbar_arrive_expect_tx(bar, bytes);
  if (bytes) bulk_g2s(st + (uint32_t)(b0 - aorig), a_bytes + b0, bytes, bar);
}

// Classify the A words j = L, L + 32, ... (< nwords) of a tile whose first
// copy byte has offset i0 and whose A window starts bit `rel0` into the
// stage: word j holds copy bytes [i0 + 32 j, +32).  Lanes read consecutive
// words (no bank conflicts); each lane's words come in increasing order, so
// the first zero it finds is its smallest.
__device__ __forceinline__ void classify_a_words(const Geo &g, const uint32_t *as, int64_t i0,
                                                 int64_t rel0, int nwords, int lane,
                                                 LaneAcc &la) {
  const int64_t w0 = rel0 >> 5;
  const int sh = (int)(rel0 & 31);
  uint32_t un = 0;
  unsigned long long first = kNone;
  if (i0 >= 0 && i0 + 32 * (int64_t)nwords <= (int64_t)g.n) {  // every bit valid
    for (int j = lane; j < nwords; j += 32) {
      const uint32_t zero = ~__funnelshift_r(as[w0 + j], as[w0 + j + 1], sh);
      un += __popc(zero);
      if (zero && first == kNone)
        first = (unsigned long long)(g.obase + i0 + 32 * (int64_t)j + __ffs(zero) - 1);
    }
    la.un += un;
    if (first != kNone && la.fun == kNone) {
      la.fun = first;
      la.open_un = 0;
    }
    return;
  }
  for (int j = lane; j < nwords; j += 32) {
    const int64_t b0 = i0 + 32 * (int64_t)j;
    const int64_t lo = b0 < 0 ? -b0 : 0;
    const int64_t rem = (int64_t)g.n - b0;
    const int64_t hi = rem < 32 ? rem : 32;
    if (hi <= lo) continue;
    const uint32_t valid = (hi == 32 ? ~0u : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
    const uint32_t zero = ~__funnelshift_r(as[w0 + j], as[w0 + j + 1], sh) & valid;
    un += __popc(zero);
    if (zero && first == kNone) first = (unsigned long long)(g.obase + b0 + __ffs(zero) - 1);
  }
  la.un += un;
  if (first != kNone && la.fun == kNone) {
      la.fun = first;
      la.open_un = 0;
    }
}

// All lanes: classify a super-tile (128 kR A words, 4096 kR bytes of copy).
__device__ __forceinline__ void consume_tile_a_super(const Geo &g, int64_t c0, const uint8_t *sp,
                                                     int lane, LaneAcc &la) {
  const int64_t p0 = g.hb0 + 128 * c0;
  const int64_t aorig = floor16(p0 >> 3);
  classify_a_words(g, reinterpret_cast<const uint32_t *>(sp), 128 * c0 - g.ax, p0 - 8 * aorig,
                   128 * kR, lane, la);
}

// The same for an ordinary tile (16 kR A words), for the kernels that
// keep 16-byte chunks (pitched rows).
__device__ __forceinline__ void consume_tile_a_only(const Geo &g, int64_t c0, const uint8_t *sp,
                                                    int lane, LaneAcc &la) {
  const int64_t p0 = g.hb0 + 16 * c0;  // host position of the tile's first byte
  const int64_t aorig = floor16(p0 >> 3);
  classify_a_words(g, reinterpret_cast<const uint32_t *>(sp + kVBytes), 16 * c0 - g.ax,
                   p0 - 8 * aorig, 16 * kR, lane, la);
}

// All lanes: classify and carry the tile at anchor chunk c0 from stage `sp`.
// U: rows unrolled (the level kernel, which inlines every kind, takes fewer
// to keep its code small).  SKIP: stop at the last row holding a chunk of
// the copy (rows past it have empty valid masks).  It pays where most tiles
// are ragged (pitched rows of a few tiles each: 16 KiB rows, 0.83 -> 0.85
// of peak) and costs the level kernel its unrolled body's shape (batched
// 0.79 -> 0.76), so only the pitched tile kernel asks for it.
template <uint32_t KIND, bool CARRY, int U = 4, bool SKIP = false>
__device__ __forceinline__ void consume_tile(const Geo &g, int64_t c0, const uint8_t *sp,
                                             int lane, LaneAcc &la) {
  if (KIND == CG_DTOH && !CARRY && !g.has_vin) {  // nothing but the destination's A bits
    consume_tile_a_only(g, c0, sp, lane, la);
    return;
  }
  const uint4 *vs = reinterpret_cast<const uint4 *>(sp);
  const uint32_t *as = reinterpret_cast<const uint32_t *>(sp + kVBytes);
  // bit offset of the tile's first chunk in the tile's A window (which
  // starts at the 16-byte-aligned A byte holding it): in [0, 136), so the
  // per-chunk A addressing below stays in 32-bit arithmetic
  const int64_t p0 = g.hb0 + 16 * c0;
  const int32_t qbase = (int32_t)(p0 - 8 * floor16(p0 >> 3));
  const int64_t i0_tile = 16 * c0 - g.ax;  // copy offset of the tile's first byte
  const bool full = i0_tile >= 0 && i0_tile + 512 * kR <= (int64_t)g.n;
  // A bits of chunk k = 32 u + lane: bit qbase + 16 k of the window, i.e.
  // word a_wi + 16 u at the lane's own shift (the same in every row)
  const int32_t a_q = qbase + 16 * lane;
  const int a_sh = a_q & 31;
  const int a_wi = a_q >> 5;
  auto a16_of = [&](int k) -> uint32_t {
    const int wi = a_wi + 16 * (k >> 5);
    const uint32_t w1 = a_sh > 16 ? as[wi + 1] : 0u;
    return __funnelshift_r(as[wi], w1, a_sh) & 0xFFFFu;
  };
  auto v_of = [&](int k) -> uint4 {
    uint4 V = vs[k];
    if (g.vin_r) V = funnel16(V, vs[k + 1], g.vin_r);
    return V;
  };
  // rows of the tile past the copy's last chunk hold nothing to classify or
  // carry (the ragged last tile of a row or a copy)
  const int64_t rem = g.nchunks - c0;
  const int urows = !SKIP || rem >= 32 * kR ? kR : (int)((rem + 31) >> 5);
  if (!CARRY && KIND != CG_DTOD && kR % 2 == 0) {
    // A check that carries nothing: each lane takes pairs of consecutive
    // chunks (pair p = 32 v + lane holds chunks 2p and 2p + 1, so a lane's
    // chunks still come in increasing order), whose A bits are one 32-bit
    // word at the same shift in every lane: one A extraction, one pair of
    // counts and one first-offset test per two chunks
    const int a_w0 = qbase >> 5, a_s = qbase & 31;
#pragma unroll U
    for (int v = 0; v < kR / 2; v++) {
      if (SKIP && 64 * v >= rem) break;
      const int p = 32 * v + lane;
      const int k = 2 * p;
      uint4 V0 = make_uint4(0, 0, 0, 0), V1 = V0;
      if (KIND == CG_HTOD || g.has_vin) {
        const uint4 x0 = vs[k], x1 = vs[k + 1];
        if (g.vin_r) {
          const uint4 x2 = vs[k + 2];
          V0 = funnel16(x0, x1, g.vin_r);
          V1 = funnel16(x1, x2, g.vin_r);
        } else {
          V0 = x0;
          V1 = x1;
        }
      }
      const uint32_t a32 = __funnelshift_r(as[a_w0 + p], as[a_w0 + p + 1], a_s);
      const int64_t c = c0 + k;
      const uint32_t vm32 = full ? ~0u
                                 : (valid_mask(16 * c - g.ax, g.n) |
                                    (valid_mask(16 * (c + 1) - g.ax, g.n) << 16));
      pair_step(g, c, V0, V1, a32, vm32, la);
    }
    return;
  }
  if (KIND == CG_DTOH && CARRY) {
    // The carry merges device V into the host V blocks that hold
    // unaddressable bytes, reading each such block first.  Rows go in
    // groups of kMergeRows: the blocks of a group are all read before any
    // of them is merged, so those reads overlap instead of each row waiting
    // for its own.
#pragma unroll 1
    for (int u0 = 0; u0 < (SKIP ? urows : kR); u0 += kMergeRows) {
      uint4 old[kMergeRows];
#pragma unroll
      for (int j = 0; j < kMergeRows; j++) {
        const int k = 32 * (u0 + j) + lane;
        const uint32_t a16 = a16_of(k);
        const uint32_t vm = full ? 0xFFFFu : valid_mask(16 * (c0 + k) - g.ax, g.n);
        old[j] = (vm == 0xFFFFu && a16 != 0xFFFFu) ? ld_plain(g.out_al + 16 * (c0 + k))
                                                   : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int j = 0; j < kMergeRows; j++) {
        const int k = 32 * (u0 + j) + lane;
        const uint4 V = g.has_vin ? v_of(k) : make_uint4(0, 0, 0, 0);
        const uint32_t vm = full ? 0xFFFFu : valid_mask(16 * (c0 + k) - g.ax, g.n);
        chunk_step<KIND, CARRY>(g, c0 + k, V, a16_of(k), vm, la, &old[j]);
      }
    }
    return;
  }
#pragma unroll U
  for (int u = 0; u < kR; u++) {
    if (SKIP && u >= urows) break;
    const int k = 32 * u + lane;
    const int64_t c = c0 + k;
    const uint4 V = (KIND == CG_HTOD || g.has_vin) ? v_of(k) : make_uint4(0, 0, 0, 0);
    const uint32_t a16 = KIND != CG_DTOD ? a16_of(k) : 0xFFFFu;
    const uint32_t vm = full ? 0xFFFFu : valid_mask(16 * c - g.ax, g.n);
    chunk_step<KIND, CARRY>(g, c, V, a16, vm, la);
  }
}


// Segment claims of the TMA kernels: static striding (no counter) or
// the next unclaimed segment from a counter; the producer half of a warp
// claims and passes each claim to the consumer half through a small ring
// in shared memory.
// ring entries (a power of two): at most 2 * kNS + 3 claims are outstanding
constexpr int kSegQ = 2 * kNS + 3 <= 8 ? 8 : (2 * kNS + 3 <= 16 ? 16 : 32);
static_assert(2 * kNS + 3 <= kSegQ, "segment-claim ring too small");

struct SegSrc {
  unsigned long long *ctr;  // null: static striding
  uint64_t *q;              // this warp's ring (dynamic only)
  uint64_t step;            // W
  uint32_t n;               // claims pushed (producer) or popped (consumer)
  bool prod;
  __device__ __forceinline__ uint64_t next(uint64_t cur, int lane) {
    if (!ctr) return cur + step;
    uint64_t v = 0;
    if (prod) {
      if (lane == 0) {
        v = step + atomicAdd(ctr, 1ull);
        q[n & (kSegQ - 1)] = v;
      }
      v = __shfl_sync(CG_FULL, v, 0);
    } else {
      __syncwarp();
      v = q[n & (kSegQ - 1)];
    }
    n++;
    return v;
  }
};

}  // namespace cgi

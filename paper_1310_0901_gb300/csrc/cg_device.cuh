// cg_device.cuh -- device helpers shared by libcg's scan kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_internal.h"

namespace cgi {

#define CG_FULL 0xffffffffu

// ------------------------------------------------------------- helpers

__device__ __forceinline__ uint4 ld_stream(const void *p) {
  return __ldcs(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ uint4 ld_plain(const void *p) {
  return __ldcg(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ void st_stream(void *p, uint4 v) {
  __stcs(reinterpret_cast<uint4 *>(p), v);
}

// bytes [r, r+16) of the 32-byte concatenation a||b, 0 <= r < 16
__device__ __forceinline__ uint4 funnel16(uint4 a, uint4 b, int r) {
  const int s = (r & 3) * 8;
  uint4 o;
  switch (r >> 2) {
    case 0:
      o.x = __funnelshift_r(a.x, a.y, s);
      o.y = __funnelshift_r(a.y, a.z, s);
      o.z = __funnelshift_r(a.z, a.w, s);
      o.w = __funnelshift_r(a.w, b.x, s);
      break;
    case 1:
      o.x = __funnelshift_r(a.y, a.z, s);
      o.y = __funnelshift_r(a.z, a.w, s);
      o.z = __funnelshift_r(a.w, b.x, s);
      o.w = __funnelshift_r(b.x, b.y, s);
      break;
    case 2:
      o.x = __funnelshift_r(a.z, a.w, s);
      o.y = __funnelshift_r(a.w, b.x, s);
      o.z = __funnelshift_r(b.x, b.y, s);
      o.w = __funnelshift_r(b.y, b.z, s);
      break;
    default:
      o.x = __funnelshift_r(a.w, b.x, s);
      o.y = __funnelshift_r(b.x, b.y, s);
      o.z = __funnelshift_r(b.y, b.z, s);
      o.w = __funnelshift_r(b.z, b.w, s);
      break;
  }
  return o;
}

// 4-bit mask of the nonzero bytes of x (bit k <-> byte k).  Bit 7 of each
// byte of t is set iff the byte is nonzero: adding 0x7F to its low 7 bits
// carries into bit 7 unless they are all zero (and never past it), OR-ing
// x adds the byte's own bit 7.  The multiply then moves bits 7, 15, 23 and
// 31 to bits 28..31 (partial products land on distinct bits: no carries).
__device__ __forceinline__ uint32_t nz4(uint32_t x) {
  const uint32_t t = (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
  return (t * 0x00204081u) >> 28;
}
__device__ __forceinline__ uint32_t nz16(uint4 v) {
  return nz4(v.x) | (nz4(v.y) << 4) | (nz4(v.z) << 8) | (nz4(v.w) << 12);
}
// 4-bit mask -> 4 bytes of 0x00 / 0xFF
__device__ __forceinline__ uint32_t expand4(uint32_t nib) {
  return ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
}
__device__ __forceinline__ uint4 expand16(uint32_t m) {
  return make_uint4(expand4(m & 0xF), expand4((m >> 4) & 0xF), expand4((m >> 8) & 0xF),
                    expand4((m >> 12) & 0xF));
}

// bytes of copy index [i0, i0+16) that lie in [0, n)
__device__ __forceinline__ uint32_t valid_mask(int64_t i0, uint64_t n) {
  int64_t lo = i0 < 0 ? -i0 : 0;
  int64_t rem = (int64_t)n - i0;
  int64_t hi = rem < 16 ? rem : 16;
  if (hi <= lo) return 0u;
  return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

__device__ __forceinline__ void store_bytes(uint8_t *p, uint4 v, uint32_t m) {
  const uint8_t *b = reinterpret_cast<const uint8_t *>(&v);
  while (m) {
    int k = __ffs(m) - 1;
    p[k] = b[k];
    m &= m - 1;
  }
}

// ----------------------------------------------------- stream geometry

struct Geo {
  uint64_t n;
  int64_t ax;       // anchor address mod 16
  int64_t nchunks;  // 16-byte chunks of the anchor grid covering the copy
  uint8_t *out_al;  // anchor address - ax
  uintptr_t vin_al, vin_lo, vin_hi;
  int vin_r;
  bool has_vin;
  int64_t hb0;  // host position of chunk 0 byte 0 (may be negative)
  int64_t hlo, hhi;
  int64_t obase;  // report offset of copy byte 0 (a row of a pitched copy)
};

__device__ __forceinline__ Geo make_geo(const ScanJob &j, const Image &img) {
  Geo g;
  const bool carry = j.mode & kModeCarry;
  const bool rdev = j.mode & kModeReadDev;
  const uintptr_t host_v = reinterpret_cast<uintptr_t>(img.v) + j.host_off;
  uintptr_t anchor;
  if (j.kind == CG_HTOD)
    anchor = carry ? (uintptr_t)j.dev_dst : host_v;
  else if (j.kind == CG_DTOH)
    anchor = host_v;
  else
    anchor = carry ? (uintptr_t)j.dev_dst : (uintptr_t)j.dev_src;
  g.n = j.n;
  g.ax = (int64_t)(anchor & 15);
  const bool work = !(j.kind == CG_DTOD && !carry && !rdev);
  g.nchunks = work ? (int64_t)((g.ax + j.n + 15) >> 4) : 0;
  g.out_al = reinterpret_cast<uint8_t *>(anchor - g.ax);
  const uintptr_t vin = j.kind == CG_HTOD ? host_v : (uintptr_t)j.dev_src;
  g.has_vin = j.kind == CG_HTOD || rdev;
  const uintptr_t vw = vin - (uintptr_t)g.ax;
  g.vin_r = (int)(vw & 15);
  g.vin_al = vw - (uintptr_t)g.vin_r;
  g.vin_lo = vin;
  g.vin_hi = vin + j.n;
  g.hb0 = (int64_t)j.host_off - g.ax;
  g.hlo = (int64_t)j.host_off;
  g.hhi = (int64_t)(j.host_off + j.n);
  g.obase = 0;
  return g;
}

// The input V window of chunk c (all 32 lanes must call it together).
__device__ __forceinline__ uint4 load_window(const Geo &g, int64_t c, int lane) {
  const uintptr_t a0 = g.vin_al + 16 * (uintptr_t)c;
  const bool in0 = a0 < g.vin_hi && a0 + 16 > g.vin_lo;
  uint4 l0 = in0 ? ld_stream((const void *)a0) : make_uint4(0, 0, 0, 0);
  if (g.vin_r == 0) return l0;  // warp-uniform
  uint4 l1;
  l1.x = __shfl_down_sync(CG_FULL, l0.x, 1);
  l1.y = __shfl_down_sync(CG_FULL, l0.y, 1);
  l1.z = __shfl_down_sync(CG_FULL, l0.z, 1);
  l1.w = __shfl_down_sync(CG_FULL, l0.w, 1);
  if (lane == 31) {
    const uintptr_t a1 = a0 + 16;
    const bool in1 = a1 < g.vin_hi && a1 + 16 > g.vin_lo;
    l1 = in1 ? ld_stream((const void *)a1) : make_uint4(0, 0, 0, 0);
  }
  return funnel16(l0, l1, g.vin_r);
}

// A bits of host positions [hb, hb+16); words outside [hlo, hhi) read as 0.
__device__ __forceinline__ uint32_t load_a16(const uint32_t *A32, int64_t hb, int64_t hlo,
                                             int64_t hhi) {
  const int64_t wi = hb >> 5;  // floor
  const int sh = (int)(hb & 31);
  const int64_t b0 = wi * 32;
  const uint32_t lo = (b0 < hhi && b0 + 32 > hlo) ? __ldg(A32 + wi) : 0u;
  uint32_t hi = 0u;
  if (sh > 16) {
    const int64_t b1 = b0 + 32;
    hi = (b1 < hhi && b1 + 32 > hlo) ? __ldg(A32 + wi + 1) : 0u;
  }
  return __funnelshift_r(lo, hi, sh) & 0xFFFFu;
}

struct LaneAcc {
  uint32_t un, ud;
  // all ones while the lane's first unaddressable (undefined) byte is still
  // to be found, else 0: one mask-and test per chunk (or pair of chunks)
  // instead of 64-bit compares
  uint32_t open_un, open_ud;
  unsigned long long fun, fud;
};

__device__ __forceinline__ void lane_acc_reset(LaneAcc &la) {
  la.un = 0;
  la.ud = 0;
  la.open_un = ~0u;
  la.open_ud = ~0u;
  la.fun = kNone;
  la.fud = kNone;
}


// Classify one 16-byte anchor chunk (copy bytes [i0, i0+16)) and carry it:
// V = the input V window, a16 = its A bits (all ones for device->device).
// old: for a device->host carry, the destination's host V block if the
// caller has read it already (else it is read here when needed).
template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ void chunk_step(const Geo &g, int64_t c, uint4 V, uint32_t a16,
                                           uint32_t vm, LaneAcc &la,
                                           const uint4 *old_in = nullptr) {
  // vm: bytes of this chunk inside the copy (0xFFFF for interior tiles)
  const bool clean = ((V.x | V.y | V.z | V.w) == 0u) && (((a16 | ~vm) & 0xFFFFu) == 0xFFFFu);
  if (!clean && vm) {
    const uint32_t un = vm & ~a16 & 0xFFFFu;
    const uint32_t ud = vm & a16 & nz16(V);
    la.un += __popc(un);
    la.ud += __popc(ud);
    if ((un & la.open_un) | (ud & la.open_ud)) {  // the lane's first bad bytes (rare)
      const int64_t i0 = g.obase + 16 * c - g.ax;
      if (un & la.open_un) {
        la.fun = (unsigned long long)(i0 + __ffs(un) - 1);
        la.open_un = 0;
      }
      if (ud & la.open_ud) {
        la.fud = (unsigned long long)(i0 + __ffs(ud) - 1);
        la.open_ud = 0;
      }
    }
  }
  if (CARRY && vm) {
    uint8_t *p = g.out_al + 16 * c;
    if (KIND == CG_HTOD) {
      uint4 o = V;
      if (a16 != 0xFFFFu) {  // unaddressable source bytes arrive undefined
        const uint4 m = expand16(~a16 & 0xFFFFu);
        o.x |= m.x;
        o.y |= m.y;
        o.z |= m.z;
        o.w |= m.w;
      }
      if (vm == 0xFFFFu)
        st_stream(p, o);
      else
        store_bytes(p, o, vm);
    } else if (KIND == CG_DTOD) {
      if (vm == 0xFFFFu)
        st_stream(p, V);
      else
        store_bytes(p, V, vm);
    } else {  // DtoH: only addressable host bytes take the device V
      const uint32_t wm = vm & a16;
      if (wm == 0xFFFFu) {
        st_stream(p, V);
      } else if (vm == 0xFFFFu) {  // interior chunk with holes: merge
        const uint4 old = old_in ? *old_in : ld_plain(p);
        const uint4 m = expand16(a16);
        uint4 o;
        o.x = (V.x & m.x) | (old.x & ~m.x);
        o.y = (V.y & m.y) | (old.y & ~m.y);
        o.z = (V.z & m.z) | (old.z & ~m.z);
        o.w = (V.w & m.w) | (old.w & ~m.w);
        st_stream(p, o);
      } else if (wm) {
        store_bytes(p, V, wm);
      }
    }
  }
}

// Classify two consecutive anchor chunks (copy bytes [i0, i0+32)) of a
// check that carries nothing: V0, V1 their input V windows, a32 their A
// bits (chunk 2p in the low half), vm32 their bytes inside the copy.  The
// counts and first offsets are chunk_step's for the two chunks in turn;
// one A word, one pair of counts and one first-offset test serve both.
__device__ __forceinline__ void pair_step(const Geo &g, int64_t c, uint4 V0, uint4 V1,
                                          uint32_t a32, uint32_t vm32, LaneAcc &la) {
  const bool clean = ((V0.x | V0.y | V0.z | V0.w | V1.x | V1.y | V1.z | V1.w) == 0u) &&
                     ((a32 | ~vm32) == ~0u);
  if (clean || !vm32) return;
  const uint32_t un = vm32 & ~a32;
  const uint32_t ud = vm32 & a32 & (nz16(V0) | (nz16(V1) << 16));
  la.un += __popc(un);
  la.ud += __popc(ud);
  if ((un & la.open_un) | (ud & la.open_ud)) {  // the lane's first bad bytes (rare)
    const int64_t i0 = g.obase + 16 * c - g.ax;
    if (un & la.open_un) {
      la.fun = (unsigned long long)(i0 + __ffs(un) - 1);
      la.open_un = 0;
    }
    if (ud & la.open_ud) {
      la.fud = (unsigned long long)(i0 + __ffs(ud) - 1);
      la.open_ud = 0;
    }
  }
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(CG_FULL, x, o);
    x = y < x ? y : x;
  }
  return x;
}

// Reduce a warp's lane accumulators into *dst (lane 0 issues the atomics).
__device__ __forceinline__ void warp_flush(LaneAcc &la, Acc *dst, int lane) {
  const uint32_t un = __reduce_add_sync(CG_FULL, la.un);
  const uint32_t ud = __reduce_add_sync(CG_FULL, la.ud);
  unsigned long long fun = kNone, fud = kNone;
  if (__any_sync(CG_FULL, la.fun != kNone)) fun = warp_min64(la.fun);
  if (__any_sync(CG_FULL, la.fud != kNone)) fud = warp_min64(la.fud);
  if (lane == 0) {
    if (un) atomicAdd(&dst->n_unaddr, (unsigned long long)un);
    if (ud) atomicAdd(&dst->n_undef, (unsigned long long)ud);
    if (fun != kNone) atomicMin(&dst->first_unaddr, fun);
    if (fud != kNone) atomicMin(&dst->first_undef, fud);
  }
  lane_acc_reset(la);
}

// Last-CTA epilogue of a single-copy kernel: publish the report, reset the
// scratch for the next launch.
__device__ __forceinline__ void single_epilogue(LaneAcc &la, SingleScratch *scr,
                                                const RangeInfo &ri, cg_report *out,
                                                uint32_t err) {
  const int lane = threadIdx.x & 31;
  warp_flush(la, &scr->acc, lane);
  if (lane == 0 && err) atomicOr(&scr->error, err);
  if (lane == 0) __threadfence();
  __syncthreads();
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(&scr->ctas_done, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    Acc tot;
    tot.n_unaddr = atomicAdd(&scr->acc.n_unaddr, 0ull);
    tot.n_undef = atomicAdd(&scr->acc.n_undef, 0ull);
    tot.first_unaddr = atomicAdd(&scr->acc.first_unaddr, 0ull);
    tot.first_undef = atomicAdd(&scr->acc.first_undef, 0ull);
    const unsigned e = atomicExch(&scr->error, 0u);
    cg_report r;
    assemble_report(&r, ri, tot);
    if (e) r.flags |= CG_F_INCOMPLETE;
    *out = r;
    scr->acc.n_unaddr = 0;
    scr->acc.n_undef = 0;
    scr->acc.first_unaddr = kNone;
    scr->acc.first_undef = kNone;
    scr->ctas_done = 0;
    scr->claim = 0;
    __threadfence_system();
  }
}

}  // namespace cgi

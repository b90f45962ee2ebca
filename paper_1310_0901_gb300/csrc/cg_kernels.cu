// cg_kernels.cu -- sm_103a kernels of libcg.
//
// The hot loop streams the shadow through HBM in 16-byte vectors: a warp
// covers 32 consecutive 16-byte chunks ("a row", 512 B), and every lane
// keeps kU rows of loads in flight before it classifies anything.  The
// chunk grid is aligned to the buffer the copy WRITES (the "anchor"), so
// stores are whole aligned vectors; an input stream with another alignment
// is realigned in registers with one warp shuffle and a byte funnel shift
// (lane 31 fetches the one chunk past the row itself).  Per-byte classes
// (Sec. 2 itemize: unaddressable / undefined) are found with bit tricks on
// 32-bit words and reduced with warp reductions, popc and ffs; counts and
// first offsets go to the request's accumulator with 64-bit atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_internal.h"

namespace cgi {

#define CG_FULL 0xffffffffu
constexpr int kThreads = 256;
constexpr int kU = 4;  // rows of loads in flight per lane

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

// 4-bit mask of the nonzero bytes of x (bit k <-> byte k)
__device__ __forceinline__ uint32_t nz4(uint32_t x) {
  uint32_t t = x | (x >> 4);
  t |= t >> 2;
  t |= t >> 1;
  t &= 0x01010101u;                       // bit 0 of each byte = OR of its bits
  return ((t * 0x00204081u) >> 21) & 0xFu;  // gather bits 0, 8, 16, 24
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
  unsigned long long fun, fud;
};

__device__ __forceinline__ void lane_acc_reset(LaneAcc &la) {
  la.un = 0;
  la.ud = 0;
  la.fun = kNone;
  la.fud = kNone;
}

// kU rows starting at row0; rows >= nrows are skipped (warp-uniform).
template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ void do_rows(const Geo &g, const uint32_t *A32, int64_t row0,
                                        int nrows, int lane, LaneAcc &la) {
  uint4 v[kU];
  uint32_t a[kU];
#pragma unroll
  for (int u = 0; u < kU; u++) {
    const int64_t c = (row0 + u) * 32 + lane;
    v[u] = make_uint4(0, 0, 0, 0);
    a[u] = 0xFFFFu;
    if (u < nrows) {
      if (KIND == CG_HTOD || g.has_vin) v[u] = load_window(g, c, lane);
      if (KIND != CG_DTOD) a[u] = load_a16(A32, g.hb0 + 16 * c, g.hlo, g.hhi);
    }
  }
#pragma unroll
  for (int u = 0; u < kU; u++) {
    if (u >= nrows) break;
    const int64_t c = (row0 + u) * 32 + lane;
    const int64_t i0 = 16 * c - g.ax;
    const uint32_t vm = valid_mask(i0, g.n);
    const uint4 V = v[u];
    const uint32_t a16 = a[u];
    const bool clean = ((V.x | V.y | V.z | V.w) == 0u) && (((a16 | ~vm) & 0xFFFFu) == 0xFFFFu);
    if (!clean && vm) {
      const uint32_t un = vm & ~a16 & 0xFFFFu;
      const uint32_t ud = vm & a16 & nz16(V);
      la.un += __popc(un);
      la.ud += __popc(ud);
      if (un && la.fun == kNone) la.fun = (unsigned long long)(i0 + __ffs(un) - 1);
      if (ud && la.fud == kNone) la.fud = (unsigned long long)(i0 + __ffs(ud) - 1);
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
          const uint4 old = ld_plain(p);
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

template <uint32_t KIND, bool CARRY>
__device__ __forceinline__ void do_range(const Geo &g, const uint32_t *A32, int64_t row_begin,
                                         int64_t row_end, int64_t row_step, int lane,
                                         LaneAcc &la) {
  for (int64_t r = row_begin; r < row_end; r += row_step) {
    const int64_t left = row_end - r;
    do_rows<KIND, CARRY>(g, A32, r, left < kU ? (int)left : kU, lane, la);
  }
}

// ---------------------------------------------------- single-copy kernel

// One copy over the whole grid.  Warps take groups of kU rows in grid-stride
// order; the last CTA to finish publishes the totals and resets the scratch.
template <uint32_t KIND, bool CARRY>
__global__ void __launch_bounds__(kThreads) scan_single_kernel(Image img, ScanJob job,
                                                               RangeInfo ri, SingleScratch *scr,
                                                               cg_report *out) {
  const int lane = threadIdx.x & 31;
  const Geo g = make_geo(job, img);
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rows = (g.nchunks + 31) >> 5;
  LaneAcc la;
  lane_acc_reset(la);
  for (int64_t r = warp * kU; r < rows; r += nwarps * kU) {
    const int64_t left = rows - r;
    do_rows<KIND, CARRY>(g, A32, r, left < kU ? (int)left : kU, lane, la);
  }
  warp_flush(la, &scr->acc, lane);
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
    cg_report r;
    assemble_report(&r, ri, tot);
    *out = r;
    scr->acc.n_unaddr = 0;
    scr->acc.n_undef = 0;
    scr->acc.first_unaddr = kNone;
    scr->acc.first_undef = kNone;
    scr->ctas_done = 0;
    __threadfence_system();
  }
}

__global__ void init_single_scratch_kernel(SingleScratch *s) {
  s->acc.n_unaddr = 0;
  s->acc.n_undef = 0;
  s->acc.first_unaddr = kNone;
  s->acc.first_undef = kNone;
  s->ctas_done = 0;
}

cudaError_t launch_init_single_scratch(SingleScratch *s, cudaStream_t st) {
  init_single_scratch_kernel<<<1, 1, 0, st>>>(s);
  return cudaGetLastError();
}

template <uint32_t KIND, bool CARRY>
static void *single_fn() {
  return reinterpret_cast<void *>(&scan_single_kernel<KIND, CARRY>);
}

static void *pick_single(uint32_t kind, bool carry) {
  switch (kind) {
    case CG_HTOD:
      return carry ? single_fn<CG_HTOD, true>() : single_fn<CG_HTOD, false>();
    case CG_DTOH:
      return carry ? single_fn<CG_DTOH, true>() : single_fn<CG_DTOH, false>();
    default:
      return carry ? single_fn<CG_DTOD, true>() : single_fn<CG_DTOD, false>();
  }
}

int scan_single_max_ctas_per_sm(uint32_t kind, uint32_t mode) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick_single(kind, mode & kModeCarry),
                                                    kThreads, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t launch_scan_single(const Image &img, const ScanJob &job, const RangeInfo &ri,
                               SingleScratch *scratch, cg_report *out, int grid,
                               cudaStream_t st) {
  const bool carry = job.mode & kModeCarry;
  switch (job.kind) {
    case CG_HTOD:
      if (carry)
        scan_single_kernel<CG_HTOD, true><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      else
        scan_single_kernel<CG_HTOD, false><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      break;
    case CG_DTOH:
      if (carry)
        scan_single_kernel<CG_DTOH, true><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      else
        scan_single_kernel<CG_DTOH, false><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      break;
    default:
      if (carry)
        scan_single_kernel<CG_DTOD, true><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      else
        scan_single_kernel<CG_DTOD, false><<<grid, kThreads, 0, st>>>(img, job, ri, scratch, out);
      break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------ batched: lookup

// Binary search of the sorted allocation table (Fig. 2's list).  Every
// `stride`-th base is staged in shared memory, so a lookup costs ~log2 of
// the splitter count in shared memory plus log2(stride) global probes.
__device__ __forceinline__ bool table_side(const DevTable &t, const uint64_t *spl, uint64_t nspl,
                                           uint32_t stride, uint64_t p, uint64_t n,
                                           uint64_t *found, uint64_t *abase, uint64_t *asize,
                                           uint64_t *shadow, uint32_t *flags, uint32_t f_unalloc,
                                           uint32_t f_overrun) {
  // last splitter <= p
  uint64_t lo = 0, hi = nspl;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (spl[mid] <= p)
      lo = mid + 1;
    else
      hi = mid;
  }
  int64_t j = -1;
  if (lo > 0) {
    uint64_t b = (lo - 1) * stride;
    uint64_t e = b + stride < t.count ? b + stride : t.count;
    while (b < e) {  // upper_bound within the block
      const uint64_t mid = (b + e) >> 1;
      if (__ldg(t.base + mid) <= p)
        b = mid + 1;
      else
        e = mid;
    }
    j = (int64_t)b - 1;
  }
  if (j >= 0) {
    const uint64_t base = __ldg(t.base + j);
    const uint64_t size = __ldg(t.size + j);
    if (p - base < size) {
      *found = base + size - p;
      *abase = base;
      *asize = size;
      *shadow = __ldg(t.shadow + j) + (p - base);
      if (n > *found) {
        *flags |= f_overrun;
        return false;
      }
      return true;
    }
  }
  *found = 0;
  *abase = 0;
  *asize = 0;
  *shadow = 0;
  *flags |= f_unalloc;
  return false;
}

__global__ void __launch_bounds__(256) lookup_kernel(DevTable t, BatchPlan p, uint32_t stride,
                                                     int carry_on) {
  extern __shared__ uint64_t spl[];
  const uint64_t nspl = (t.count + stride - 1) / stride;
  for (uint64_t k = threadIdx.x; k < nspl; k += blockDim.x) spl[k] = __ldg(t.base + k * stride);
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nreq;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const cg_copy q = p.reqs[i];
    RangeInfo ri;
    ri.flags = 0;
    ri.kind = q.kind;
    ri.n = q.n;
    ri.found_dst = ri.found_src = 0;
    ri.base_dst = ri.size_dst = ri.base_src = ri.size_src = 0;
    ScanJob j;
    j.kind = q.kind;
    j.mode = 0;
    j.n = q.n;
    j.host_off = q.kind == CG_HTOD ? q.src : (q.kind == CG_DTOH ? q.dst : 0);
    j.dev_src = 0;
    j.dev_dst = 0;
    Acc a;
    a.n_unaddr = 0;
    a.n_undef = 0;
    a.first_unaddr = kNone;
    a.first_undef = kNone;
    if (q.n > 0) {
      bool dst_ok = true, src_ok = true;
      uint64_t dsh = 0, ssh = 0;
      if (q.kind != CG_DTOH)
        dst_ok = table_side(t, spl, nspl, stride, q.dst, q.n, &ri.found_dst, &ri.base_dst,
                            &ri.size_dst, &dsh, &ri.flags, CG_F_UNALLOC_DST, CG_F_OVERRUN_DST);
      if (q.kind != CG_HTOD)
        src_ok = table_side(t, spl, nspl, stride, q.src, q.n, &ri.found_src, &ri.base_src,
                            &ri.size_src, &ssh, &ri.flags, CG_F_UNALLOC_SRC, CG_F_OVERRUN_SRC);
      if (q.kind == CG_DTOD) {
        const uint64_t dist = q.src <= q.dst ? q.dst - q.src : q.src - q.dst;
        if (dist < q.n) ri.flags |= CG_F_DTOD_OVERLAP;
      }
      if (q.kind != CG_HTOD && src_ok) {
        j.mode |= kModeReadDev;
        j.dev_src = p.stage[i] ? p.stage[i] : ssh;
      }
      if (carry_on && dst_ok && src_ok) {
        j.mode |= kModeCarry;
        j.dev_dst = dsh;  // 0 for DtoH: the host image is the destination
      }
    }
    p.jobs[i] = j;
    p.info[i] = ri;
    p.acc[i] = a;
  }
}

cudaError_t launch_lookup(const DevTable &t, const BatchPlan &p, int strict, int carry,
                          cudaStream_t st) {
  (void)strict;
  if (p.nreq == 0) return cudaSuccess;
  uint32_t stride = 256;
  while ((t.count + stride - 1) / stride > 6144) stride <<= 1;
  const uint64_t nspl = (t.count + stride - 1) / stride;
  const size_t smem = (size_t)(nspl ? nspl : 1) * sizeof(uint64_t);
  uint64_t blocks = (p.nreq + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  lookup_kernel<<<(unsigned)blocks, 256, smem, st>>>(t, p, stride, carry);
  return cudaGetLastError();
}

// ---------------------------------------------------- batched: one level

// Persistent-style kernel over the byte segments of every copy of one
// dependency level.  Warp w takes segments w, w + W, ...; a segment maps to
// its copy by binary search over the level's segment prefix.
__global__ void __launch_bounds__(kThreads) scan_level_kernel(Image img, BatchPlan p,
                                                              uint64_t pos_begin, uint64_t pos_end,
                                                              uint64_t n_segs) {
  const int lane = threadIdx.x & 31;
  const uint32_t *A32 = reinterpret_cast<const uint32_t *>(img.a_bits);
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t seg_rows = p.seg_chunks >> 5;
  LaneAcc la;
  lane_acc_reset(la);
  for (uint64_t s = warp; s < n_segs; s += nwarps) {
    uint64_t lo = pos_begin, hi = pos_end;  // last position with seg_first <= s
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (__ldg(p.seg_first + mid) <= s)
        lo = mid;
      else
        hi = mid;
    }
    const uint32_t req = __ldg(p.order + lo);
    const ScanJob job = p.jobs[req];
    const Geo g = make_geo(job, img);
    const int64_t k = (int64_t)(s - __ldg(p.seg_first + lo));
    const int64_t rows = (g.nchunks + 31) >> 5;
    const int64_t r0 = k * seg_rows;
    const int64_t r1 = r0 + seg_rows < rows ? r0 + seg_rows : rows;
    if (r0 < r1) {
      const bool carry = job.mode & kModeCarry;
      switch (job.kind) {
        case CG_HTOD:
          if (carry)
            do_range<CG_HTOD, true>(g, A32, r0, r1, kU, lane, la);
          else
            do_range<CG_HTOD, false>(g, A32, r0, r1, kU, lane, la);
          break;
        case CG_DTOH:
          if (carry)
            do_range<CG_DTOH, true>(g, A32, r0, r1, kU, lane, la);
          else
            do_range<CG_DTOH, false>(g, A32, r0, r1, kU, lane, la);
          break;
        default:
          if (carry)
            do_range<CG_DTOD, true>(g, A32, r0, r1, kU, lane, la);
          else
            do_range<CG_DTOD, false>(g, A32, r0, r1, kU, lane, la);
          break;
      }
      warp_flush(la, &p.acc[req], lane);
    }
  }
}

cudaError_t launch_scan_level(const Image &img, const BatchPlan &p, uint64_t pos_begin,
                              uint64_t pos_end, uint64_t n_segs, int grid, cudaStream_t st) {
  if (n_segs == 0 || pos_end <= pos_begin) return cudaSuccess;
  const uint64_t warps_needed = n_segs;
  const uint64_t ctas_needed = (warps_needed + (kThreads / 32) - 1) / (kThreads / 32);
  const unsigned g = (unsigned)(ctas_needed < (uint64_t)grid ? ctas_needed : (uint64_t)grid);
  scan_level_kernel<<<g, kThreads, 0, st>>>(img, p, pos_begin, pos_end, n_segs);
  return cudaGetLastError();
}

// --------------------------------------- batched: reports and records

// Block-wide exclusive scan of per-thread values (256 threads).
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t x, uint64_t *total) {
  __shared__ uint64_t warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(CG_FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint64_t before = 0, all = 0;
  for (int k = 0; k < kThreads / 32; k++) {
    if (k < w) before += warp_tot[k];
    all += warp_tot[k];
  }
  __syncthreads();
  if (total) *total = all;
  return before + incl - x;
}

constexpr int kPerThread = kFinalizeItems / kThreads;

__global__ void __launch_bounds__(kThreads) finalize_kernel(BatchPlan p, cg_report *reps,
                                                            uint32_t *counts,
                                                            uint64_t *block_sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kFinalizeItems + threadIdx.x * kPerThread;
  uint64_t mine = 0;
  for (int k = 0; k < kPerThread; k++) {
    const uint64_t i = base + k;
    if (i >= p.nreq) break;
    cg_report r;
    assemble_report(&r, p.info[i], p.acc[i]);
    reps[i] = r;
    const uint32_t c = record_count(r.flags);
    counts[i] = c;
    mine += c;
  }
  uint64_t total;
  block_exclusive_scan(mine, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Exclusive scan of the block sums in one CTA; total count at block_sums[nblocks].
__global__ void __launch_bounds__(kThreads) scan_block_sums_kernel(uint64_t *sums,
                                                                   uint64_t nblocks) {
  uint64_t carry = 0;
  for (uint64_t b0 = 0; b0 < nblocks; b0 += kThreads) {
    const uint64_t i = b0 + threadIdx.x;
    const uint64_t x = i < nblocks ? sums[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan(x, &tot);
    if (i < nblocks) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nblocks] = carry;
}

__global__ void __launch_bounds__(kThreads) emit_records_kernel(BatchPlan p, const cg_report *reps,
                                                                const uint32_t *counts,
                                                                const uint64_t *block_off,
                                                                int strict, cg_err_record *recs,
                                                                uint64_t rec_cap) {
  const uint64_t base = (uint64_t)blockIdx.x * kFinalizeItems + threadIdx.x * kPerThread;
  uint64_t mine = 0;
  for (int k = 0; k < kPerThread; k++) {
    const uint64_t i = base + k;
    if (i < p.nreq) mine += counts[i];
  }
  uint64_t off = block_off[blockIdx.x] + block_exclusive_scan(mine, nullptr);
  for (int k = 0; k < kPerThread; k++) {
    const uint64_t i = base + k;
    if (i >= p.nreq) break;
    const uint32_t c = counts[i];
    if (c && off < rec_cap) {
      const cg_report r = reps[i];
      write_records(r, p.reqs[i], i, strict, recs + off, rec_cap - off);
    }
    off += c;
  }
}

cudaError_t launch_finalize(const BatchPlan &p, cg_report *reps, uint32_t *counts,
                            uint64_t *block_sums, int items_per_block, cudaStream_t st) {
  (void)items_per_block;
  const uint64_t nb = (p.nreq + kFinalizeItems - 1) / kFinalizeItems;
  if (nb == 0) return cudaSuccess;
  finalize_kernel<<<(unsigned)nb, kThreads, 0, st>>>(p, reps, counts, block_sums);
  return cudaGetLastError();
}

cudaError_t launch_scan_block_sums(uint64_t *block_sums, uint64_t nblocks, uint64_t *total,
                                   cudaStream_t st) {
  (void)total;
  scan_block_sums_kernel<<<1, kThreads, 0, st>>>(block_sums, nblocks);
  return cudaGetLastError();
}

cudaError_t launch_emit_records(const BatchPlan &p, const cg_report *reps, const uint32_t *counts,
                                const uint64_t *block_sums, int items_per_block, int strict,
                                cg_err_record *recs, uint64_t rec_cap, cudaStream_t st) {
  (void)items_per_block;
  const uint64_t nb = (p.nreq + kFinalizeItems - 1) / kFinalizeItems;
  if (nb == 0 || rec_cap == 0) return cudaSuccess;
  emit_records_kernel<<<(unsigned)nb, kThreads, 0, st>>>(p, reps, counts, block_sums, strict,
                                                         recs, rec_cap);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fill

// Fill shadow ranges (256-byte aligned, multiples of 256 bytes) with a value.
__global__ void fill_kernel(const uint64_t *ptrs, const uint64_t *sizes, uint64_t count,
                            uint32_t word) {
  for (uint64_t e = blockIdx.x; e < count; e += gridDim.x) {
    uint4 *p = reinterpret_cast<uint4 *>(ptrs[e]);
    const uint64_t nv = sizes[e] >> 4;
    const uint4 w = make_uint4(word, word, word, word);
    for (uint64_t k = threadIdx.x; k < nv; k += blockDim.x) p[k] = w;
  }
}

cudaError_t launch_fill(const uint64_t *ptrs, const uint64_t *sizes, uint64_t count,
                        uint8_t value, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const uint32_t word = 0x01010101u * value;
  const unsigned blocks = (unsigned)(count < 65535 ? count : 65535);
  fill_kernel<<<blocks, 256, 0, st>>>(ptrs, sizes, count, word);
  return cudaGetLastError();
}

}  // namespace cgi

// cg_devops_kernels.cu -- kernels for the memset wrappers and kernel-argument checks.
//
// A memset or a kernel's write argument makes its device bytes defined:
// their V shadow is filled with zeros (1 byte written per byte, HBM-bound).
// Fills are laid out on the 16-byte grid of the span they cover: whole
// aligned vectors inside, byte stores at a ragged head or tail.  The
// undefined-byte scan of a kernel's read arguments runs on the batched scan
// kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_device.cuh"
#include "cg_launch.h"

namespace cgi {

constexpr int kFThreads = 256;
constexpr int kFU = 8;  // chunks per lane per item on long spans

// Fill chunk c of the span [p, p+n) (16-byte grid of p) with `w`.
__device__ __forceinline__ void fill_chunk(uintptr_t p, uint64_t n, int64_t c, uint4 w) {
  const int64_t ax = (int64_t)(p & 15);
  const uint32_t m = valid_mask(16 * c - ax, n);
  if (!m) return;
  uint8_t *q = reinterpret_cast<uint8_t *>((p & ~(uintptr_t)15) + 16 * (uintptr_t)c);
  if (m == 0xFFFFu)
    st_stream(q, w);
  else
    store_bytes(q, w, m);
}

// Rows of a pitched memset: items (row, group of P*U chunks), P = 2^lp lanes
// per item and 32/P items per warp at once; `groups` groups per row.
__global__ void __launch_bounds__(kFThreads) fill_rows_kernel(uint8_t *base, uint64_t pitch,
                                                              uint64_t width, uint64_t rows,
                                                              uint32_t word, uint32_t lp,
                                                              uint32_t u, uint64_t groups,
                                                              RangeInfo ri, cg_report *out) {
  if (out && blockIdx.x == 0 && threadIdx.x == 0) {  // the verdict is known at launch
    const Acc none{0, 0, kNone, kNone};
    cg_report r;
    assemble_report(&r, ri, none);
    *out = r;
  }
  const int lane = threadIdx.x & 31;
  const uint32_t P = 1u << lp;
  const uint32_t ls = lane & (P - 1);
  const uint64_t per_warp = 32u >> lp;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t items = rows * groups;
  const uint4 w = make_uint4(word, word, word, word);
  for (uint64_t t = warp * per_warp + (lane >> lp); t < items; t += nwarps * per_warp) {
    const uint64_t row = groups == 1 ? t : t / groups;
    const uint64_t g = t - row * groups;
    const uintptr_t p = reinterpret_cast<uintptr_t>(base) + row * pitch;
    for (uint32_t k = 0; k < u; k++)
      fill_chunk(p, width, (int64_t)(g * P * u + k * P + ls), w);
  }
}

cudaError_t launch_fill_rows(uint8_t *base, uint64_t pitch, uint64_t width, uint64_t rows,
                             uint8_t value, const RangeInfo &ri, cg_report *out, int sm_count,
                             cudaStream_t st) {
  const uint64_t chunks = (width + 30) >> 4;  // any alignment
  uint32_t lp = 0, u = 1;
  uint64_t groups = 1;
  if (chunks > 32) {
    lp = 5;
    u = kFU;
    groups = (chunks + 32 * kFU - 1) / (32 * kFU);
  } else {
    while ((1ull << lp) < chunks) lp++;
  }
  const uint64_t per_warp = 32u >> lp;
  const uint64_t warps = (rows * groups + per_warp - 1) / per_warp;
  const uint64_t need = (warps + kFThreads / 32 - 1) / (kFThreads / 32);
  const uint64_t cap = (uint64_t)sm_count * 8;
  const unsigned grid = (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
  fill_rows_kernel<<<grid, kFThreads, 0, st>>>(base, pitch, width, rows, 0x01010101u * value, lp,
                                              u, groups, ri, out);
  return cudaGetLastError();
}

// A list of spans (ptr[i], n[i]); span i owns groups seg_first[i] ..
// seg_first[i+1]-1 (of 32*kFU chunks); a warp takes one group at a time.
__global__ void __launch_bounds__(kFThreads) fill_spans_kernel(const uint64_t *ptr,
                                                               const uint64_t *n,
                                                               const uint64_t *seg_first,
                                                               uint64_t count, uint64_t nsegs,
                                                               uint32_t word) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint4 w = make_uint4(word, word, word, word);
  for (uint64_t s = warp; s < nsegs; s += nwarps) {
    uint64_t lo = 0, hi = count;  // last span with seg_first <= s
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (__ldg(seg_first + mid) <= s)
        lo = mid;
      else
        hi = mid;
    }
    const uint64_t len = __ldg(n + lo);
    if (!len) continue;
    const uintptr_t p = (uintptr_t)__ldg(ptr + lo);
    const int64_t c0 = (int64_t)(s - __ldg(seg_first + lo)) * 32 * kFU;
#pragma unroll
    for (int k = 0; k < kFU; k++) fill_chunk(p, len, c0 + 32 * k + lane, w);
  }
}

uint64_t fill_span_groups(uint64_t n) { return n ? (((n + 30) >> 4) + 32 * kFU - 1) / (32 * kFU) : 0; }

cudaError_t launch_fill_spans(const uint64_t *ptr, const uint64_t *n, const uint64_t *seg_first,
                              uint64_t count, uint64_t nsegs, uint8_t value, int sm_count,
                              cudaStream_t st) {
  if (!nsegs || !count) return cudaSuccess;
  const uint64_t need = (nsegs + kFThreads / 32 - 1) / (kFThreads / 32);
  const uint64_t cap = (uint64_t)sm_count * 8;
  const unsigned grid = (unsigned)(need < cap ? need : cap);
  fill_spans_kernel<<<grid, kFThreads, 0, st>>>(ptr, n, seg_first, count, nsegs,
                                                0x01010101u * value);
  return cudaGetLastError();
}

// ------------------------------------------------------ kernel arguments

}  // namespace cgi

// cg_pitched.cpp -- pitched 2-D / 3-D copy checks and device arrays.
//
// The context keeps two lists, as Fig. 2 draws them: linear allocations
// (cg_register_alloc) and device arrays keyed by handle (cg_register_array).
// A pitched copy is validated and range-checked here on the host (the
// extent of a linear side must lie in one allocation; an array side must
// fit its array per dimension) and then scanned by one launch of the
// pitched kernel, which reads and classifies only the copied bytes.
#include <cuda_runtime.h>

#include "cg_ctx.h"

using namespace cgi;

namespace {

// Where the copy's bytes lie on one side.
struct SideGeo {
  uint64_t start = 0;  // host offset / device address / dense array position of byte (0,0,0)
  uint64_t pitch = 0;
  uint64_t slice = 0;
  uint64_t extent = 0;  // first to one past the last copied byte (linear sides)
};

bool mul_over(uint64_t a, uint64_t b, uint64_t *out) { return __builtin_mul_overflow(a, b, out); }
bool add_over(uint64_t a, uint64_t b, uint64_t *out) { return __builtin_add_overflow(a, b, out); }

// Linear side: origin and extent in 64 bits, or CG_E_WRAP.
cg_status linear_geo(const cg_side3d &s, uint64_t w, uint64_t h, uint64_t d, SideGeo *g) {
  uint64_t slice, oz, oy, off, start, ez, ey, ext;
  if (mul_over(s.pitch, s.rows, &slice) || mul_over(s.z, slice, &oz) ||
      mul_over(s.y, s.pitch, &oy) || add_over(oz, oy, &off) || add_over(off, s.x, &off) ||
      add_over(s.ptr, off, &start) || mul_over(d - 1, slice, &ez) ||
      mul_over(h - 1, s.pitch, &ey) || add_over(ez, ey, &ext) || add_over(ext, w, &ext))
    return set_error(CG_E_WRAP, "pitched copy geometry exceeds 64 bits");
  g->start = start;
  g->pitch = s.pitch;
  g->slice = slice;
  g->extent = ext;
  return CG_OK;
}

cg_status side_args(const cg_side3d &s, uint64_t w, uint64_t h, uint64_t d) {
  if (s.is_array) return CG_OK;
  if ((h > 1 || d > 1) && s.pitch < w)
    return set_error(CG_E_ARG, "pitch smaller than the row width");
  if (d > 1 && s.rows < h) return set_error(CG_E_ARG, "rows per slice smaller than the height");
  return CG_OK;
}

// One device side: array lookup with per-dimension bounds, or the linear
// range check of its extent.  *ok = the range passed; *shadow_start,
// *pitch, *slice give the shadow placement of the copied bytes.
cg_status device_side3d(const cg_ctx *c, const cg_side3d &s, uint64_t w, uint64_t h, uint64_t d,
                        uint64_t *found, uint64_t *abase, uint64_t *asize, uint32_t *flags,
                        uint32_t f_unalloc, uint32_t f_overrun, bool *ok, uint64_t *shadow_start,
                        uint64_t *pitch, uint64_t *slice) {
  *ok = false;
  if (s.is_array) {
    *found = *abase = *asize = 0;
    auto it = c->arrays.find(s.ptr);
    if (it == c->arrays.end()) {
      *flags |= f_unalloc;
      return CG_OK;
    }
    const cg_ctx::ArrayInfo &a = it->second;
    *abase = s.ptr;
    *asize = a.w * a.h * a.d;
    if (s.x < a.w && s.y < a.h && s.z < a.d) *found = *asize - ((s.z * a.h + s.y) * a.w + s.x);
    const bool fits = s.x <= a.w && w <= a.w - s.x && s.y <= a.h && h <= a.h - s.y &&
                      s.z <= a.d && d <= a.d - s.z;
    if (!fits) {
      *flags |= f_overrun;
      return CG_OK;
    }
    *shadow_start = a.shadow + (s.z * a.h + s.y) * a.w + s.x;
    *pitch = a.w;
    *slice = a.w * a.h;
    *ok = true;
    return CG_OK;
  }
  SideGeo g;
  CG_TRY(linear_geo(s, w, h, d, &g));
  uint64_t sh = 0;
  *ok = host_side(c, g.start, g.extent, found, abase, asize, &sh, flags, f_unalloc, f_overrun);
  *shadow_start = sh;
  *pitch = g.pitch;
  *slice = g.slice;
  return CG_OK;
}

// R22: the spans of a device->device copy intersect (arrays: the same
// array, spans in its dense layout).
bool spans_meet(const cg_ctx *c, const cg_copy3d &q) {
  const uint64_t w = q.width, h = q.height, d = q.depth;
  if (q.dst.is_array != q.src.is_array) return false;
  uint64_t ds, ss, dext, sext;
  if (q.dst.is_array) {
    if (q.dst.ptr != q.src.ptr) return false;
    auto it = c->arrays.find(q.dst.ptr);
    if (it == c->arrays.end()) return false;
    const cg_ctx::ArrayInfo &a = it->second;
    ds = (q.dst.z * a.h + q.dst.y) * a.w + q.dst.x;
    ss = (q.src.z * a.h + q.src.y) * a.w + q.src.x;
    dext = sext = ((d - 1) * a.h + (h - 1)) * a.w + w;
    return ds < ss + sext && ss < ds + dext;
  }
  SideGeo gd, gs;
  if (linear_geo(q.dst, w, h, d, &gd) != CG_OK || linear_geo(q.src, w, h, d, &gs) != CG_OK)
    return false;
  return gd.start - gs.start < gs.extent || gs.start - gd.start < gd.extent;
}

struct Prepared {
  RangeInfo ri{};
  PitchedJob job{};
  bool trivial = false;
  bool stage = false;
};

cg_status prepare3d(cg_ctx *c, const cg_copy3d &q, Prepared *P) {
  const uint32_t kind = q.kind;
  if (kind != CG_HTOD && kind != CG_DTOH && kind != CG_DTOD)
    return set_error(CG_E_KIND, "copy kind must be CG_HTOD, CG_DTOH or CG_DTOD");
  if (q.reserved || q.dst.reserved || q.src.reserved)
    return set_error(CG_E_ARG, "reserved fields must be 0");
  const uint64_t w = q.width, h = q.height, d = q.depth;
  uint64_t wh = 0, n = 0;
  if (mul_over(w, h, &wh) || mul_over(wh, d, &n))
    return set_error(CG_E_WRAP, "width*height*depth exceeds 64 bits");
  if ((kind == CG_HTOD && q.src.is_array) || (kind == CG_DTOH && q.dst.is_array))
    return set_error(CG_E_ARG, "the host side of a copy cannot be an array");
  P->ri = RangeInfo{};
  P->ri.kind = kind;
  P->ri.n = n;
  P->job = PitchedJob{};
  P->job.kind = kind;
  P->job.width = w;
  P->job.height = h;
  P->job.depth = d;
  P->trivial = n == 0;  // R9
  P->stage = false;
  if (n == 0) return CG_OK;
  CG_TRY(side_args(q.dst, w, h, d));
  CG_TRY(side_args(q.src, w, h, d));
  if (kind != CG_DTOD) {
    if (!c->img_bound) return set_error(CG_E_NO_HOST, "no host shadow image bound");
    SideGeo g;
    CG_TRY(linear_geo(kind == CG_HTOD ? q.src : q.dst, w, h, d, &g));
    if (g.start > c->img.n || g.extent > c->img.n - g.start)
      return set_error(CG_E_HOST_RANGE, "host extent outside the bound host image");
    P->job.host_start = g.start;
    P->job.host_pitch = g.pitch;
    P->job.host_slice = g.slice;
  }
  bool dst_ok = true, src_ok = true;
  RangeInfo &ri = P->ri;
  if (kind != CG_DTOH)
    CG_TRY(device_side3d(c, q.dst, w, h, d, &ri.found_dst, &ri.base_dst, &ri.size_dst, &ri.flags,
                         CG_F_UNALLOC_DST, CG_F_OVERRUN_DST, &dst_ok, &P->job.dst_start,
                         &P->job.dst_pitch, &P->job.dst_slice));
  if (kind != CG_HTOD)
    CG_TRY(device_side3d(c, q.src, w, h, d, &ri.found_src, &ri.base_src, &ri.size_src, &ri.flags,
                         CG_F_UNALLOC_SRC, CG_F_OVERRUN_SRC, &src_ok, &P->job.src_start,
                         &P->job.src_pitch, &P->job.src_slice));
  const bool overlap = kind == CG_DTOD && spans_meet(c, q);
  if (overlap) ri.flags |= CG_F_DTOD_OVERLAP;
  if (kind != CG_HTOD && src_ok) P->job.mode |= kModeReadDev;
  if (c->cfg.carry && dst_ok && src_ok) P->job.mode |= kModeCarry;
  if (kind == CG_DTOD && !(P->job.mode & (kModeCarry | kModeReadDev))) P->trivial = true;
  P->stage = overlap && (P->job.mode & kModeCarry);  // R22: read the whole source first
  return CG_OK;
}

// 16-byte chunks of a row on the grid of the buffer the scan writes (the
// kernels' anchor): exact when every row starts at the same address mod 16,
// else the bound for any alignment.
uint64_t row_chunks(const cg_ctx *c, const PitchedJob &j) {
  const bool carry = j.mode & kModeCarry;
  const uint64_t host = reinterpret_cast<uint64_t>(c->img.v) + j.host_start;
  uint64_t a = 0, pitch = 0, slice = 0;
  if (j.kind == CG_DTOH || (j.kind == CG_HTOD && !carry)) {
    a = host, pitch = j.host_pitch, slice = j.host_slice;
  } else if (carry) {
    a = j.dst_start, pitch = j.dst_pitch, slice = j.dst_slice;
  } else {
    a = j.src_start, pitch = j.src_pitch, slice = j.src_slice;
  }
  const bool uniform = (j.height == 1 || pitch % 16 == 0) && (j.depth == 1 || slice % 16 == 0);
  return uniform ? ((a & 15) + j.width + 15) >> 4 : (j.width + 30) >> 4;
}

cg_status enqueue3d(cg_ctx *c, Prepared &P, cg_report *out, cudaStream_t st) {
  NvtxRange range("cg check pitched copy");
  CG_TRY(flush_fills(c, st));
  if (P.trivial) {  // no byte to read: the report alone
    ScanJob none{};
    none.kind = CG_DTOD;
    CG_CUDA(launch_scan_single(c->img, none, P.ri, c->d_scratch, out, 1, st));
    c->stats.kernels++;
    return CG_OK;
  }
  PitchedJob job = P.job;
  if (P.stage) {
    const uint64_t n = job.width * job.height * job.depth;
    CG_TRY(c->stage.ensure(round_up(n, 256)));
    CG_CUDA(launch_gather_rows(reinterpret_cast<const uint8_t *>(job.src_start), job.src_pitch,
                               job.src_slice, job.width, job.height, job.depth, c->stage.p,
                               c->sm_count, st));
    job.src_start = reinterpret_cast<uint64_t>(c->stage.p);
    job.src_pitch = job.width;
    job.src_slice = job.width * job.height;
    c->stats.kernels++;
  }
  CG_CUDA(launch_scan_pitched(c->img, job, P.ri, c->d_scratch, out, c->sm_count,
                              row_chunks(c, job), !c->img_on_host || job.kind == CG_DTOD, st));
  c->stats.kernels++;
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_register_array(cg_ctx *c, uint64_t handle, uint64_t width, uint64_t height,
                            uint64_t depth) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c) return set_error(CG_E_ARG, "ctx is NULL");
  if (width == 0 || height == 0 || depth == 0)
    return set_error(CG_E_ZERO_SIZE, "zero-size array");
  uint64_t wh, bytes;
  if (mul_over(width, height, &wh) || mul_over(wh, depth, &bytes))
    return set_error(CG_E_WRAP, "array size exceeds 64 bits");
  if (c->arrays.count(handle)) return set_error(CG_E_OVERLAP, "array handle already live");
  if (c->fault_pending & CG_FAULT_SHADOW_ALLOC) {
    c->fault_pending &= ~CG_FAULT_SHADOW_ALLOC;
    return set_error(CG_E_NOMEM, "shadow allocation failed (injected fault)");
  }
  uint64_t sh = 0;
  CG_TRY(c->arena.alloc(bytes, &sh));
  c->arrays[handle] = cg_ctx::ArrayInfo{width, height, depth, sh};
  c->freed_arrays.erase(handle);
  return CG_OK;
}

cg_status cg_free_array(cg_ctx *c, uint64_t handle, uint32_t *verdict) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !verdict) return set_error(CG_E_ARG, "NULL argument");
  auto it = c->arrays.find(handle);
  if (it == c->arrays.end()) {
    *verdict = c->freed_arrays.count(handle) ? CG_FREE_DOUBLE : CG_FREE_UNKNOWN;
    return CG_OK;
  }
  const uint64_t bytes = it->second.w * it->second.h * it->second.d;
  c->arena.release(it->second.shadow, bytes);
  c->fill_ptr.push_back(it->second.shadow);  // back to 0xFF before reuse
  c->fill_size.push_back(bytes);
  c->arrays.erase(it);
  c->freed_arrays.insert(handle);
  *verdict = CG_FREE_OK;
  return CG_OK;
}

cg_status cg_read_array_shadow(cg_ctx *c, uint64_t handle, uint64_t off, uint64_t n,
                               uint8_t *out) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || (n && !out)) return set_error(CG_E_ARG, "NULL argument");
  auto it = c->arrays.find(handle);
  if (it == c->arrays.end()) return set_error(CG_E_RANGE, "no live array with this handle");
  const uint64_t bytes = it->second.w * it->second.h * it->second.d;
  if (off > bytes || n > bytes - off) return set_error(CG_E_RANGE, "span outside the array");
  if (n == 0) return CG_OK;
  CG_TRY(flush_fills(c, 0));
  CG_CUDA(cudaDeviceSynchronize());
  CG_CUDA(cudaMemcpy(out, reinterpret_cast<const void *>(it->second.shadow + off), n,
                     cudaMemcpyDeviceToHost));
  return CG_OK;
}

cg_status cg_check_copy3d(cg_ctx *c, const cg_copy3d *req, cg_report *rep, void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !req || !rep) return set_error(CG_E_ARG, "NULL argument");
  Prepared P;
  CG_TRY(prepare3d(c, *req, &P));
  if (P.trivial) {
    const Acc none{0, 0, kNone, kNone};
    assemble_report(rep, P.ri, none);
    count_stats(c, *rep);
    return CG_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CG_TRY(enqueue3d(c, P, c->d_result, st));
  CG_CUDA(cudaStreamSynchronize(st));
  std::memcpy(rep, c->h_result, sizeof(cg_report));
  if (rep->flags & CG_F_INCOMPLETE)
    return set_error(CG_E_TIMEOUT, "a bounded wait in the scan kernel ran out");
  count_stats(c, *rep);
  return CG_OK;
}

cg_status cg_check_copy3d_async(cg_ctx *c, const cg_copy3d *req, cg_report *rep_dev,
                                void *stream) {
  if (c && c->serve) return set_error(CG_E_STATE, "not allowed while serving");
  if (!c || !req || !rep_dev) return set_error(CG_E_ARG, "NULL argument");
  Prepared P;
  CG_TRY(prepare3d(c, *req, &P));
  CG_TRY(enqueue3d(c, P, rep_dev, static_cast<cudaStream_t>(stream)));
  c->stats.checks++;
  c->stats.bytes_checked += P.ri.n;
  return CG_OK;
}

}  // extern "C"

// cg_noalloc.cu -- cg_scan_noalloc: the single-copy scan for callers that
// must not allocate device memory.
//
// Why it exists: a checker that sits inside a program's own allocation and
// copy calls -- for example an interposer that wraps the driver's memory
// functions the way the paper's wrappers do -- cannot itself call
// cudaMalloc: it would re-enter the allocator it is wrapping, or take memory
// from a budget that another allocator (a framework's caching allocator)
// owns completely.  cg_create allocates (the allocation table's shadow
// pool, pinned staging, scratch), so such callers cannot use a context.
// This entry point allocates nothing: the caller passes every buffer, and
// the kernel's scratch (its accumulators and a staging area for
// overlapping device->device copies) lives in a fixed array compiled into
// the library.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "cg_internal.h"
#include "cg_launch.h"

namespace cgi {

// Scratch of the allocation-free scan: one SingleScratch (the
// accumulators and the count of finished CTAs, reset by the kernel's last
// CTA) followed by the staging area.  Every GPU that loads this library
// holds it until the process exits.
constexpr uint64_t kNoAllocHead = 256;
constexpr uint64_t kNoAllocStageMax = 8ull << 20;  // largest overlapping DtoD carry
constexpr uint64_t kNoAllocBytes = kNoAllocHead + kNoAllocStageMax;
static_assert(sizeof(SingleScratch) <= kNoAllocHead, "scratch head too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host-side address of g_noalloc_scratch on each device (the symbol itself
// is only a host-side stand-in), plus the device's SM count.
constexpr int kMaxDevices = 64;
static unsigned char *g_scratch_addr[kMaxDevices];
static int g_sm_count[kMaxDevices];
static std::once_flag g_once[kMaxDevices];
static cudaError_t g_setup_err[kMaxDevices];

static void setup_device(int dev) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  } else {
    cudaGetLastError();
  }
  g_setup_err[dev] = e;
}

}  // namespace cgi

using namespace cgi;

static cg_status fail(cg_status st, const std::string &msg) {
  set_error_text(msg.c_str());  // read back with cg_last_error()
  return st;
}

extern "C" cg_status cg_scan_noalloc(uint32_t kind, const uint8_t *a_bits_dev, uint8_t *host_v_dev,
                                     uint64_t host_n, uint64_t host_off,
                                     const uint8_t *dev_src_shadow, uint8_t *dev_dst_shadow,
                                     uint64_t n, uint32_t carry, cg_report *rep_dev,
                                     void *stream) {
  if (kind != CG_HTOD && kind != CG_DTOH && kind != CG_DTOD)
    return fail(CG_E_KIND, "kind must be CG_HTOD, CG_DTOH or CG_DTOD");
  if (!rep_dev) return fail(CG_E_ARG, "rep_dev is NULL");
  if (kind != CG_DTOD) {
    if (!a_bits_dev || !host_v_dev) return fail(CG_E_ARG, "host image pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(a_bits_dev) | reinterpret_cast<uintptr_t>(host_v_dev)) & 15)
      return fail(CG_E_ALIGN, "host image arrays must be 16-byte aligned");
    if (host_n % 128) return fail(CG_E_ALIGN, "host image size must be a multiple of 128");
    if (host_off > host_n || n > host_n - host_off)
      return fail(CG_E_HOST_RANGE, "host range outside the host image");
    for (const void *p : {static_cast<const void *>(a_bits_dev), static_cast<const void *>(host_v_dev)}) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(CG_E_ARG, "host image pointer unknown to CUDA");
      }
      if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(CG_E_ARG, "the host image must be in device memory for cg_scan_noalloc");
    }
  }
  // the device shadows feed the bulk copies, which read device memory only
  for (const void *p : {static_cast<const void *>(kind != CG_HTOD ? dev_src_shadow : nullptr),
                        static_cast<const void *>(kind != CG_DTOH ? dev_dst_shadow : nullptr)}) {
    if (!p) continue;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return fail(CG_E_ARG, "device shadow pointer unknown to CUDA");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return fail(CG_E_ARG, "device shadows must be in device memory for cg_scan_noalloc");
  }
  const bool has_src = kind != CG_HTOD && dev_src_shadow != nullptr;
  const bool has_dst = kind != CG_DTOH && dev_dst_shadow != nullptr;
  const bool do_carry = carry != 0 && (kind == CG_HTOD   ? has_dst
                                       : kind == CG_DTOH ? has_src
                                                         : has_src && has_dst);
  bool overlap = false;
  if (kind == CG_DTOD && has_src && has_dst) {
    const uintptr_t s = reinterpret_cast<uintptr_t>(dev_src_shadow);
    const uintptr_t d = reinterpret_cast<uintptr_t>(dev_dst_shadow);
    overlap = (s <= d ? d - s : s - d) < n;
  }
  if (overlap && do_carry && n > kNoAllocStageMax)
    return fail(CG_E_TOO_BIG, "overlapping device->device carry larger than the 8 MiB "
                              "staging area of cg_scan_noalloc");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CG_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CG_E_ARG, "device index above 63");
  std::call_once(g_once[dev], setup_device, dev);
  if (g_setup_err[dev] != cudaSuccess)
    return fail(CG_E_CUDA, std::string("cudaGetSymbolAddress: ") +
                               cudaGetErrorString(g_setup_err[dev]));
  unsigned char *base = g_scratch_addr[dev];
  SingleScratch *scr = reinterpret_cast<SingleScratch *>(base);
  unsigned char *stage = base + kNoAllocHead;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  RangeInfo ri{};
  ri.kind = kind;
  ri.n = n;
  if (overlap) ri.flags |= CG_F_DTOD_OVERLAP;
  ScanJob job{};
  job.kind = kind;
  job.n = n;
  job.host_off = kind == CG_DTOD ? 0 : host_off;
  if (has_src) {
    job.mode |= kModeReadDev;
    job.dev_src = reinterpret_cast<uint64_t>(dev_src_shadow);
  }
  if (do_carry) {
    job.mode |= kModeCarry;
    if (kind != CG_DTOH) job.dev_dst = reinterpret_cast<uint64_t>(dev_dst_shadow);
  }
  Image img{a_bits_dev, host_v_dev, host_n};
  // the accumulators must start from zero (and the "no offset" marker):
  // a call that ended early may have left them dirty
  e = launch_init_single_scratch(scr, st);
  if (e == cudaSuccess && overlap && do_carry && n) {
    e = cudaMemcpyAsync(stage, dev_src_shadow, n, cudaMemcpyDeviceToDevice, st);
    job.dev_src = reinterpret_cast<uint64_t>(stage);
  }
  if (e == cudaSuccess) {
    if (n == 0 || (kind == CG_DTOD && !(job.mode & (kModeCarry | kModeReadDev)))) {
      job.mode = 0;  // no chunks: the kernel only writes the report
      job.kind = CG_DTOD;
    }
    e = launch_scan_single_tma(img, job, ri, scr, rep_dev, scan_single_tma_grid(g_sm_count[dev], n),
                               st);
  }
  if (e != cudaSuccess) return fail(CG_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return CG_OK;
}
